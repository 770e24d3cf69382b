"""Input bound of the large-state LTI workload (workloads.large_lti), computed with the oracle.

The workload asks for box bounds that are active on about a fifth of the stages. This script
solves the first instances of the seeded workload with the input bound removed (|x| <= 5 kept),
takes |u| over all stages and inputs of the converged oracle solutions, and prints the 80th
percentile: with that bound, about 20 % of the unconstrained input values would exceed it.
It calls the oracle only; the value is stored in workloads.LARGE_LTI_UMAX.

    python tests/golden/calibrate_large_lti.py [instances]
"""
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import oracle  # noqa: E402
from paper_2601_14414_gb300 import workloads as W  # noqa: E402


def main(count=2):
    insts = W.large_lti(batch=count, umax=np.inf)
    mags = []
    for inst in insts:
        r = oracle.solve(inst, eps=1e-10, max_iters=20000, accel=1)
        print(f"instance: {r['iters']} iterations, status {r['status']}, c {r['c']:.2e}", flush=True)
        mags.append(np.abs(r["u"]).ravel())
    umax = float(np.percentile(np.concatenate(mags), 80))
    print(f"LARGE_LTI_UMAX = {umax:.6g}")
    return umax


if __name__ == "__main__":
    main(int(sys.argv[1]) if len(sys.argv) > 1 else 2)
