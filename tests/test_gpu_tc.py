"""Tensor-core schedule (family 6) against the oracle (needs a GB300).

Stage-invariant instances with FP32 iterations: the per-stage products of 127-stage tiles run
as tcgen05 matrix products with TF32 operands split into hi/lo pairs (three MMAs per K step).
Tolerances of the other FP32 tests: at a fixed iteration count of the plain iteration (or with
the oracle's restart decisions replayed) 1e-4 on (u, x) against the FP64 oracle, and the
converged FP32 solution within 1e-5 (relative to max(1, |w*|)) of the converged oracle. Sizes
cover the large-state shape (nx 48, nu 16: no padding), padded shapes (nx 12, nu 4; nx 20, nu 5),
horizons that are a multiple of the tile, one more, one less, a single stage, and several
tiles per work item.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W
from test_gpu_parity import relerr, solution_error

pytestmark = pytest.mark.gpu


def lti_batch(seed, shapes):
    out = []
    for i, (nx, nu, N) in enumerate(shapes):
        inst = W.large_lti(seed=seed * 10 + i, batch=1, nx=nx, nu=nu, N=N, umax=0.08)[0]
        inst["ref"] = np.linspace(-0.3, 0.3, nx + nu)  # a nonzero constant reference
        out.append(inst)
    return out


SHAPES = [(48, 16, 300), (48, 16, 127), (48, 16, 128), (48, 16, 254), (48, 16, 1),
          (12, 4, 200), (20, 5, 131)]


@pytest.mark.parametrize("item_scale", [0, 1, 3])
def test_tc_plain_fixed_iterations_match_oracle(item_scale):
    insts = lti_batch(1, SHAPES)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=150, accel=0)
    s.set_schedule(6, 0, item_scale)
    assert s.schedule()["family"] == 6
    r = s.solve()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=150, accel=0)
    for j, o in enumerate(ora):
        assert relerr(r["u"][j], o["u"]) <= 1e-4, j
        assert relerr(r["x"][j], o["x"]) <= 1e-4, j
    s.close()


def test_tc_accelerated_with_replayed_restarts_matches_oracle():
    insts = lti_batch(2, SHAPES[:4])
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=120, accel=1, history=True)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=120, accel=1)
    s.set_schedule(6)
    mask = np.stack([o["mask"] for o in ora]).astype(np.uint8)
    pimpc.pimpc_set_restart_mask(s.h, mask, 120)
    r = s.solve()
    for j, o in enumerate(ora):
        assert relerr(r["u"][j], o["u"]) <= 1e-4, j
        assert relerr(r["x"][j], o["x"]) <= 1e-4, j
    s.close()


def test_tc_agrees_with_the_blocked_schedule_and_converges():
    insts = lti_batch(3, [(48, 16, 200), (20, 5, 90)])
    res = {}
    for fam in (5, 6):
        s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=100, accel=0)
        s.set_schedule(fam)
        res[fam] = s.solve()
        s.close()
    for j in range(len(insts)):
        assert relerr(res[6]["u"][j], res[5]["u"][j]) <= 1e-4
        assert relerr(res[6]["x"][j], res[5]["x"][j]) <= 1e-4
    # Converged: on well-conditioned instances (Q = I, R = 0.1 I) the FP32 solve stopped by the
    # stall test is within 1e-5 of the converged oracle.
    conv = lti_batch(6, [(48, 16, 60), (20, 5, 90)])
    for inst in conv:
        inst["q"], inst["r"] = np.ones(inst["nx"]), 0.1 * np.ones(inst["nu"])
    ora = oracle.solve_batch(conv, eps=1e-22, max_iters=100000, accel=1)
    s = pimpc.Solver(conv, precision=pimpc.F32, eps=1e-14, max_iters=30000, accel=1)
    s.set_schedule(6)
    pimpc.pimpc_set_stall(s.h, 100, 0.5, 1e-9, 0.3)
    r = s.solve()
    for j, o in enumerate(ora):
        assert solution_error(r["u"][j], r["x"][j], o["u"], o["x"]) <= 1e-5, j
    s.close()


def test_tc_rejects_what_it_does_not_serve():
    ltv = [W.random_ltv(7, 6, 2, 30)]
    s = pimpc.Solver(ltv, precision=pimpc.F32)
    with pytest.raises(pimpc.PimpcError):
        s.set_schedule(6)   # stage-varying dynamics
    s.close()
    big = lti_batch(4, [(52, 8, 20)])  # 64 + 16 > 64 once padded
    s = pimpc.Solver(big, precision=pimpc.F32)
    with pytest.raises(pimpc.PimpcError):
        s.set_schedule(6)
    s.close()
    s = pimpc.Solver(lti_batch(5, [(12, 4, 20)]), precision=pimpc.F64)
    with pytest.raises(pimpc.PimpcError):
        s.set_schedule(6)   # FP64 iterations
    s.close()
