"""The stall stop test (pimpc_set_stall) on FP32 iterations (needs a GB300).

With eps below what FP32 iterations can reach, Algorithm 1's stop test alone would run every
instance to max_iters; the stall test ends each instance once its residual c has levelled off at
the FP32 floor, with status PIMPC_STALLED, and the result must then match the converged FP64
oracle to the FP32 parity tolerance (1e-4 on u and x, relative to max(1, |w*|)). With the
window 0 (off) the solve is that of Algorithm 1: same iterations as without the call.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import pimpc
from test_gpu_parity import ragged_batch, solution_error

pytestmark = pytest.mark.gpu


def test_stall_ends_fp32_solves_at_the_floor_with_accurate_results():
    insts = ragged_batch(5)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=1e-14, max_iters=20000, accel=1)
    pimpc.pimpc_set_stall(s.h, 200, 0.5)
    r = s.solve()
    ora = oracle.solve_batch(insts, eps=1e-22, max_iters=60000, accel=1)
    st = np.asarray(r["status"])
    assert np.all((st == pimpc.STALLED) | (st == pimpc.CONVERGED)), st
    assert np.any(st == pimpc.STALLED)
    assert np.all(np.asarray(r["iters"]) < 20000)
    for j, o in enumerate(ora):
        assert solution_error(r["u"][j], r["x"][j], o["u"], o["x"]) <= 1e-4, j
    # window 0: Algorithm 1's stop test only, as on a solver that never enabled the test
    pimpc.pimpc_set_stall(s.h, 0, 0.5)
    pimpc.pimpc_set_options(s.h, 1.0, 1e-14, 3000, 1, 0.999)
    r0 = s.solve()
    s2 = pimpc.Solver(insts, precision=pimpc.F32, eps=1e-14, max_iters=3000, accel=1)
    r1 = s2.solve()
    np.testing.assert_array_equal(r0["iters"], r1["iters"])
    for a, b in zip(r0["u"], r1["u"]):
        np.testing.assert_array_equal(a, b)
    with pytest.raises(pimpc.PimpcError):
        pimpc.pimpc_set_stall(s.h, -1, 0.5)
    with pytest.raises(pimpc.PimpcError):
        pimpc.pimpc_set_stall(s.h, 10, 1.5)
    s.close()
    s2.close()
