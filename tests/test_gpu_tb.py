"""Temporal blocking of the plain iteration (schedule family 7) against the oracle (needs a GB300).

Windows of stages are iterated T times in shared memory with T halo stages on each open side;
after T iterations the interior equals T iterations of Algorithm 1 on the whole horizon. So at a
fixed iteration count the iterates match the oracle's plain iteration to 1e-10 in FP64 (every
iterate) and 1e-4 in FP32 (u, x), with instances split into several windows (long horizons,
large n), windows that are whole horizons, iteration counts that are and are not multiples of T,
and T = 1, 4, 5, 6 (FP64) and 8, 12 (FP32). With eps >= 0 the stop test runs every T iterations: an instance stops at
the first multiple of T (or max_iters) where c <= eps, with the oracle's iterate at that count.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W
from test_gpu_parity import check_iterates, relerr

pytestmark = pytest.mark.gpu

DIMS = [(24, 8, 300), (14, 2, 190), (4, 2, 37), (9, 5, 500), (6, 3, 1), (20, 7, 64)]


def batch(seed, dims=DIMS):
    return [W.random_ltv(seed * 100 + i, nx, nu, N) for i, (nx, nu, N) in enumerate(dims)]


# FP64 windows of the widest instance (n 32) hold 15 stages: T up to 7
@pytest.mark.parametrize("T,iters", [(4, 200), (6, 123), (1, 40)])
def test_tb_fp64_fixed_iterations_match_oracle(T, iters):
    insts = batch(1)
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=iters, accel=0)
    s.set_schedule(7, 0, T)
    sch = s.schedule()
    assert sch["family"] == 7 and sch["items"] > len(insts)  # some instances span windows
    r = s.solve()
    assert np.all(np.asarray(r["iters"]) == iters)
    its = s.iterates()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=iters, accel=0)
    for j, o in enumerate(ora):
        check_iterates(its[j], o, 1e-10)
    s.close()


@pytest.mark.parametrize("T", [0, 12])
def test_tb_fp32_fixed_iterations_match_oracle(T):
    insts = batch(2)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=150, accel=0)
    s.set_schedule(7, 0, T)  # 0: the default T = 8
    r = s.solve()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=150, accel=0)
    for j, o in enumerate(ora):
        assert relerr(r["u"][j], o["u"]) <= 1e-4, j
        assert relerr(r["x"][j], o["x"]) <= 1e-4, j
    s.close()


def test_tb_stops_at_the_first_checked_multiple_of_T():
    insts = batch(3, DIMS[:4])
    T = 5
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=1e-6, max_iters=5000, accel=0)
    s.set_schedule(7, 0, T)
    r = s.solve()
    its = s.iterates()
    ref = oracle.solve_batch(insts, eps=1e-6, max_iters=5000, accel=0)
    for j, o in enumerate(ref):
        want = -(-o["iters"] // T) * T  # the oracle's count rounded up to a multiple of T
        assert r["iters"][j] == want and r["status"][j] == pimpc.CONVERGED, j
        same = oracle.solve(insts[j], eps=-1.0, max_iters=want, accel=0)
        check_iterates(its[j], same, 1e-10)
    s.close()


def test_tb_runs_the_plain_iteration_only():
    s = pimpc.Solver(batch(4, DIMS[:2]), precision=pimpc.F32, eps=-1.0, max_iters=20, accel=1)
    s.set_schedule(7)
    with pytest.raises(pimpc.PimpcError) as e:
        s.solve()
    assert e.value.code == pimpc.ESTATE
    s.close()


def test_tb_windows_at_the_full_shared_memory_budget():
    # Every state size of the batched workload with inputs 2, 5 and 8: the widest windows of the
    # wide instances fill the shared memory of a CTA next to the kernel's static shared memory.
    dims = [(nx, nu, 60) for nx in range(4, 25) for nu in (2, 5, 8)]
    insts = batch(8, dims)
    for T in (4, 8):
        s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=2 * T + 1, accel=0)
        s.set_schedule(7, 0, T)
        r = s.solve()
        ora = oracle.solve_batch(insts, eps=-1.0, max_iters=2 * T + 1, accel=0)
        for j, o in enumerate(ora):
            assert relerr(r["u"][j], o["u"]) <= 1e-4, (T, j)
            assert relerr(r["x"][j], o["x"]) <= 1e-4, (T, j)
        s.close()
