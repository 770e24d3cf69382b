"""Failure paths of the solve that can be made without faulting a GPU (needs a GB300).

* A bounded wait that runs out: the grid barrier of the persistent launch is limited to one poll
  (pimpc_set_wait_limit), so CTAs that reach it before the last one give up. The launch must end
  (no hang), report every unfinished instance as PIMPC_TIMEOUT, and leave the context usable: the
  next solve with the default limit gives the same results as a solver that never timed out.
  Only the grid barrier is shortened; every CTA has finished its copies when it reaches it.
* A failed factorisation: dynamics with a NaN make a pivot of the FP64 Cholesky NaN, and the
  next solve reports that instance (and only that one) as PIMPC_FACTOR_FAILED.
"""
import numpy as np
import pytest

from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def uneven_batch(seed, count):
    rng = np.random.default_rng(seed)
    return [W.random_ltv(seed * 1000 + i, int(rng.integers(4, 17)), int(rng.integers(2, 7)),
                         int(rng.integers(20, 200))) for i in range(count)]


@pytest.mark.parametrize("precision", [pimpc.F32, pimpc.F64])
def test_grid_barrier_timeout_reports_timeout_and_recovers(precision):
    insts = uneven_batch(7, 96)
    s = pimpc.Solver(insts, precision=precision, eps=1e-6, max_iters=400, accel=1)
    pimpc.pimpc_set_wait_limit(s.h, 1)
    r = s.solve()
    st = np.asarray(r["status"])
    assert np.all(st == pimpc.TIMEOUT), np.bincount(st)
    assert np.all(np.asarray(r["iters"]) < 400)
    pimpc.pimpc_set_wait_limit(s.h, 0)
    r2 = s.solve()
    ref = pimpc.Solver(insts, precision=precision, eps=1e-6, max_iters=400, accel=1)
    r3 = ref.solve()
    assert np.all(np.asarray(r2["status"]) != pimpc.TIMEOUT)
    np.testing.assert_array_equal(r2["iters"], r3["iters"])
    for a, b in zip(r2["u"], r3["u"]):
        np.testing.assert_array_equal(a, b)
    with pytest.raises(pimpc.PimpcError) as e:
        pimpc.pimpc_set_wait_limit(s.h, -1)
    assert e.value.code == pimpc.EINVAL
    s.close()
    ref.close()


@pytest.mark.parametrize("precision", [pimpc.F32, pimpc.F64])
def test_nan_dynamics_report_a_failed_factorisation(precision):
    insts = uneven_batch(8, 5)
    insts[2]["A"] = insts[2]["A"].copy()
    insts[2]["A"][3, 0, 0] = np.nan
    s = pimpc.Solver(insts, precision=precision, eps=1e-6, max_iters=2000, accel=1)
    r = s.solve()
    st = np.asarray(r["status"])
    assert st[2] == pimpc.FACTOR_FAILED
    assert np.all(st[[0, 1, 3, 4]] == pimpc.CONVERGED)
    # valid dynamics clear the flag at the next factorisation
    good = uneven_batch(8, 5)
    pimpc.pimpc_set_dynamics(s.h, *[pimpc.pack(good)[k] for k in ("A", "B", "e")])
    r = s.solve()
    assert np.all(np.asarray(r["status"]) == pimpc.CONVERGED)
    s.close()
