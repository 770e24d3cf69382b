"""Non-box input sets on the GPU against the oracle (needs a GB300).

The remark after Theorem 1: with U an l2 ball, an l1 ball, a halfspace or a second-order cone the
z-update is still a Euclidean projection, and the kernels project the input part of w onto U
with lane-group reductions. Tolerances as for the box: FP64 iterations match the oracle at a
fixed iteration count to 1e-10 on every iterate (plain and accelerated), FP32 plain iterations
to 1e-4 on (u, x); the FP64 polish of an FP32 solve reaches the converged oracle to 1e-5. Every
batch mixes the set kinds (and boxes) across instances; the sizes cover lane groups of 4, 8 and
16 lanes in the blocked family, groups of 8, 16 and 32 lanes in the plain family, and an
instance with n > 32 whose inputs straddle the two component slots of a lane.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W
from test_gpu_parity import check_iterates, relerr, solution_error

pytestmark = pytest.mark.gpu

DIMS = [(4, 2, 37), (14, 2, 19), (24, 8, 11), (6, 3, 70), (9, 5, 17), (12, 4, 33), (3, 3, 9),
        (20, 7, 45), (5, 4, 26), (8, 6, 40)]


def uset_for(i, nu, rng):
    kind = i % 5
    if kind == 0:
        return None
    if kind == 1:
        return dict(kind=pimpc.USET_BALL2, r=0.6)
    if kind == 2:
        return dict(kind=pimpc.USET_BALL1, r=0.8)
    if kind == 3:
        return dict(kind=pimpc.USET_HALFSPACE, r=0.2, a=rng.standard_normal(nu))
    return dict(kind=pimpc.USET_SOC, r=0.0)


def set_batch(seed, dims=DIMS, lti=False):
    rng = np.random.default_rng(seed)
    out = []
    for i, (nx, nu, N) in enumerate(dims):
        inst = (W.random_ltv(seed * 100 + i, nx, nu, N) if not lti else
                W.large_lti(seed=seed * 100 + i, batch=1, nx=nx, nu=nu, N=N)[0])
        us = uset_for(i + seed, nu, rng)
        if us is not None:
            inst["uset"] = us
            inst["umin"], inst["umax"] = -np.inf * np.ones(nu), np.inf * np.ones(nu)
        out.append(inst)
    return out


@pytest.mark.parametrize("family", [pimpc.FAMILY_LANES, pimpc.FAMILY_BLOCKED])
@pytest.mark.parametrize("accel", [0, 1])
def test_fp64_fixed_iterations_with_input_sets_match_oracle(family, accel):
    insts = set_batch(1)
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=200, accel=accel)
    s.set_schedule(family)
    s.solve()
    its = s.iterates()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=200, accel=accel)
    for j, o in enumerate(ora):
        check_iterates(its[j], o, 1e-10)
    s.close()


@pytest.mark.parametrize("family", [pimpc.FAMILY_LANES, pimpc.FAMILY_BLOCKED])
def test_fp32_plain_iterations_with_input_sets_match_oracle(family):
    insts = set_batch(2)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=150, accel=0)
    s.set_schedule(family)
    r = s.solve()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=150, accel=0)
    moved = 0
    for j, o in enumerate(ora):
        assert relerr(r["u"][j], o["u"]) <= 1e-4, j
        assert relerr(r["x"][j], o["x"]) <= 1e-4, j
        if insts[j].get("uset") is not None:
            free = oracle.solve(dict(insts[j], uset=None), eps=-1.0, max_iters=150, accel=0)
            moved += np.max(np.abs(free["u"] - o["u"])) > 1e-3
    assert moved >= 5   # the sets are active


def test_stage_invariant_instance_with_inputs_across_lane_slots():
    # n = 36 > 32: a plain lane group of 32 lanes holds components c and c + 32 per lane, so the
    # inputs (c = 30..35) sit in two slots of different lanes.
    insts = set_batch(3, dims=[(30, 6, 40), (30, 6, 25), (28, 8, 30)], lti=True)
    insts[0]["uset"] = dict(kind=pimpc.USET_BALL1, r=0.05)
    insts[1]["uset"] = dict(kind=pimpc.USET_SOC, r=0.0)
    insts[2]["uset"] = dict(kind=pimpc.USET_HALFSPACE, r=0.0, a=np.linspace(-1, 1, 8))
    for i in insts:
        i["umin"], i["umax"] = -np.inf * np.ones(i["nu"]), np.inf * np.ones(i["nu"])
    for family in (pimpc.FAMILY_LANES, pimpc.FAMILY_BLOCKED):
        s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=120, accel=1)
        s.set_schedule(family)
        s.solve()
        its = s.iterates()
        ora = oracle.solve_batch(insts, eps=-1.0, max_iters=120, accel=1)
        for j, o in enumerate(ora):
            check_iterates(its[j], o, 1e-10)
        s.close()


def test_fp64_polish_with_input_sets_reaches_the_converged_oracle():
    insts = set_batch(4, dims=DIMS[:6])
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=1e-9, max_iters=20000, accel=1)
    s.set_polish(4000, 1e-20)
    r = s.solve()
    ora = oracle.solve_batch(insts, eps=1e-22, max_iters=100000, accel=1)
    for j, o in enumerate(ora):
        assert solution_error(r["u"][j], r["x"][j], o["u"], o["x"]) <= 1e-5, j
    s.close()


def test_input_sets_keep_to_the_families_that_project_them():
    insts = set_batch(5, dims=DIMS[:3])
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=50, accel=0)
    with pytest.raises(pimpc.PimpcError) as e:
        s.set_schedule(pimpc.FAMILY_RESIDENT)
    assert e.value.code == pimpc.EINVAL
    s.solve()
    with pytest.raises(pimpc.PimpcError) as e:
        s.backward([np.zeros((i["N"], i["nu"])) for i in insts],
                   [np.zeros((i["N"], i["nx"])) for i in insts])
    assert e.value.code == pimpc.ESTATE
    res = pimpc.pimpc_autotune(s.h, 5)
    assert s.schedule()["family"] in (pimpc.FAMILY_LANES, pimpc.FAMILY_BLOCKED), res
    with pytest.raises(pimpc.PimpcError):
        pimpc.pimpc_set_input_set(s.h, np.array([7, 0, 0]), np.zeros(3))
    s.close()
