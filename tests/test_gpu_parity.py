"""CUDA path vs the FP64 oracle, element by element, through the C ABI (needs a GB300).

Tolerances: FP64 iterations match the oracle at a fixed iteration count to a normwise relative
error of 1e-10 on every iterate; FP32 iterations to 1e-4 on (u, x); converged FP32 solutions
match the converged oracle to 1e-5. Restart decisions are discrete, so fixed-count FP32 tests of
the accelerated mode replay the oracle's decisions (pimpc_set_restart_mask); FP64 tests take
their own decisions.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W

pytestmark = pytest.mark.gpu

KEYS = ("z", "v", "th", "be", "la")


def relerr(a, b):
    a = np.asarray(a, np.float64)
    b = np.asarray(b, np.float64)
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-12))


def solution_error(u, x, u_ref, x_ref):
    """max |w - w*| / max(1, max |w*|) over w = (u, x): the accuracy measure of the benchmark."""
    w = np.concatenate([np.ravel(u), np.ravel(x)])
    ws = np.concatenate([np.ravel(u_ref), np.ravel(x_ref)])
    return float(np.max(np.abs(w - ws)) / max(1.0, np.max(np.abs(ws))))


# (nx, nu, N): lane groups of 8, 16 and 32, ragged last chunks, N = 1, and several chunks.
RAGGED = [(4, 2, 37), (14, 2, 19), (24, 8, 11), (3, 1, 70), (6, 2, 1), (12, 4, 33), (5, 3, 9),
          (20, 7, 45), (9, 9, 17)]


def ragged_batch(seed=0, dims=RAGGED, **kw):
    return [W.random_ltv(seed * 1000 + i, nx, nu, N, **kw) for i, (nx, nu, N) in enumerate(dims)]


def oracle_runs(insts, **opts):
    return oracle.solve_batch(insts, **opts)


def check_iterates(gpu_its, ora, tol):
    for key in KEYS:
        assert relerr(gpu_its[key], ora[key]) <= tol, key


@pytest.mark.parametrize("accel", [0, 1])
def test_fp64_fixed_iterations_match_oracle(accel):
    insts = ragged_batch(1)
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=200, accel=accel)
    res = s.solve()
    its = s.iterates()
    ora = oracle_runs(insts, eps=-1.0, max_iters=200, accel=accel)
    for j, o in enumerate(ora):
        check_iterates(its[j], o, 1e-10)
        assert relerr(res["u"][j], o["u"]) <= 1e-10
        assert relerr(res["x"][j], o["x"]) <= 1e-10
        assert res["iters"][j] == 200 and res["status"][j] == pimpc.MAXITER
        # c is a sum of squared changes; once an instance has converged it is rounding noise
        assert abs(res["c"][j] - o["c"]) <= 1e-8 * o["c"] + 1e-24


def test_fp32_plain_fixed_iterations_match_oracle():
    insts = ragged_batch(2)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=200, accel=0)
    res = s.solve()
    ora = oracle_runs(insts, eps=-1.0, max_iters=200, accel=0)
    for j, o in enumerate(ora):
        assert relerr(res["u"][j], o["u"]) <= 1e-4
        assert relerr(res["x"][j], o["x"]) <= 1e-4


def test_fp32_accel_with_replayed_restarts_matches_oracle():
    insts = ragged_batch(3)
    K = 200
    ora = [oracle.solve(i, eps=-1.0, max_iters=K, accel=1, history=True) for i in insts]
    mask = np.ascontiguousarray(np.stack([o["mask"] for o in ora]).astype(np.uint8))
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=K, accel=1)
    pimpc.pimpc_set_restart_mask(s.h, mask, K)
    res = s.solve()
    for j, o in enumerate(ora):
        assert relerr(res["u"][j], o["u"]) <= 1e-4
        assert relerr(res["x"][j], o["x"]) <= 1e-4


def test_converged_fp32_matches_converged_oracle():
    insts = ragged_batch(4, dims=[(4, 2, 37), (14, 2, 19), (12, 4, 33), (6, 2, 1), (9, 9, 17)])
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=1e-11, max_iters=20000, accel=1)
    res = s.solve()
    ora = oracle_runs(insts, eps=1e-22, max_iters=200000, accel=1)
    for j, o in enumerate(ora):
        assert o["status"] == oracle.CONVERGED
        assert solution_error(res["u"][j], res["x"][j], o["u"], o["x"]) <= 1e-5


def test_lti_up_to_n64_fp64():
    insts = [W.plain_lti(seed=s, nx=nx, nu=nu, N=N) for s, (nx, nu, N) in
             enumerate([(48, 16, 23), (4, 2, 20), (30, 10, 9), (40, 3, 1)])]
    for inst in insts:
        inst["e"] = np.random.default_rng(inst["nx"]).uniform(-0.3, 0.3, inst["nx"])
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=120, accel=1)
    s.solve()
    its = s.iterates()
    ora = oracle_runs(insts, eps=-1.0, max_iters=120, accel=1)
    for j, o in enumerate(ora):
        check_iterates(its[j], o, 1e-10)


def test_lti_fp32_plain():
    insts = [W.plain_lti(seed=7, nx=48, nu=16, N=40), W.plain_lti(seed=8)]
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=150, accel=0)
    res = s.solve()
    ora = oracle_runs(insts, eps=-1.0, max_iters=150, accel=0)
    for j, o in enumerate(ora):
        assert relerr(res["u"][j], o["u"]) <= 1e-4
        assert relerr(res["x"][j], o["x"]) <= 1e-4


def test_plain_lti_single_instance():
    inst = W.plain_lti(seed=1)
    for prec, tol in ((pimpc.F64, 1e-10), (pimpc.F32, 1e-4)):
        s = pimpc.Solver([inst], precision=prec, eps=-1.0, max_iters=200, accel=0)
        res = s.solve()
        o = oracle.solve(inst, eps=-1.0, max_iters=200, accel=0)
        assert relerr(res["u"][0], o["u"]) <= tol
        assert relerr(res["x"][0], o["x"]) <= tol


@pytest.mark.parametrize("mode", [1, 2])
def test_warm_start_matches_oracle(mode):
    insts = ragged_batch(5, dims=[(4, 2, 37), (14, 2, 19), (24, 8, 11)])
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=60, accel=1)
    s.solve()
    first = [oracle.solve(i, eps=-1.0, max_iters=60, accel=1) for i in insts]
    s.solve(warm_start=mode)
    its = s.iterates()
    for j, (inst, f) in enumerate(zip(insts, first)):
        warm = {k: f[k].copy() for k in KEYS}
        if mode == 2:
            for k in KEYS:
                warm[k] = np.concatenate([f[k][1:], f[k][-1:]], axis=0)
        o = oracle.solve(inst, eps=-1.0, max_iters=60, accel=1, warm=warm)
        check_iterates(its[j], o, 1e-10)


def test_batch_invariance():
    insts = ragged_batch(6)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=80, accel=1)
    res = s.solve()
    for j in (0, 2, 5):
        one = pimpc.Solver([insts[j]], precision=pimpc.F32, eps=-1.0, max_iters=80, accel=1)
        r1 = one.solve()
        assert np.array_equal(r1["u"][0], res["u"][j]) and np.array_equal(r1["x"][0], res["x"][j])


def test_status_codes_and_iteration_counts():
    insts = ragged_batch(7, dims=[(4, 2, 12), (6, 2, 9)])
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=1e-6, max_iters=5000, accel=1)
    res = s.solve()
    ora = oracle_runs(insts, eps=1e-6, max_iters=5000, accel=1)
    for j, o in enumerate(ora):
        assert res["status"][j] == pimpc.CONVERGED
        assert res["iters"][j] == o["iters"]
    s.set_options(eps=1e-30, max_iters=7, accel=1)
    res = s.solve()
    assert np.all(res["status"] == pimpc.MAXITER) and np.all(res["iters"] == 7)
    x0 = s.p["x0"].copy()
    x0[0] = np.nan
    res = s.solve(x0=x0)
    assert res["status"][0] == pimpc.NONFINITE
    assert res["status"][1] == pimpc.MAXITER


def test_invalid_arguments_are_rejected():
    s = pimpc.Solver(ragged_batch(8, dims=[(4, 2, 5)]), precision=pimpc.F32)
    with pytest.raises(pimpc.PimpcError) as e:
        pimpc.pimpc_set_bounds(s.h, np.array([1.0] * 4), np.array([0.0] * 4), -np.ones(2), np.ones(2))
    assert e.value.code == pimpc.EINVAL
    with pytest.raises(pimpc.PimpcError) as e:
        pimpc.pimpc_set_options(s.h, -1.0, 1e-6, 10, 1)
    assert e.value.code == pimpc.EINVAL


@pytest.mark.parametrize("model,params,lti", [
    (W.MODEL_QUADROTOR, W.QUAD_PARAMS, 0),
    (W.MODEL_CARTPOLE, W.CARTPOLE_PARAMS, 0),
    (W.MODEL_CARTPOLE, W.CARTPOLE_PARAMS, 1),
    (W.MODEL_CSTR, np.append(W.CSTR_PARAMS, 298.15), 0),
])
def test_linearise_matches_oracle(model, params, lti):
    nx, nu = oracle.model_dims(model)
    rng = np.random.default_rng(model)
    Ns = [7, 1, 13]
    P = len(params)
    prm = np.ascontiguousarray(np.tile(params, len(Ns)))
    h = pimpc.pimpc_create([nx] * 3, [nu] * 3, Ns, lti, pimpc.F64)
    try:
        pts = [1 if lti else N for N in Ns]
        if model == W.MODEL_CSTR:
            xb = [np.column_stack([rng.uniform(2, 9, p), rng.uniform(300, 360, p)]) for p in pts]
            ub = [rng.uniform(280, 320, (p, nu)) for p in pts]
        else:
            xb = [rng.uniform(-0.5, 0.5, (p, nx)) for p in pts]
            ub = [rng.uniform(0.5, 3.0, (p, nu)) for p in pts]
        pimpc.pimpc_linearise(h, model, prm, 0.02, np.concatenate([a.ravel() for a in xb]),
                              np.concatenate([a.ravel() for a in ub]))
        nA = sum(p * nx * nx for p in pts)
        A = np.zeros(nA); B = np.zeros(sum(p * nx * nu for p in pts)); e = np.zeros(sum(p * nx for p in pts))
        pimpc.pimpc_get_dynamics(h, A, B, e)
        oA, oB, oe = [], [], []
        for j in range(3):
            a, b, c = oracle.linearise(model, params, 0.02, xb[j], ub[j])
            oA.append(a.ravel()); oB.append(b.ravel()); oe.append(c.ravel())
        for got, want in ((A, np.concatenate(oA)), (B, np.concatenate(oB)), (e, np.concatenate(oe))):
            np.testing.assert_allclose(got, want, rtol=1e-12, atol=1e-12 * max(1.0, np.abs(want).max()))
    finally:
        pimpc.pimpc_destroy(h)


def test_plant_step_matches_oracle():
    h = pimpc.pimpc_create([12, 12], [4, 4], [3, 3], 0, pimpc.F64)
    try:
        rng = np.random.default_rng(0)
        x = rng.uniform(-0.5, 0.5, 24)
        u = rng.uniform(0, 4, 8)
        prm = np.tile(W.QUAD_PARAMS, 2)
        xn = np.zeros(24)
        pimpc.pimpc_plant_step(h, W.MODEL_QUADROTOR, prm, 0.02, x, u, xn)
        for j in range(2):
            want = oracle.plant_step(0, W.QUAD_PARAMS, 0.02, x[12 * j:12 * j + 12], u[4 * j:4 * j + 4])
            np.testing.assert_allclose(xn[12 * j:12 * j + 12], want, rtol=1e-13, atol=1e-14)
    finally:
        pimpc.pimpc_destroy(h)


def test_device_memory_calls_match_host_calls():
    import torch
    insts = ragged_batch(9, dims=[(4, 2, 13), (14, 2, 19)])
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=50, accel=1)
    host = s.solve()
    dev = {k: torch.from_numpy(np.asarray(s.p[k])).cuda() for k in ("x0", "ref")}
    tot_u = int(np.sum(s.N * s.nu)); tot_x = int(np.sum(s.N * s.nx))
    u = torch.zeros(tot_u, dtype=torch.float64, device="cuda")
    x = torch.zeros(tot_x, dtype=torch.float64, device="cuda")
    it = torch.zeros(2, dtype=torch.int32, device="cuda")
    pimpc.pimpc_solve(s.h, dev["x0"], None, dev["ref"], s.p["ref_per_stage"], 0, u, x, it)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(u.cpu().numpy(), np.concatenate([a.ravel() for a in host["u"]]))
    np.testing.assert_array_equal(x.cpu().numpy(), np.concatenate([a.ravel() for a in host["x"]]))
    assert it.cpu().numpy().tolist() == [50, 50]


# ---- FP64 polish of FP32 solves -------------------------------------------------------------

POLISH_DIMS = [(4, 2, 37), (14, 2, 19), (12, 4, 33), (6, 2, 1), (9, 9, 17), (24, 8, 45)]


@pytest.mark.parametrize("family", [pimpc.FAMILY_LANES, pimpc.FAMILY_TILES, pimpc.FAMILY_BLOCKED])
def test_fp64_polish_reaches_the_fp64_solution(family):
    """FP32 iterations to eps = 1e-8, then FP64 iterations to 1e-22: the result must match the
    converged FP64 oracle to 1e-9, far below what FP32 iterations alone reach (about 1e-6)."""
    insts = ragged_batch(31, dims=POLISH_DIMS)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=1e-8, max_iters=20000, accel=1)
    if family != pimpc.FAMILY_LANES:
        s.set_schedule(family)
    plain = s.solve()
    s.set_polish(200000, 1e-22)
    res = s.solve()
    ora = oracle_runs(insts, eps=1e-22, max_iters=200000, accel=1)
    for j, o in enumerate(ora):
        assert o["status"] == oracle.CONVERGED
        assert res["status"][j] == pimpc.CONVERGED and res["c"][j] <= 1e-22
        assert res["iters"][j] > plain["iters"][j]        # FP32 iterations + polish iterations
        assert solution_error(res["u"][j], res["x"][j], o["u"], o["x"]) <= 1e-9, j


def test_polish_is_ignored_by_fp64_solvers_and_refused_by_the_adjoint():
    insts = ragged_batch(32, dims=POLISH_DIMS[:2])
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=50, accel=0)
    a = s.solve()
    s.set_polish(100, 1e-20)
    b = s.solve()
    for j in range(len(insts)):
        assert np.array_equal(a["u"][j], b["u"][j]) and b["iters"][j] == 50
    f = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=50, accel=0)
    f.set_polish(10, -1.0)
    r = f.solve()
    assert all(it == 60 for it in r["iters"])
    gu = [np.ones((i["N"], i["nu"])) for i in insts]
    gx = [np.ones((i["N"], i["nx"])) for i in insts]
    with pytest.raises(pimpc.PimpcError) as e:
        f.backward(gu, gx)
    assert e.value.code == pimpc.ESTATE
    with pytest.raises(pimpc.PimpcError) as e:
        f.set_polish(-1)
    assert e.value.code == pimpc.EINVAL
