"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test checks the oracle against a fact that the paper or the mathematics fixes:
  * one oracle iteration == one generic scaled-form ADMM pass on the velocity-form splitting,
    built as explicit F, G, h (Theorem 2's problem) and solved by dense least squares and BVLS;
  * the converged iterate == the KKT point of the MPC QP found by brute-force active-set
    enumeration (tiny LTV), and == the equality-constrained closed form when no bound is active;
  * invariants: c non-increasing for plain ADMM (He & Yuan, Thm 4.1), z always in the box, fixed
    point at convergence, rho-independence of the optimum, u_prev-independence when W_du = 0,
    accelerated mode with eta = 0 reduces to the plain iteration;
  * a scalar case computed by hand.
"""
import numpy as np
import pytest

import oracle
import qp_reference as qp


def tiny_ltv(seed, nx=2, nu=1, N=3, xabs=2.0, uabs=0.5, rdu=False, ref_scale=0.0, x0_abs=2.5):
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((N, nx, nx)) * 0.6
    B = rng.standard_normal((N, nx, nu))
    e = rng.uniform(-0.2, 0.2, (N, nx))
    n = nx + nu
    return dict(nx=nx, nu=nu, N=N, lti=False, A=A, B=B, e=e,
                q=rng.uniform(0.5, 2.0, nx), r=rng.uniform(0.1, 1.0, nu),
                rdu=rng.uniform(0.05, 0.5, nu) if rdu else None,
                xmin=-xabs * np.ones(nx), xmax=xabs * np.ones(nx),
                umin=-uabs * np.ones(nu), umax=uabs * np.ones(nu),
                x0=rng.uniform(-x0_abs, x0_abs, nx),
                u_prev=rng.uniform(-uabs, uabs, nu),
                ref=ref_scale * rng.standard_normal((N, n)), rho=float(rng.uniform(0.5, 2.0)))


# ---------------------------------------------------------------------------------------------
# One iteration against the generic scaled ADMM on explicit F, G, h.
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed,rdu,hat_scale,bound", [
    (0, False, 0.3, 5.0),   # nothing clamps
    (1, True, 0.3, 5.0),    # with an input-increment weight
    (2, False, 3.0, 0.4),   # many components clamp
    (3, True, 3.0, 0.4),
    (4, False, 1.0, 1.0),
])
def test_one_iteration_equals_generic_admm(seed, rdu, hat_scale, bound):
    inst = tiny_ltv(seed, nx=3, nu=2, N=4, xabs=bound, uabs=bound, rdu=rdu, ref_scale=1.0)
    N, nx, nu = inst["N"], inst["nx"], inst["nu"]
    n = nx + nu
    rng = np.random.default_rng(100 + seed)
    hats = {k: hat_scale * rng.standard_normal((N, n)) for k in ("z", "v", "th", "be", "la")}
    H, J = oracle.cache(inst)
    out = oracle.iteration(inst, H, J, hats)

    sys_ = qp.velocity_FGh(inst)
    qhat = np.concatenate([hats["v"].ravel(), hats["z"].ravel()])
    shat = np.concatenate([hats["th"].ravel(), hats["be"].ravel(), hats["la"].ravel()])
    p, q, s, c = qp.generic_admm_step(sys_, inst["rho"], qhat, shat)

    np.testing.assert_allclose(out["du"].ravel(), p[: N * nu], rtol=0, atol=1e-11)
    np.testing.assert_allclose(out["xb"].ravel(), p[N * nu:], rtol=0, atol=1e-11)
    np.testing.assert_allclose(out["v"].ravel(), q[: N * n], rtol=0, atol=1e-10)
    np.testing.assert_allclose(out["z"].ravel(), q[N * n:], rtol=0, atol=1e-10)
    np.testing.assert_allclose(out["th"].ravel(), s[: N * n], rtol=0, atol=1e-10)
    np.testing.assert_allclose(out["be"].ravel(), s[N * n: 2 * N * n], rtol=0, atol=1e-10)
    np.testing.assert_allclose(out["la"].ravel(), s[2 * N * n:], rtol=0, atol=1e-10)
    assert abs(out["c"] - c) <= 1e-10 * max(1.0, c)
    if bound < 1.0:
        z = out["z"]
        lo = np.concatenate([inst["xmin"], inst["umin"]])
        hi = np.concatenate([inst["xmax"], inst["umax"]])
        assert np.sum(np.isclose(z, lo) | np.isclose(z, hi)) >= 5  # the projection really acted


# ---------------------------------------------------------------------------------------------
# Converged solution against brute-force KKT enumeration and the equality-constrained form.
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed,rdu", [(7, False), (18, False), (16, True), (8, True)])
def test_converged_equals_kkt_enumeration(seed, rdu):
    inst = tiny_ltv(seed, nx=2, nu=1, N=3, xabs=1.5, uabs=0.4, rdu=rdu, ref_scale=0.5)
    P, c, Aeq, beq, lb, ub, idx = qp.original_qp(inst)
    cands = qp.kkt_enumerate(P, c, Aeq, beq, lb, ub)
    assert len(cands) >= 1
    ystar = cands[0][0]
    for y, _ in cands[1:]:  # degenerate duplicates must be the same point
        np.testing.assert_allclose(y, ystar, atol=1e-8)
    n_active = int(np.sum(np.isclose(ystar, lb, atol=1e-9) | np.isclose(ystar, ub, atol=1e-9)))
    assert n_active >= 1, "fixture must have active bounds"
    N = inst["N"]
    for accel in (0, 1):
        res = oracle.solve(inst, eps=1e-26, max_iters=400000, accel=accel)
        y = np.zeros_like(ystar)
        for k in range(N):
            y[idx(k, "u")] = res["u"][k]
            y[idx(k, "x")] = res["x"][k]
        np.testing.assert_allclose(y, ystar, rtol=0, atol=1e-8)


def test_unbounded_equals_equality_qp():
    inst = tiny_ltv(21, nx=4, nu=2, N=20, ref_scale=1.0)
    for key in ("xmin", "umin"):
        inst[key] = -np.inf * np.ones_like(inst[key])
    for key in ("xmax", "umax"):
        inst[key] = np.inf * np.ones_like(inst[key])
    P, c, Aeq, beq, lb, ub, idx = qp.original_qp(inst)
    ystar, _ = qp.equality_qp(P, c, Aeq, beq)
    res = oracle.solve(inst, eps=1e-26, max_iters=200000, accel=1)
    y = np.zeros_like(ystar)
    for k in range(inst["N"]):
        y[idx(k, "u")] = res["u"][k]
        y[idx(k, "x")] = res["x"][k]
    np.testing.assert_allclose(y, ystar, rtol=0, atol=1e-9 * max(1.0, np.abs(ystar).max()))


# ---------------------------------------------------------------------------------------------
# Invariants.
# ---------------------------------------------------------------------------------------------

@pytest.mark.parametrize("seed", [31, 32, 33])
def test_plain_residual_is_monotone(seed):
    # He & Yuan (2015), Thm 4.1: c^{i+1} <= c^i for the plain iteration.
    inst = tiny_ltv(seed, x0_abs=0.8, nx=3, nu=2, N=12, xabs=1.0, uabs=0.3, ref_scale=1.0)
    res = oracle.solve(inst, eps=-1.0, max_iters=400, accel=0, history=True)
    ch = res["c_hist"]
    assert np.all(ch[1:] <= ch[:-1] * (1 + 1e-9) + 1e-300)


def test_z_stays_in_box_every_iteration():
    inst = tiny_ltv(41, x0_abs=0.8, nx=3, nu=2, N=8, xabs=0.8, uabs=0.2, ref_scale=2.0)
    lo = np.concatenate([inst["xmin"], inst["umin"]])
    hi = np.concatenate([inst["xmax"], inst["umax"]])
    for K in (1, 2, 3, 7, 20, 61):
        for accel in (0, 1):
            res = oracle.solve(inst, eps=-1.0, max_iters=K, accel=accel)
            assert np.all(res["z"] >= lo) and np.all(res["z"] <= hi)


def test_fixed_point_and_dynamics_at_convergence():
    inst = tiny_ltv(51, x0_abs=0.8, nx=3, nu=2, N=10, xabs=1.0, uabs=0.3, ref_scale=1.0)
    res = oracle.solve(inst, eps=1e-28, max_iters=300000, accel=1)
    assert res["status"] == oracle.CONVERGED
    H, J = oracle.cache(inst)
    out = oracle.iteration(inst, H, J, res)
    for k in ("z", "v", "th", "be", "la"):
        np.testing.assert_allclose(out[k], res[k], rtol=0, atol=1e-11)
    # xbar = z, Bbar du = v, and xbar_{k+1} = Abar_k xbar_k + Bbar_k du_k + ebar_k at the optimum
    nx, nu = inst["nx"], inst["nu"]
    np.testing.assert_allclose(out["xb"], out["z"], atol=1e-10)
    xprev = np.concatenate([inst["x0"], inst["u_prev"]])
    for k in range(inst["N"]):
        A, B, e = inst["A"][k], inst["B"][k], inst["e"][k]
        x_next = A @ xprev[:nx] + B @ (xprev[nx:] + out["du"][k]) + e
        np.testing.assert_allclose(out["xb"][k, :nx], x_next, atol=1e-10)
        np.testing.assert_allclose(out["xb"][k, nx:], xprev[nx:] + out["du"][k], atol=1e-10)
        xprev = out["xb"][k]


def test_optimum_independent_of_rho():
    inst = tiny_ltv(61, x0_abs=0.8, nx=3, nu=2, N=10, xabs=1.0, uabs=0.3, ref_scale=1.0)
    sols = []
    for rho in (0.3, 1.0, 4.0):
        inst["rho"] = rho
        res = oracle.solve(inst, eps=1e-26, max_iters=400000, accel=1)
        sols.append(np.concatenate([res["u"].ravel(), res["x"].ravel()]))
    np.testing.assert_allclose(sols[0], sols[1], atol=1e-8)
    np.testing.assert_allclose(sols[0], sols[2], atol=1e-8)


def test_optimum_independent_of_u_prev_without_du_weight():
    inst = tiny_ltv(71, x0_abs=0.8, nx=3, nu=2, N=10, xabs=1.0, uabs=0.3, ref_scale=1.0)
    a = oracle.solve(inst, eps=1e-26, max_iters=400000, accel=1)
    inst["u_prev"] = np.array([0.25, -0.1])
    b = oracle.solve(inst, eps=1e-26, max_iters=400000, accel=1)
    np.testing.assert_allclose(a["u"], b["u"], atol=1e-8)
    np.testing.assert_allclose(a["x"], b["x"], atol=1e-8)


def test_accel_with_eta_zero_is_plain():
    # eta = 0: the momentum branch needs c <= 0, so every step restarts and hats = iterates.
    inst = tiny_ltv(81, x0_abs=0.8, nx=3, nu=2, N=9, xabs=1.0, uabs=0.3, ref_scale=1.0)
    a = oracle.solve(inst, eps=-1.0, max_iters=150, accel=0)
    b = oracle.solve(inst, eps=-1.0, max_iters=150, accel=1, eta=0.0)
    for k in ("z", "v", "th", "be", "la"):
        assert np.array_equal(a[k], b[k])


def test_accel_converges_faster_than_plain():
    inst = tiny_ltv(91, x0_abs=0.8, nx=3, nu=2, N=30, xabs=2.0, uabs=0.5, ref_scale=1.0)
    a = oracle.solve(inst, eps=1e-12, max_iters=200000, accel=0)
    b = oracle.solve(inst, eps=1e-12, max_iters=200000, accel=1)
    assert a["status"] == oracle.CONVERGED and b["status"] == oracle.CONVERGED
    assert b["iters"] < a["iters"]


def test_forced_mask_replays_decisions():
    inst = tiny_ltv(95, x0_abs=0.8, nx=3, nu=2, N=9, xabs=1.0, uabs=0.3, ref_scale=1.0)
    a = oracle.solve(inst, eps=-1.0, max_iters=120, accel=1, history=True)
    b = oracle.solve(inst, eps=-1.0, max_iters=120, accel=1, force_mask=a["mask"])
    assert a["mask"].any() and not a["mask"].all()
    for k in ("z", "v", "th", "be", "la"):
        assert np.array_equal(a[k], b[k])


# ---------------------------------------------------------------------------------------------
# A scalar case computed by hand (nx = nu = 1, N = 1, plain iteration from zero).
# ---------------------------------------------------------------------------------------------

def test_scalar_case_by_hand():
    inst = dict(nx=1, nu=1, N=1, lti=True, A=np.array([[0.5]]), B=np.array([[1.0]]),
                e=np.array([0.25]), q=np.array([1.0]), r=np.array([1.0]), rdu=None,
                xmin=np.array([-10.0]), xmax=np.array([10.0]), umin=np.array([-0.1]),
                umax=np.array([0.1]), x0=np.array([2.0]), u_prev=None,
                ref=np.array([1.0, 1.0]), rho=1.0)
    # Iteration 1 (all hats 0): du = 0; H = (Qbar + I)^-1 = I/2, h = Qbar ref = (1, 1), so
    # xbar_1 = (0.5, 0.5). Abar xbar_0 = (0.5*2 + 1*0, 0) = (1, 0), ebar = (0.25, 0).
    # gamma = (-1.25, 0); w = ((2*(0.5+1+0.25) - 1.25)/3, (2*0.5)/3) = (0.75, 1/3) -> z = (0.75, 0.1)
    # v = (z + gamma)/2 = (-0.25, 0.05); theta = xbar - z = (-0.25, 0.4); beta = -v = (0.25, -0.05)
    # lambda = z - Abar xbar_0 - v - ebar = (-0.25, 0.05)
    # c = (0.0625*4 + 0.5625 + 1) + (0.16 + 0.0025*4 + 0.01) = 1.8125 + 0.18 = 1.9925
    r1 = oracle.solve(inst, eps=-1.0, max_iters=1)
    np.testing.assert_allclose(r1["z"], [[0.75, 0.1]], atol=1e-15)
    np.testing.assert_allclose(r1["v"], [[-0.25, 0.05]], atol=1e-15)
    np.testing.assert_allclose(r1["th"], [[-0.25, 0.4]], atol=1e-15)
    np.testing.assert_allclose(r1["be"], [[0.25, -0.05]], atol=1e-15)
    np.testing.assert_allclose(r1["la"], [[-0.25, 0.05]], atol=1e-15)
    np.testing.assert_allclose(r1["xb"], [[0.5, 0.5]], atol=1e-15)
    assert abs(r1["c"] - 1.9925) < 1e-14
    # Iteration 2 (hats = iteration-1 iterates): J = (Bbar'Bbar)^-1 Bbar' = (1/2, 1/2),
    # du = ((-0.25-0.25) + (0.05+0.05))/2 = -0.2; h = (1 + 0.75 + 0.25, 1 + 0.1 - 0.4) = (2, 0.7),
    # xbar_1 = (1, 0.35); Bbar du = (-0.2, -0.2); gamma = (-1.45, -0.2);
    # w = ((2*2.25 - 1.45)/3, (2*0.7 - 0.2)/3) = (61/60, 0.4) -> z = (61/60, 0.1)
    # v = (-13/60, -0.05); theta = (-4/15, 0.65); beta = (4/15, -0.2); lambda = (-4/15, 0.2)
    # c = 459/3600 + 0.1275 = 0.255
    r2 = oracle.solve(inst, eps=-1.0, max_iters=2)
    np.testing.assert_allclose(r2["du"], [[-0.2]], atol=1e-15)
    np.testing.assert_allclose(r2["xb"], [[1.0, 0.35]], atol=1e-15)
    np.testing.assert_allclose(r2["z"], [[61 / 60, 0.1]], atol=1e-15)
    np.testing.assert_allclose(r2["v"], [[-13 / 60, -0.05]], atol=1e-15)
    np.testing.assert_allclose(r2["th"], [[-4 / 15, 0.65]], atol=1e-15)
    np.testing.assert_allclose(r2["be"], [[4 / 15, -0.2]], atol=1e-15)
    np.testing.assert_allclose(r2["la"], [[-4 / 15, 0.2]], atol=1e-15)
    assert abs(r2["c"] - 0.255) < 1e-14


# ---------------------------------------------------------------------------------------------
# The accelerated branch (Algorithm 1 steps 6-7) on the same scalar case, by hand.
#
# Steps 6-7 with the readings taken: after iteration i+1 with residual c^{i+1},
#   * if c^{i+1} <= eta c^i: alpha_{i+1} = (1 + sqrt(1 + 4 alpha_i^2)) / 2, and every hat is
#     hat^{i+1} = new^{i+1} + ((alpha_i - 1) / alpha_{i+1}) (new^{i+1} - new^i), the momentum
#     taken from the previous NON-hat iterate (accelerated ADMM with restart, Goldstein et al.);
#   * otherwise (restart): hat^{i+1} = new^{i+1} and alpha_{i+1} = 1;
#   * in both branches c^{i+1} becomes the comparison value of the next test; alpha_0 = 1, c^0 = 1.
# ---------------------------------------------------------------------------------------------

def _scalar_inst():
    return dict(nx=1, nu=1, N=1, lti=True, A=np.array([[0.5]]), B=np.array([[1.0]]),
                e=np.array([0.25]), q=np.array([1.0]), r=np.array([1.0]), rdu=None,
                xmin=np.array([-10.0]), xmax=np.array([10.0]), umin=np.array([-0.1]),
                umax=np.array([0.1]), x0=np.array([2.0]), u_prev=None,
                ref=np.array([1.0, 1.0]), rho=1.0)


def _check_iterates(res, expect, atol):
    for key, val in zip(("z", "v", "th", "be", "la"), expect):
        np.testing.assert_allclose(res[key], [val], rtol=0, atol=atol, err_msg=key)


PHI = (1.0 + 5.0 ** 0.5) / 2.0                       # alpha_2 = (1 + sqrt(5)) / 2
ALPHA3 = (1.0 + (7.0 + 2.0 * 5.0 ** 0.5) ** 0.5) / 2.0  # 1 + 4 phi^2 = 7 + 2 sqrt(5)
F3 = (PHI - 1.0) / ALPHA3                            # (alpha_2 - 1) / alpha_3 = 0.2817535...


def test_accelerated_scalar_case_by_hand():
    inst = _scalar_inst()
    # Iteration 1 (the plain case above): c^1 = 1.9925 > 0.999 * c^0 = 0.999, so RESTART:
    # hats = iteration-1 iterates, alpha_1 = 1.
    # Iteration 2: same as the plain case, c^2 = 0.255 <= 0.999 * 1.9925: MOMENTUM with
    # alpha_2 = phi and factor (alpha_1 - 1) / alpha_2 = 0, so the hats are still the iterates.
    # Iteration 3, from the iteration-2 iterates z = (61/60, 1/10), v = (-13/60, -1/20),
    # theta = (-4/15, 13/20), beta = (4/15, -1/5), lambda = (-4/15, 1/5):
    #   du = ((-13/60 - 16/60) + (-1/20 + 1/5)) / 2 = -1/6
    #   h = (1 + 61/60 + 16/60, 1 + 1/10 - 13/20) = (137/60, 9/20), xbar_1 = h/2 = (137/120, 9/40)
    #   gamma = (-1/6 + 4/15 - 1 - 1/4 - 4/15, -1/6 - 1/5 + 1/5) = (-17/12, -1/6)
    #   w = ((2 (137/120 - 4/15 + 5/4 + 4/15) - 17/12)/3, (2 (9/40 + 13/20 - 1/5) - 1/6)/3)
    #     = (101/90, 71/180) -> z = (101/90, 1/10)
    #   v = (-53/360, -1/30), theta = (-89/360, 31/40), beta = (89/360, -1/3), lambda = (-89/360, 1/3)
    #   differences to the iteration-2 iterates (= its hats): dtheta = (7/360, 1/8),
    #   dbeta = (-7/360, -2/15), dlambda = (7/360, 2/15), dz = (38/360, 0), dv = (25/360, 1/60),
    #   d(z - v) = (13/360, -1/60), so c^3 = (2385 + 2025 + 2 * 2304 + 2 * 36) / 129600 = 101/1440.
    r3 = oracle.solve(inst, eps=-1.0, max_iters=3, accel=1)
    _check_iterates(r3, [(101 / 90, 0.1), (-53 / 360, -1 / 30), (-89 / 360, 0.775),
                         (89 / 360, -1 / 3), (-89 / 360, 1 / 3)], 1e-15)
    assert abs(r3["c"] - 101 / 1440) < 1e-15
    # c^3 = 101/1440 <= 0.999 * 0.255: MOMENTUM, alpha_3 = (1 + sqrt(7 + 2 sqrt 5))/2 = 2.1935271,
    # first nonzero factor f3 = (phi - 1)/alpha_3 = 0.28175353, applied to new^3 - new^2 (the
    # differences listed above):
    #   zhat = (101/90 + 38 f3/360, 1/10), vhat = (-53/360 + 25 f3/360, -1/30 + f3/60),
    #   thetahat = (-89/360 + 7 f3/360, 31/40 + f3/8), betahat = (89/360 - 7 f3/360, -1/3 - 2 f3/15),
    #   lambdahat = (-89/360 + 7 f3/360, 1/3 + 2 f3/15).
    # Iteration 4 from these hats:
    #   du = ((vhat - betahat)_1 + (vhat - betahat)_2)/2 = (-17 + 43 f3)/360
    #   xbar_1 = (1 + zhat - thetahat)/2 = ((853 + 31 f3)/720, 13/80 - f3/16)
    #   gamma = (du + betahat_1 - 5/4 + lambdahat_1, du + betahat_2 + lambdahat_2) = (du - 5/4, du)
    #   w_1 = (2 (xbar_1 + thetahat_1 + 5/4 - lambdahat_1) + gamma_1)/3 = (2 xbar_1 + 5/4 + du)/3
    #   w_2 = (2 (xbar_2 + thetahat_2 - lambdahat_2) + du)/3 = 0.3850 -> z_2 = 1/10
    #   v = (z + gamma)/2, theta = thetahat + xbar - z, beta = betahat + Bbar du - v,
    #   lambda = lambdahat + z - (1, 0) - v - (1/4, 0).
    du4 = (-17.0 + 43.0 * F3) / 360.0
    xb4 = ((853.0 + 31.0 * F3) / 720.0, 13.0 / 80.0 - F3 / 16.0)
    th_h = (-89 / 360 + 7 * F3 / 360, 31 / 40 + F3 / 8)
    be_h = (89 / 360 - 7 * F3 / 360, -1 / 3 - 2 * F3 / 15)
    la_h = (-89 / 360 + 7 * F3 / 360, 1 / 3 + 2 * F3 / 15)
    z4 = ((2 * xb4[0] + 1.25 + du4) / 3, 0.1)
    v4 = ((z4[0] + du4 - 1.25) / 2, (0.1 + du4) / 2)
    expect4 = [z4, v4,
               (th_h[0] + xb4[0] - z4[0], th_h[1] + xb4[1] - z4[1]),
               (be_h[0] + du4 - v4[0], be_h[1] + du4 - v4[1]),
               (la_h[0] + z4[0] - 1.25 - v4[0], la_h[1] + z4[1] - v4[1])]
    r4 = oracle.solve(inst, eps=-1.0, max_iters=4, accel=1)
    np.testing.assert_allclose(r4["du"], [[du4]], rtol=0, atol=1e-15)
    np.testing.assert_allclose(r4["xb"], [xb4], rtol=0, atol=1e-15)
    _check_iterates(r4, expect4, 1e-15)
    # Numerically: z = (1.2100461, 0.1), v = (-0.0267611, 0.0432158), ...; c^4 = 0.0346982 <=
    # 0.999 c^3: MOMENTUM, alpha_4 = 2.7497913, factor (alpha_3 - 1)/alpha_4 = 0.4340428 applied to
    # new^4 - new^3 (NOT to new^4 - hat^3). Carrying the same lines on (40-digit arithmetic)
    # gives iteration 5 and the residual / decision sequence below; the momentum streak
    # 2..7 ends in a restart at iteration 8 (c^8 = 0.0189793 > 0.999 c^7 = 0.0132236).
    r5 = oracle.solve(inst, eps=-1.0, max_iters=5, accel=1)
    _check_iterates(r5, [(1.3042030488894554, 0.1), (0.10518100701190204, 0.12807948256717436),
                         (-0.30926275538916858, 0.89494029350028678),
                         (0.30926275538916858, -0.44055765323350115),
                         (-0.30926275538916858, 0.44055765323350115)], 2e-15)
    r10 = oracle.solve(inst, eps=-1.0, max_iters=10, accel=1, history=True)
    np.testing.assert_array_equal(r10["mask"], [0, 1, 1, 1, 1, 1, 1, 0, 1, 1])
    np.testing.assert_allclose(
        r10["c_hist"],
        [1.9925, 0.255, 0.070138888888888889, 0.034698242066906957, 0.024775047451832719,
         0.01650067174732074, 0.013236803707351405, 0.018979293279754719,
         0.0089498935296779736, 0.0031235443201129231], rtol=1e-13, atol=0)
    # After the restart at 8, alpha_8 = 1: iteration 9 takes momentum with factor 0 again and
    # iteration 10 with (phi - 1)/alpha_3 (the alpha sequence starts over).
    _check_iterates(r10, [(1.3415668319288078, 0.1), (0.0722366306786494, 0.076453214714245497),
                          (-0.34058150835395322, 0.90098532357485459),
                          (0.34058150835395322, -0.3469652210416442),
                          (-0.34058150835395322, 0.3469652210416442)], 1e-14)


def test_accelerated_restart_after_a_momentum_streak_by_hand():
    # Same scalar case with eta = 0.4. Iterations 1-4 are those above (c^4 = 0.0346982);
    # iteration 3 took momentum (c^3/c^2 = 0.275 <= 0.4), iteration 4 restarts
    # (c^4/c^3 = 0.4947 > 0.4): alpha := 1, hats := new^4. Iteration 5 is then a plain step from
    # the iteration-4 iterates; c^5 = 0.0217754 is compared with c^4 (the value computed in the
    # restarting iteration), 0.0217754 > 0.4 * 0.0346982, so iteration 5 restarts as well (with a
    # comparison value reset to c^0 = 1 it would wrongly take momentum). Ratios then run
    # 0.551 (restart), 0.427 (restart), 0.332 (momentum, factor 0 since alpha = 1),
    # 0.340 (momentum, factor (phi - 1)/alpha_3: alpha restarted from 1), 0.561 (restart).
    inst = _scalar_inst()
    r = oracle.solve(inst, eps=-1.0, max_iters=10, accel=1, eta=0.4, history=True)
    np.testing.assert_array_equal(r["mask"], [0, 1, 1, 0, 0, 0, 0, 1, 1, 0])
    np.testing.assert_allclose(
        r["c_hist"],
        [1.9925, 0.255, 0.070138888888888889, 0.034698242066906957, 0.021775415634775444,
         0.011991158748049989, 0.0051179576332096188, 0.0017007691688496881,
         0.00057744099740557136, 0.00032384853594166815], rtol=1e-13, atol=0)
    r5 = oracle.solve(inst, eps=-1.0, max_iters=5, accel=1, eta=0.4)
    _check_iterates(r5, [(1.2698613287114396, 0.1), (0.057231380213347481, 0.097300715857627703),
                         (-0.29230653105127328, 0.87755479766016628),
                         (0.29230653105127328, -0.43038391863076397),
                         (-0.29230653105127328, 0.43038391863076397)], 2e-15)
    r9 = oracle.solve(inst, eps=-1.0, max_iters=9, accel=1, eta=0.4)
    _check_iterates(r9, [(1.3679444603362244, 0.1), (0.11875474239762131, 0.10978251222950911),
                         (-0.36934728548246401, 0.89859717485376039),
                         (0.36934728548246401, -0.35109508004423997),
                         (-0.36934728548246401, 0.35109508004423997)], 1e-14)
