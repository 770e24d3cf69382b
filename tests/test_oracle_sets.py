"""Pins of the oracle's non-box input sets (the remark after Theorem 1: the (v, z) update keeps
its closed form for any closed convex set, only the projection changes). CPU only.

* Each projection p = P_U(y) satisfies what characterises the Euclidean projection onto a
  closed convex set: p in U, (y - p)'(q - p) <= 0 for points q of U sampled independently, and
  P_U(p) = p; it also equals the minimiser found by a general NLP routine (scipy SLSQP). The l1
  projection is also checked against the root of sum max(|y_i| - tau, 0) = r found by bisection.
* One oracle iteration with an input set equals one generic scaled-ADMM pass on the explicit
  F, G, h of Theorem 2's problem whose q-update is solved by SLSQP with the set as constraints.
* The converged oracle equals the MPC problem with u_k in U solved directly by SLSQP.
"""
import numpy as np
import pytest

import oracle
import qp_reference as qp
from test_oracle_pins import tiny_ltv

SETS = {
    "ball2": dict(kind=oracle.USET_BALL2, r=0.3),
    "ball1": dict(kind=oracle.USET_BALL1, r=0.4),
    "halfspace": dict(kind=oracle.USET_HALFSPACE, r=0.1, a=np.array([1.0, -0.5])),
    "soc": dict(kind=oracle.USET_SOC, r=0.0),
}


def inst_with(name, seed=3, **kw):
    inst = tiny_ltv(seed, nx=2, nu=2, N=3, xabs=3.0, uabs=1.0, ref_scale=1.0, x0_abs=2.0, **kw)
    inst["umin"], inst["umax"] = -np.inf * np.ones(2), np.inf * np.ones(2)  # unused by U
    inst["uset"] = SETS[name]
    return inst


def sample_in_set(name, rng, m):
    us = SETS[name]
    if name == "ball2":
        d = rng.standard_normal((m, 2))
        d /= np.linalg.norm(d, axis=1, keepdims=True)
        return d * us["r"] * rng.uniform(0, 1, (m, 1)) ** 0.5
    if name == "ball1":
        pts = rng.uniform(-us["r"], us["r"], (4 * m, 2))
        return pts[np.abs(pts).sum(1) <= us["r"]][:m]
    if name == "halfspace":
        pts = rng.uniform(-3, 3, (4 * m, 2))
        return pts[pts @ us["a"] <= us["r"]][:m]
    s = rng.uniform(-2, 2, m)
    return np.stack([np.abs(s) + rng.uniform(0, 1, m), s], axis=1)


def in_set(name, p, tol=1e-12):
    us = SETS[name]
    if name == "ball2":
        return np.linalg.norm(p) <= us["r"] + tol
    if name == "ball1":
        return np.abs(p).sum() <= us["r"] + tol
    if name == "halfspace":
        return p @ us["a"] <= us["r"] + tol
    return np.linalg.norm(p[1:]) <= p[0] + tol


@pytest.mark.parametrize("name", list(SETS))
def test_projection_is_the_euclidean_projection(name):
    from scipy.optimize import minimize
    inst = inst_with(name)
    rng = np.random.default_rng(11)
    qs = sample_in_set(name, rng, 400)
    moved = 0
    for y in rng.uniform(-2.0, 2.0, (60, 2)):
        p = oracle.project_u(inst, y)
        assert in_set(name, p)
        assert np.max((qs - p) @ (y - p)) <= 1e-12
        np.testing.assert_allclose(oracle.project_u(inst, p), p, rtol=0, atol=1e-14)
        cons = qp.set_constraints(dict(inst, N=1), [slice(0, 2)])
        ref = minimize(lambda z: 0.5 * np.sum((z - y) ** 2), p + 0.01, jac=lambda z: z - y,
                       method="SLSQP", constraints=cons, options=dict(ftol=1e-16)).x
        np.testing.assert_allclose(p, ref, rtol=0, atol=1e-6)
        moved += np.linalg.norm(p - y) > 1e-9
    assert moved >= 20      # most points lay outside the set


def test_l1_projection_threshold_by_bisection():
    rng = np.random.default_rng(5)
    for nu in (2, 3, 5, 8):
        inst = dict(nx=1, nu=nu, N=1, uset=dict(kind=oracle.USET_BALL1, r=0.7), q=[1.0],
                    r=np.ones(nu), xmin=[-1.0], xmax=[1.0], umin=-np.ones(nu), umax=np.ones(nu),
                    A=np.zeros((1, 1)), B=np.zeros((1, nu)), e=np.zeros(1), x0=np.zeros(1),
                    ref=np.zeros(1 + nu), rho=1.0, lti=True)
        for _ in range(20):
            y = rng.standard_normal(nu) * 0.8
            y[rng.integers(nu)] = y[0]                 # a tie in |y|
            p = oracle.project_u(inst, y)
            if np.abs(y).sum() <= 0.7:
                np.testing.assert_array_equal(p, y)
                continue
            lo, hi = 0.0, np.abs(y).max()
            for _ in range(200):
                mid = 0.5 * (lo + hi)
                if np.maximum(np.abs(y) - mid, 0).sum() > 0.7:
                    lo = mid
                else:
                    hi = mid
            ref = np.sign(y) * np.maximum(np.abs(y) - 0.5 * (lo + hi), 0.0)
            np.testing.assert_allclose(p, ref, rtol=0, atol=1e-13)


@pytest.mark.parametrize("name", list(SETS))
def test_one_iteration_with_an_input_set_equals_generic_admm(name):
    inst = inst_with(name, seed=4)
    N, nx, nu = inst["N"], inst["nx"], inst["nu"]
    n = nx + nu
    rng = np.random.default_rng(21)
    hats = {k: 0.7 * rng.standard_normal((N, n)) for k in ("z", "v", "th", "be", "la")}
    H, J = oracle.cache(inst)
    out = oracle.iteration(inst, H, J, hats)
    sys_ = qp.velocity_FGh(inst)
    qhat = np.concatenate([hats["v"].ravel(), hats["z"].ravel()])
    shat = np.concatenate([hats["th"].ravel(), hats["be"].ravel(), hats["la"].ravel()])
    p, q, s, c = qp.generic_admm_step_set(sys_, inst["rho"], qhat, shat, inst)
    np.testing.assert_allclose(out["xb"].ravel(), p[N * nu:], rtol=0, atol=1e-11)
    np.testing.assert_allclose(out["v"].ravel(), q[: N * n], rtol=0, atol=1e-7)
    np.testing.assert_allclose(out["z"].ravel(), q[N * n:], rtol=0, atol=1e-7)
    np.testing.assert_allclose(out["la"].ravel(), s[2 * N * n:], rtol=0, atol=1e-7)
    assert abs(out["c"] - c) <= 1e-6 * max(1.0, c)
    zu = out["z"][:, nx:]
    assert all(in_set(name, u, tol=1e-12) for u in zu)


@pytest.mark.parametrize("name", list(SETS))
def test_converged_with_an_input_set_equals_the_constrained_qp(name):
    inst = inst_with(name, seed=6)
    r = oracle.solve(inst, eps=1e-26, max_iters=200000, accel=1)
    y, idx = qp.solve_set_qp(inst)
    N = inst["N"]
    u = np.array([y[idx(k, "u")] for k in range(N)])
    x = np.array([y[idx(k, "x")] for k in range(N)])
    np.testing.assert_allclose(r["u"], u, rtol=0, atol=2e-6)
    np.testing.assert_allclose(r["x"], x, rtol=0, atol=2e-6)
    for k in range(N):
        assert in_set(name, r["u"][k], tol=1e-9)
    free = oracle.solve(dict(inst, uset=None), eps=1e-26, max_iters=200000, accel=1)
    assert np.max(np.abs(free["u"] - r["u"])) > 1e-2       # U changes the optimum
