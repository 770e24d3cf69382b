"""Pins of the gradient oracle (central finite differences of the unrolled FP64 oracle, CPU only).

The unrolled solve converges to the QP optimum, whose derivative at a strictly complementary
solution is the implicit derivative of the KKT system with the active bounds held as equalities.
That derivative is computed here from the dense QP of the problem statement (tests/qp_reference.py),
independently of the ADMM iteration, and compared with the finite-difference gradient of the
oracle unrolled to convergence.
"""
import numpy as np
import pytest

import oracle
import qp_reference as qp
from test_oracle_pins import tiny_ltv


def kkt_loss(inst, active, Wu, Wx):
    P, c, Aeq, beq, lb, ub, idx = qp.original_qp(inst)
    fixed = [(i, lb[i] if side < 0 else ub[i]) for i, side in active]
    y, _ = qp.equality_qp(P, c, Aeq, beq, fixed)
    L = 0.0
    for k in range(inst["N"]):
        L += np.sum(Wu[k] * y[idx(k, "u")]) + np.sum(Wx[k] * y[idx(k, "x")])
    return L


def kkt_gradient(inst, active, Wu, Wx, name, h=1e-6):
    base = np.array(oracle.reference(inst) if name == "ref" else inst[name], dtype=np.float64)
    g = np.zeros_like(base)
    for ix in np.ndindex(base.shape):
        p = base.copy(); p[ix] += h
        m = base.copy(); m[ix] -= h
        g[ix] = (kkt_loss(oracle.with_params(inst, **{name: p}), active, Wu, Wx) -
                 kkt_loss(oracle.with_params(inst, **{name: m}), active, Wu, Wx)) / (2 * h)
    return g


@pytest.mark.parametrize("seed", [7, 18])
def test_unrolled_gradient_matches_implicit_kkt(seed):
    inst = tiny_ltv(seed, nx=2, nu=1, N=3, xabs=1.5, uabs=0.4, ref_scale=0.5)
    P, c, Aeq, beq, lb, ub, idx = qp.original_qp(inst)
    cands = qp.kkt_enumerate(P, c, Aeq, beq, lb, ub)
    y, states = cands[0]
    bounded = [i for i in range(len(y)) if np.isfinite(lb[i]) or np.isfinite(ub[i])]
    active = [(i, -1 if s == 1 else 1) for i, s in zip(bounded, states) if s != 0]
    assert active, "fixture must have active bounds"
    rng = np.random.default_rng(seed)
    Wu = rng.standard_normal((inst["N"], inst["nu"]))
    Wx = rng.standard_normal((inst["N"], inst["nx"]))
    iters = 60000
    for name in ("x0", "q", "r", "ref", "umax", "umin", "xmax", "xmin"):
        g_fd = oracle.fd_gradient(inst, Wu, Wx, iters, name, h=1e-6)
        g_kkt = kkt_gradient(inst, active, Wu, Wx, name)
        np.testing.assert_allclose(g_fd, g_kkt, rtol=0, atol=2e-5, err_msg=name)


def test_fd_gradient_is_step_size_consistent():
    inst = tiny_ltv(3, x0_abs=0.8, nx=3, nu=2, N=6, xabs=1.0, uabs=0.3, ref_scale=1.0)
    rng = np.random.default_rng(0)
    Wu = rng.standard_normal((inst["N"], inst["nu"]))
    Wx = rng.standard_normal((inst["N"], inst["nx"]))
    for name in ("x0", "q", "r"):
        a = oracle.fd_gradient(inst, Wu, Wx, 40, name, h=1e-6)
        b = oracle.fd_gradient(inst, Wu, Wx, 40, name, h=1e-5)
        np.testing.assert_allclose(a, b, rtol=1e-5, atol=1e-7)
