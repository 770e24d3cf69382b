"""Pins of the oracle's nonlinear models and explicit-Euler linearisation (CPU only).

The models are not printed in the paper except the CSTR (Sec. V); the quadrotor and cart-pole are
textbook rigid-body models. They are pinned by physics that any correct implementation obeys
(equilibria, energy balance, rotation kinematics) and the linearisation by central finite
differences and by its exactness at the linearisation point.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import workloads as W

QUAD = W.QUAD_PARAMS
CP = W.CARTPOLE_PARAMS


def rot_zyx(phi, th, psi):
    cx, sx, cy, sy, cz, sz = np.cos(phi), np.sin(phi), np.cos(th), np.sin(th), np.cos(psi), np.sin(psi)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def skew(w):
    return np.array([[0, -w[2], w[1]], [w[2], 0, -w[0]], [-w[1], w[0], 0]])


def quad_state(rng):
    x = np.zeros(12)
    x[0:3] = rng.uniform(-2, 2, 3)
    x[3:6] = rng.uniform(-1, 1, 3)
    x[6:9] = rng.uniform(-0.5, 0.5, 3)
    x[9:12] = rng.uniform(-1, 1, 3)
    return x


def test_quadrotor_hover_is_equilibrium():
    m, g = QUAD[0], QUAD[1]
    x = np.zeros(12)
    x[0:3] = [1.0, -2.0, 3.0]
    x[8] = 0.4  # any yaw
    u = np.full(4, m * g / 4)
    np.testing.assert_allclose(oracle.model_f(0, QUAD, x, u), 0.0, atol=1e-14)


def test_quadrotor_translational_dynamics_and_kinematics():
    rng = np.random.default_rng(0)
    m, g, Jx, Jy, Jz, l, ky = QUAD
    for _ in range(5):
        x = quad_state(rng)
        u = rng.uniform(0, m * g / 2, 4)
        f = oracle.model_f(0, QUAD, x, u)
        R = rot_zyx(*x[6:9])
        np.testing.assert_allclose(f[0:3], x[3:6], atol=1e-15)
        np.testing.assert_allclose(f[3:6], R @ np.array([0, 0, u.sum()]) / m - np.array([0, 0, g]),
                                   atol=1e-12)
        # Euler-angle rates must reproduce dR/dt = R [w]_x
        d = 1e-6
        dR = (rot_zyx(*(x[6:9] + d * f[6:9])) - rot_zyx(*(x[6:9] - d * f[6:9]))) / (2 * d)
        np.testing.assert_allclose(dR, R @ skew(x[9:12]), atol=1e-8)


def test_quadrotor_rotational_dynamics():
    rng = np.random.default_rng(1)
    m, g, Jx, Jy, Jz, l, ky = QUAD
    J = np.diag([Jx, Jy, Jz])
    for _ in range(5):
        x = quad_state(rng)
        w = x[9:12]
        # equal thrusts -> zero torque -> rotational kinetic energy is conserved
        f = oracle.model_f(0, QUAD, x, np.full(4, 2.0))
        assert abs(w @ J @ f[9:12]) < 1e-12
        # angular momentum balance J dw/dt = tau - w x J w with tau from the rotor layout
        u = rng.uniform(0, m * g / 2, 4)
        f = oracle.model_f(0, QUAD, x, u)
        tau = np.array([l * (u[1] - u[3]), l * (u[2] - u[0]), ky * (u[0] - u[1] + u[2] - u[3])])
        np.testing.assert_allclose(J @ f[9:12], tau - np.cross(w, J @ w), atol=1e-12)


def cartpole_energy(x):
    mc, mp, l, g = CP
    M = mc + mp
    return (0.5 * M * x[1] ** 2 + mp * l * x[1] * x[3] * np.cos(x[2])
            + 0.5 * (4.0 / 3.0) * mp * l ** 2 * x[3] ** 2 + mp * g * l * np.cos(x[2]))


def test_cartpole_energy_balance():
    rng = np.random.default_rng(2)
    for _ in range(10):
        x = rng.uniform(-2, 2, 4)
        F = rng.uniform(-5, 5)
        f = oracle.model_f(1, CP, x, np.array([F]))
        d = 1e-6
        dE = (cartpole_energy(x + d * f) - cartpole_energy(x - d * f)) / (2 * d)
        # dE/dt = power of the applied force
        assert abs(dE - F * x[1]) < 1e-7


def test_cartpole_upright_equilibrium():
    np.testing.assert_allclose(oracle.model_f(1, CP, np.zeros(4), np.zeros(1)), 0.0, atol=1e-15)


def test_cstr_initial_state_is_near_steady_state():
    # The printed low-conversion state (C_A = 8.57, T = 311 K) is (to the printed digits) a steady
    # state of the paper's CSTR at the classic coolant temperature T_c = 300 K and T_i = 298.15 K.
    f = oracle.model_f(2, np.append(W.CSTR_PARAMS, 298.15), np.array([8.57, 311.0]),
                       np.array([300.0]))
    assert abs(f[0]) < 0.1 and abs(f[1]) < 1.5


@pytest.mark.parametrize("model,params,nx,nu", [
    (0, QUAD, 12, 4),
    (1, CP, 4, 1),
    (2, np.append(W.CSTR_PARAMS, 300.0), 2, 1),
])
def test_linearisation_matches_finite_differences(model, params, nx, nu):
    rng = np.random.default_rng(3)
    N, dt = 4, 0.02
    if model == 2:
        xbar = np.column_stack([rng.uniform(2, 9, N), rng.uniform(300, 360, N)])
        ubar = rng.uniform(280, 320, (N, nu))
    else:
        xbar = rng.uniform(-0.5, 0.5, (N, nx))
        ubar = rng.uniform(0.5, 3.0, (N, nu))
    A, B, e = oracle.linearise(model, params, dt, xbar, ubar)
    for k in range(N):
        Fk = lambda x, u: x + dt * oracle.model_f(model, params, x, u)
        hx = 1e-6 * np.maximum(1.0, np.abs(xbar[k]))
        hu = 1e-6 * np.maximum(1.0, np.abs(ubar[k]))
        Afd = np.column_stack([(Fk(xbar[k] + hx[j] * np.eye(nx)[j], ubar[k]) -
                                Fk(xbar[k] - hx[j] * np.eye(nx)[j], ubar[k])) / (2 * hx[j])
                               for j in range(nx)])
        Bfd = np.column_stack([(Fk(xbar[k], ubar[k] + hu[j] * np.eye(nu)[j]) -
                                Fk(xbar[k], ubar[k] - hu[j] * np.eye(nu)[j])) / (2 * hu[j])
                               for j in range(nu)])
        scale = max(1.0, np.abs(Afd).max())
        np.testing.assert_allclose(A[k], Afd, atol=1e-7 * scale)
        np.testing.assert_allclose(B[k], Bfd, atol=1e-7 * max(1.0, np.abs(Bfd).max()))
        # exact at the linearisation point: A xbar + B ubar + e = F(xbar, ubar)
        np.testing.assert_allclose(A[k] @ xbar[k] + B[k] @ ubar[k] + e[k], Fk(xbar[k], ubar[k]),
                                   atol=1e-10 * max(1.0, np.abs(xbar[k]).max()))


def test_plant_step_is_explicit_euler():
    rng = np.random.default_rng(4)
    x = quad_state(rng)
    u = rng.uniform(0, 4, 4)
    xn = oracle.plant_step(0, QUAD, 0.02, x, u)
    np.testing.assert_allclose(xn, x + 0.02 * oracle.model_f(0, QUAD, x, u), atol=1e-15)
