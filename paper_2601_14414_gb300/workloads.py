"""Seeded synthetic workloads shaped like the paper's experiments (arXiv 2601.14414, Sec. V).

This module only draws inputs: it holds none of the solver's arithmetic, and both the CUDA path
and the FP64 CPU oracle read the same instances from it. Every instance is a plain dict:

    nx, nu, N          state size, input size, horizon
    lti                True: A [nx,nx], B [nx,nu], e [nx] shared by all stages;
                       False: A [N,nx,nx], B [N,nx,nu], e [N,nx] (one triple per stage)
    q [nx], r [nu]     diagonals of C^T W_y C and W_u (C = I)
    rdu [nu] or None   optional weight on the input increment (None = 0)
    xmin, xmax [nx]    state box;  umin, umax [nu] input box (+-inf allowed)
    x0 [nx]            measured state x(t);  u_prev [nu] or None (u(t-1), None = 0)
    ref [n] or [N,n]   reference for xbar_{k+1} = (x_{k+1}, u_k), n = nx + nu
    rho                ADMM penalty

Nonlinear (RTI) workloads add ``model`` (0 quadrotor, 1 cart-pole, 2 CSTR), ``params`` and ``dt``.

Random linear systems follow the paper's recipe (Sec. V-B): A and B with N(0, 1) entries and A
scaled to a chosen spectral radius. For the batched time-varying workload each stage's A_k is a
random signed-permutation similarity of one of a few eigen-analysed Gaussian base matrices per
instance, rescaled to its own spectral radius: the entries stay N(0, 1)-distributed before scaling,
the spectral radius is exact, and generation needs 4 eigen-decompositions per instance instead of
one per stage.
"""
from __future__ import annotations

import numpy as np

MODEL_QUADROTOR, MODEL_CARTPOLE, MODEL_CSTR = 0, 1, 2

# Quadrotor parameters: m [kg], g [m/s^2], Jx, Jy, Jz [kg m^2], arm l [m], yaw-torque coefficient.
QUAD_PARAMS = np.array([1.0, 9.81, 0.01, 0.01, 0.02, 0.2, 0.02])
# Cart-pole parameters: cart mass, pole mass, pole half-length, g.
CARTPOLE_PARAMS = np.array([1.0, 0.1, 0.5, 9.81])
# CSTR parameters of the paper's nonlinear example: C_Ai, k0, EaR; T_i is appended per sample.
CSTR_PARAMS = np.array([10.0, 34930800.0, 5963.6])


def _scaled_gaussian(rng, nx, radius):
    A = rng.standard_normal((nx, nx))
    sr = np.max(np.abs(np.linalg.eigvals(A)))
    return A * (radius / sr)


def _box(nx, nu, xabs, uabs):
    return dict(xmin=-xabs * np.ones(nx), xmax=xabs * np.ones(nx),
                umin=-uabs * np.ones(nu), umax=uabs * np.ones(nu))


def plain_lti(seed=1, nx=4, nu=2, N=20, radius=0.95, rho=1.0):
    """Plain linear MPC, one instance: A ~ N(0,1) scaled to spectral radius 0.95, B ~ N(0,1),
    Q = I, R = 0.1 I, |u| <= 1, |x| <= 5, x0 ~ U[-3, 3], reference 0, rho = 1."""
    rng = np.random.default_rng(seed)
    A = _scaled_gaussian(rng, nx, radius)
    B = rng.standard_normal((nx, nu))
    inst = dict(nx=nx, nu=nu, N=N, lti=True, A=A, B=B, e=np.zeros(nx),
                q=np.ones(nx), r=0.1 * np.ones(nu), rdu=None,
                x0=rng.uniform(-3, 3, nx), u_prev=None, ref=np.zeros(nx + nu), rho=rho)
    inst.update(_box(nx, nu, 5.0, 1.0))
    return inst


def random_ltv(seed, nx, nu, N, radius_lo=0.9, radius_hi=1.05, e_scale=0.3, xabs=5.0, uabs=1.0,
               rho=1.0, n_base=4, x0_abs=3.0):
    """One random linear time-varying instance (paper's random-system recipe, per stage)."""
    rng = np.random.default_rng(seed)
    bases = []
    for _ in range(n_base):
        A0 = rng.standard_normal((nx, nx))
        bases.append(A0 / np.max(np.abs(np.linalg.eigvals(A0))))
    bases = np.stack(bases)
    pick = rng.integers(0, n_base, N)
    radius = rng.uniform(radius_lo, radius_hi, N)
    perm = np.argsort(rng.random((N, nx)), axis=1)
    sign = rng.choice([-1.0, 1.0], (N, nx))
    # A_k = radius_k * S_k P_k A0 P_k^T S_k with a signed permutation S_k P_k.
    Abase = bases[pick]
    rows = np.take_along_axis(Abase, perm[:, :, None], axis=1)
    A = np.take_along_axis(rows, perm[:, None, :], axis=2)
    A = A * sign[:, :, None] * sign[:, None, :] * radius[:, None, None]
    B = rng.standard_normal((N, nx, nu))
    e = rng.uniform(-e_scale, e_scale, (N, nx))
    inst = dict(nx=nx, nu=nu, N=N, lti=False, A=A, B=B, e=e,
                q=np.ones(nx), r=0.1 * np.ones(nu), rdu=None,
                x0=rng.uniform(-x0_abs, x0_abs, nx), u_prev=None, ref=np.zeros(nx + nu), rho=rho)
    inst.update(_box(nx, nu, xabs, uabs))
    return inst


def batched_uneven(seed=3, batch=4096, nx_range=(4, 24), nu_range=(2, 8), N_range=(50, 500),
                   **kw):
    """Batched uneven workload: independent random LTV instances with nx ~ U{4..24},
    nu ~ U{2..8}, N ~ U{50..500}; per-stage spectral radius ~ U[0.9, 1.05]."""
    rng = np.random.default_rng(seed)
    nxs = rng.integers(nx_range[0], nx_range[1] + 1, batch)
    nus = rng.integers(nu_range[0], nu_range[1] + 1, batch)
    Ns = rng.integers(N_range[0], N_range[1] + 1, batch)
    seeds = rng.integers(0, 2**63 - 1, batch)
    return [random_ltv(int(s), int(a), int(b), int(c), **kw) for s, a, b, c in zip(seeds, nxs, nus, Ns)]


def batched_dims(seed=3, batch=4096, nx_range=(4, 24), nu_range=(2, 8), N_range=(50, 500)):
    """The (nx, nu, N) triples of ``batched_uneven`` without drawing the matrices."""
    rng = np.random.default_rng(seed)
    nxs = rng.integers(nx_range[0], nx_range[1] + 1, batch)
    nus = rng.integers(nu_range[0], nu_range[1] + 1, batch)
    Ns = rng.integers(N_range[0], N_range[1] + 1, batch)
    return nxs, nus, Ns


def large_lti(seed=5, batch=256, nx=48, nu=16, N=1000, radius=0.95, umax=None, rho=1.0,
              e_scale=0.3):
    """Large-state LTI stress workload: Q = diag U[0.1, 10], R = diag U[0.01, 1], a constant
    disturbance e ~ U[-0.3, 0.3] (the paper's random-system recipe; it keeps the inputs busy over
    the whole horizon), |x| <= 5 and an input bound chosen so that roughly a fifth of the input
    values would exceed it without the bound."""
    rng = np.random.default_rng(seed)
    umax = LARGE_LTI_UMAX if umax is None else umax
    out = []
    for _ in range(batch):
        A = _scaled_gaussian(rng, nx, radius)
        B = rng.standard_normal((nx, nu))
        e = rng.uniform(-e_scale, e_scale, nx)
        inst = dict(nx=nx, nu=nu, N=N, lti=True, A=A, B=B, e=e,
                    q=rng.uniform(0.1, 10.0, nx), r=rng.uniform(0.01, 1.0, nu), rdu=None,
                    x0=rng.uniform(-3, 3, nx), u_prev=None, ref=np.zeros(nx + nu), rho=rho)
        inst.update(_box(nx, nu, 5.0, umax))
        out.append(inst)
    return out


# Input bound of the large-state workload: the 80th percentile of |u| over the input-unconstrained
# oracle solutions of the first two instances (tests/golden/calibrate_large_lti.py prints it).
LARGE_LTI_UMAX = 0.0871132


def cartpole_batch(seed=4, batch=1024, N=100, dt=0.05, umax=10.0, rho=1.0):
    """Differentiable cart-pole workload: the model is linearised at the upright equilibrium by
    the solver's own linearisation; x0 has small random angles U[-0.3, 0.3]; reference 0."""
    rng = np.random.default_rng(seed)
    nx, nu = 4, 1
    out = []
    for _ in range(batch):
        x0 = np.zeros(nx)
        x0[2] = rng.uniform(-0.3, 0.3)
        inst = dict(nx=nx, nu=nu, N=N, lti=True, model=MODEL_CARTPOLE,
                    params=CARTPOLE_PARAMS.copy(), dt=dt,
                    op_x=np.zeros(nx), op_u=np.zeros(nu),
                    q=np.array([10.0, 1.0, 10.0, 1.0]), r=np.array([0.1]), rdu=None,
                    x0=x0, u_prev=None, ref=np.zeros(nx + nu), rho=rho,
                    xmin=-np.inf * np.ones(nx), xmax=np.inf * np.ones(nx),
                    umin=-umax * np.ones(nu), umax=umax * np.ones(nu))
        out.append(inst)
    return out


def quadrotor_rti(seed=2, N=200, dt=0.02, n_waypoints=10, switch_every=5, rti_steps=50,
                  iters=100, rho=1.0):
    """Quadrotor NMPC with real-time iteration: 12 states, 4 rotor thrusts in [0, m g / 2],
    roll/pitch/yaw box +-0.6 rad, random waypoints U[-5, 5]^3 switching every 5 samples."""
    rng = np.random.default_rng(seed)
    m, g = QUAD_PARAMS[0], QUAD_PARAMS[1]
    nx, nu = 12, 4
    waypoints = rng.uniform(-5, 5, (n_waypoints, 3))
    xmin = -np.inf * np.ones(nx)
    xmax = np.inf * np.ones(nx)
    xmin[6:9], xmax[6:9] = -0.6, 0.6
    q = np.array([10, 10, 10, 1, 1, 1, 1, 1, 1, 0.1, 0.1, 0.1], dtype=np.float64)
    return dict(nx=nx, nu=nu, N=N, lti=False, model=MODEL_QUADROTOR, params=QUAD_PARAMS.copy(),
                dt=dt, q=q, r=0.1 * np.ones(nu), rdu=None, xmin=xmin, xmax=xmax,
                umin=np.zeros(nu), umax=0.5 * m * g * np.ones(nu), x0=np.zeros(nx),
                u_prev=None, hover_u=0.25 * m * g * np.ones(nu), waypoints=waypoints,
                switch_every=switch_every, rti_steps=rti_steps, iters=iters, rho=rho)


def quadrotor_reference(wl, step):
    """The [n] reference (position waypoint, zero velocity/attitude/rates, hover thrust) that is
    active at RTI sample ``step``."""
    wp = wl["waypoints"][(step // wl["switch_every"]) % len(wl["waypoints"])]
    ref = np.zeros(wl["nx"] + wl["nu"])
    ref[0:3] = wp
    ref[wl["nx"]:] = wl["hover_u"]
    return ref


def cstr_nmpc(N=5000, dt=0.5, rho=1.0, tc_bounds=(250.0, 350.0)):
    """CSTR NMPC of the paper's nonlinear example: C_A from 8.57 to 2 kgmol/m^3, T(0) = 311 K,
    forward Euler T_s = 0.5 min, W_y = 1 on C_A, W_u = 0, W_du = 0.1. The coolant bounds are not
    printed in the paper and are assumed here."""
    nx, nu = 2, 1
    return dict(nx=nx, nu=nu, N=N, lti=False, model=MODEL_CSTR, params=CSTR_PARAMS.copy(), dt=dt,
                q=np.array([1.0, 0.0]), r=np.array([0.0]), rdu=np.array([0.1]),
                xmin=-np.inf * np.ones(nx), xmax=np.inf * np.ones(nx),
                umin=np.array([tc_bounds[0]]), umax=np.array([tc_bounds[1]]),
                x0=np.array([8.57, 311.0]), u_prev=np.array([300.0]),
                ref=np.array([2.0, 0.0, 0.0]), rho=rho)


def cstr_inlet_temperature(t_min):
    """T_i(t) = 298.15 + 5 sin(0.05 t) K (t in minutes)."""
    return 298.15 + 5.0 * np.sin(0.05 * t_min)


# AFTI-16 aircraft, continuous-time linearised model printed in the paper's first example
# (Sec. V-A): four states, two control surfaces, outputs y = (x_2, x_4) (attack and pitch angle).
AFTI16_AC = np.array([[-0.0151, -60.5651, 0.0, -32.174],
                      [-0.0001, -1.3411, 0.9929, 0.0],
                      [0.00018, 43.2541, -0.86939, 0.0],
                      [0.0, 0.0, 1.0, 0.0]])
AFTI16_BC = np.array([[-2.516, -13.136],
                      [-0.1689, -0.2514],
                      [-17.251, -1.5766],
                      [0.0, 0.0]])


def zoh(Ac, Bc, dt, terms=40, squarings=8):
    """Zero-order-hold discretisation: [[A, B], [0, I]] = exp([[Ac, Bc], [0, 0]] dt), the
    exponential by scaling and squaring of a truncated Taylor series (input generation only)."""
    nx, nu = Bc.shape
    M = np.zeros((nx + nu, nx + nu))
    M[:nx, :nx] = Ac
    M[:nx, nx:] = Bc
    M *= dt / 2.0 ** squarings
    E = np.eye(nx + nu)
    term = np.eye(nx + nu)
    for k in range(1, terms):
        term = term @ M / k
        E = E + term
    for _ in range(squarings):
        E = E @ E
    return E[:nx, :nx], E[:nx, nx:]


def afti16(N=5, dt=0.05, rho=10.0, steps=200, amplitude=10.0, period=100):
    """AFTI-16 tracking MPC of the paper's first example: ZOH at 0.05 s, |u_i| <= 25 (degrees),
    |y_1| <= 0.5, |y_2| <= 100 (state bounds on x_2 and x_4, C selects them), W_y = diag(100, 100)
    (so Q = C^T W_y C = diag(0, 100, 0, 100)), W_u = 0, W_du = diag(0.1, 0.1), N = 5, 200 MPC steps
    from rest. The paper does not print the pitch reference r_2 or rho: here r_2 is a square wave
    of +-amplitude degrees with the given period in steps (y_1 is regulated to 0), and rho = 10,
    the value of {0.1, 1, 3, 5, 10, 20, 30, 100} with the fewest iterations on this reference."""
    A, B = zoh(AFTI16_AC, AFTI16_BC, dt)
    nx, nu = 4, 2
    inf = np.inf
    return dict(nx=nx, nu=nu, N=N, lti=True, A=A, B=B, e=np.zeros(nx),
                q=np.array([0.0, 100.0, 0.0, 100.0]), r=np.zeros(nu), rdu=np.array([0.1, 0.1]),
                xmin=np.array([-inf, -0.5, -inf, -100.0]), xmax=np.array([inf, 0.5, inf, 100.0]),
                umin=-25.0 * np.ones(nu), umax=25.0 * np.ones(nu),
                x0=np.zeros(nx), u_prev=np.zeros(nu), ref=np.zeros(nx + nu), rho=rho, dt=dt,
                steps=steps, amplitude=amplitude, period=period)


def afti16_reference(wl, step):
    """Reference of xbar_{k+1} = (x, u) at MPC step `step`: pitch x_4 -> r_2(step), the rest 0."""
    ref = np.zeros(wl["nx"] + wl["nu"])
    ref[3] = wl["amplitude"] if (step // (wl["period"] // 2)) % 2 == 0 else -wl["amplitude"]
    return ref
