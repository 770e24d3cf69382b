"""Real-time-iteration NMPC closed loop on the GPU against the same loop run by the oracle.

Quadrotor workload at full size (12 states, 4 rotor thrusts, N = 200, dt = 0.02, 50 samples of
100 iterations, random waypoints). Every sample: linearise the model along the previous solution
shifted by one stage (the measured state first, the last input repeated), factorise, solve with
a warm start from the previous iterates, apply u_0 to the plant (one explicit-Euler step).

* FP64: the GPU loop and the oracle loop run independently; the applied inputs and the plant
  states agree to 1e-8 over the 50 samples (1e-10 per fixed-count solve, propagated through the
  loop).
* FP32 (plain iterations, so that the iterates do not depend on discrete restart decisions):
  every sample is re-solved by the oracle from exactly the GPU's inputs (its linearisation and
  its warm-start iterates) and must agree to 1e-4 on (u, x).
* The closed loop respects the input box exactly and keeps the attitudes near their box.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W
from test_gpu_parity import relerr

pytestmark = pytest.mark.gpu

KEYS = ("z", "v", "th", "be", "la")


def rti_instance(wl, ref, u_prev=None):
    inst = {k: wl[k] for k in ("nx", "nu", "N", "q", "r", "rdu", "xmin", "xmax", "umin", "umax",
                               "rho")}
    inst.update(lti=False, x0=wl["x0"].copy(), ref=ref, u_prev=u_prev)
    return inst


def quad_ref(wl, t):
    return W.quadrotor_reference(wl, t)


def hover_start(wl):
    return wl["hover_u"]


QUAD = dict(ref=quad_ref, params=lambda wl, t: wl["params"], u_init=hover_start, track_uprev=False)
CSTR = dict(ref=lambda wl, t: wl["ref"],
            params=lambda wl, t: np.append(wl["params"], W.cstr_inlet_temperature(t * wl["dt"])),
            u_init=lambda wl: wl["u_prev"], track_uprev=True)


def linearisation_point(x_meas, prev, wl, u_init):
    N = wl["N"]
    if prev is None:
        return np.tile(x_meas, (N, 1)), np.tile(u_init, (N, 1))
    u_old, x_old = prev
    xbar = np.vstack([x_meas[None, :], x_old[1:]])
    ubar = np.vstack([u_old[1:], u_old[-1:]])
    return xbar, ubar


def gpu_loop(wl, precision, accel, steps, record=None, how=QUAD):
    nx, nu, N = wl["nx"], wl["nu"], wl["N"]
    up = how["u_init"](wl).copy() if how["track_uprev"] else None
    s = pimpc.Solver([rti_instance(wl, how["ref"](wl, 0), up)], precision=precision, eps=-1.0,
                     max_iters=wl["iters"], accel=accel)
    x = wl["x0"].copy()
    prev = None
    us, xs = [], [x.copy()]
    for t in range(steps):
        prm = np.ascontiguousarray(how["params"](wl, t), np.float64)
        xbar, ubar = linearisation_point(x, prev, wl, how["u_init"](wl))
        pimpc.pimpc_linearise(s.h, wl["model"], prm, wl["dt"], xbar.ravel(), ubar.ravel())
        if record is not None:
            warm = s.iterates()[0] if t > 0 else None
            A = np.zeros(N * nx * nx); B = np.zeros(N * nx * nu); e = np.zeros(N * nx)
            pimpc.pimpc_get_dynamics(s.h, A, B, e)
        ref = how["ref"](wl, t)
        u_out = np.zeros(N * nu)
        x_out = np.zeros(N * nx)
        pimpc.pimpc_solve(s.h, x, up, ref, False, 1 if t > 0 else 0, u_out, x_out)
        u_sol, x_sol = u_out.reshape(N, nu), x_out.reshape(N, nx)
        if record is not None:
            record.append(dict(x=x.copy(), ref=ref, warm=warm, A=A.reshape(N, nx, nx),
                               B=B.reshape(N, nx, nu), e=e.reshape(N, nx), u=u_sol, xp=x_sol,
                               up=None if up is None else up.copy()))
        xn = np.zeros(nx)
        pimpc.pimpc_plant_step(s.h, wl["model"], prm, wl["dt"], x, u_sol[0].copy(), xn)
        us.append(u_sol[0].copy())
        if up is not None:
            up = u_sol[0].copy()
        x = xn
        xs.append(x.copy())
        prev = (u_sol, x_sol)
    s.close()
    return np.array(us), np.array(xs)


def oracle_loop(wl, accel, steps, how=QUAD):
    x = wl["x0"].copy()
    up = how["u_init"](wl).copy() if how["track_uprev"] else None
    prev = None
    warm = None
    us, xs = [], [x.copy()]
    for t in range(steps):
        prm = how["params"](wl, t)
        xbar, ubar = linearisation_point(x, prev, wl, how["u_init"](wl))
        A, B, e = oracle.linearise(wl["model"], prm, wl["dt"], xbar, ubar)
        inst = rti_instance(wl, how["ref"](wl, t), up)
        inst.update(A=A, B=B, e=e, x0=x.copy())
        r = oracle.solve(inst, eps=-1.0, max_iters=wl["iters"], accel=accel, warm=warm)
        warm = {k: r[k] for k in KEYS}
        us.append(r["u"][0].copy())
        if up is not None:
            up = r["u"][0].copy()
        x = oracle.plant_step(wl["model"], prm, wl["dt"], x, r["u"][0])
        xs.append(x.copy())
        prev = (r["u"], r["x"])
    return np.array(us), np.array(xs)


def test_rti_closed_loop_fp64_matches_the_oracle_loop():
    wl = W.quadrotor_rti()
    steps = wl["rti_steps"]
    gu, gx = gpu_loop(wl, pimpc.F64, 1, steps)
    ou, ox = oracle_loop(wl, 1, steps)
    assert np.all(np.isfinite(gx))
    np.testing.assert_allclose(gu, ou, rtol=0, atol=1e-8 * max(1.0, np.abs(ou).max()))
    np.testing.assert_allclose(gx, ox, rtol=0, atol=1e-8 * max(1.0, np.abs(ox).max()))
    m, g = W.QUAD_PARAMS[0], W.QUAD_PARAMS[1]
    assert gu.min() >= 0.0 and gu.max() <= 0.5 * m * g      # the input box holds exactly
    assert np.abs(gx[:, 6:9]).max() <= 0.6 + 0.05            # attitudes near their box


def test_rti_fp32_every_sample_matches_the_oracle_on_the_same_inputs():
    wl = W.quadrotor_rti()
    steps = 20
    rec = []
    gpu_loop(wl, pimpc.F32, 0, steps, record=rec)
    for t, r in enumerate(rec):
        inst = rti_instance(wl, r["ref"])
        inst.update(A=r["A"], B=r["B"], e=r["e"], x0=r["x"])
        o = oracle.solve(inst, eps=-1.0, max_iters=wl["iters"], accel=0, warm=r["warm"])
        assert relerr(r["u"], o["u"]) <= 1e-4, t
        assert relerr(r["xp"], o["x"]) <= 1e-4, t


def test_cstr_rti_closed_loop_fp64_matches_the_oracle_loop():
    """The paper's CSTR example (C_A from 8.57 towards 2 kgmol/m^3, input-increment weight,
    u_prev = the previously applied coolant temperature, time-varying inlet temperature), with a
    shorter horizon: 30 samples of 200 iterations at N = 300."""
    wl = W.cstr_nmpc(N=300)
    wl["iters"] = 200
    steps = 30
    gu, gx = gpu_loop(wl, pimpc.F64, 1, steps, how=CSTR)
    ou, ox = oracle_loop(wl, 1, steps, how=CSTR)
    assert np.all(np.isfinite(gx))
    np.testing.assert_allclose(gu, ou, rtol=0, atol=1e-8 * max(1.0, np.abs(ou).max()))
    np.testing.assert_allclose(gx, ox, rtol=0, atol=1e-8 * max(1.0, np.abs(ox).max()))
    assert gu.min() >= wl["umin"][0] and gu.max() <= wl["umax"][0]
    assert gx[-1, 0] < gx[0, 0]      # the concentration moves towards the set point
