"""Closed-loop drivers of the paper's linear example (AFTI-16, Sec. V-A) on the library.

Driver code only: every solve goes through the C ABI (pimpc_solve); the plant step of this
linear example is the discrete model itself, x <- A x + B u_0, evaluated here on the host.
Every MPC step solves Algorithm 1 to c <= eps from the previous step's iterates (warm start),
with u_prev = the input applied at the previous step (the W_du term of the example).
"""
from __future__ import annotations

import time

import numpy as np

from . import pimpc
from . import workloads as W


def afti16_step_instance(wl, x, u_prev, t):
    inst = {k: wl[k] for k in ("nx", "nu", "N", "lti", "A", "B", "e", "q", "r", "rdu", "xmin",
                               "xmax", "umin", "umax", "rho")}
    inst.update(x0=x.copy(), u_prev=u_prev.copy(), ref=W.afti16_reference(wl, t))
    return inst


def afti16_gpu_loop(wl, steps, precision, eps=1e-6, max_iters=10000, accel=1, family=None):
    """Returns applied inputs [steps, nu], states [steps + 1, nx], iterations [steps] and the
    wall seconds of the solves (host-memory calls, each synchronising)."""
    x = wl["x0"].copy()
    up = wl["u_prev"].copy()
    s = pimpc.Solver([afti16_step_instance(wl, x, up, 0)], precision=precision, eps=eps,
                     max_iters=max_iters, accel=accel)
    if family is not None:
        s.set_schedule(family)
    N, nx, nu = wl["N"], wl["nx"], wl["nu"]
    us, xs, its = [], [x.copy()], []
    u_out, x_out = np.zeros(N * nu), np.zeros(N * nx)
    it, st = np.zeros(1, np.int32), np.zeros(1, np.int32)
    secs = 0.0
    for t in range(steps):
        t0 = time.perf_counter()
        pimpc.pimpc_solve(s.h, x, up, W.afti16_reference(wl, t), False, 1 if t > 0 else 0,
                          u_out, x_out, it, None, st)
        secs += time.perf_counter() - t0
        up = u_out[:nu].copy()
        its.append(int(it[0]))
        us.append(up.copy())
        x = wl["A"] @ x + wl["B"] @ up
        xs.append(x.copy())
    s.close()
    return np.array(us), np.array(xs), np.array(its), secs
