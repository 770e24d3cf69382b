"""The oracle's AFTI-16 closed loop (the paper's first example), the counterpart of
paper_2601_14414_gb300.closed_loop.afti16_gpu_loop: same steps, solved by the FP64 oracle."""
import numpy as np

import oracle
from paper_2601_14414_gb300.closed_loop import afti16_step_instance

KEYS = ("z", "v", "th", "be", "la")


def oracle_loop(wl, steps, eps=1e-6, max_iters=10000, accel=1):
    x = wl["x0"].copy()
    up = wl["u_prev"].copy()
    warm = None
    us, xs, its = [], [x.copy()], []
    for t in range(steps):
        r = oracle.solve(afti16_step_instance(wl, x, up, t), eps=eps, max_iters=max_iters,
                         accel=accel, warm=warm)
        warm = {k: r[k] for k in KEYS}
        up = r["u"][0].copy()
        its.append(r["iters"])
        us.append(up.copy())
        x = wl["A"] @ x + wl["B"] @ up
        xs.append(x.copy())
    return np.array(us), np.array(xs), np.array(its)
