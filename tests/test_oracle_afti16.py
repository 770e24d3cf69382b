"""AFTI-16 sanity run of the paper's first example on the oracle (CPU).

The paper prints the continuous model, the ZOH sampling time, the bounds, the weights and N, and
reports about 2030 iterations per MPC step on average to reach a residual of 1e-6 over 200 steps;
it prints neither rho nor the pitch reference, so that count cannot be reproduced exactly (parity
unpinned): this test checks the discretisation against a library matrix exponential, that the
closed loop respects every bound and follows the reference, and that the mean iteration count is
of the paper's order (within a factor of three).
"""
import numpy as np
import scipy.linalg

from afti16_loop import oracle_loop
from paper_2601_14414_gb300 import workloads as W


def test_zoh_matches_the_matrix_exponential():
    dt = 0.05
    A, B = W.zoh(W.AFTI16_AC, W.AFTI16_BC, dt)
    M = np.zeros((6, 6))
    M[:4, :4] = W.AFTI16_AC
    M[:4, 4:] = W.AFTI16_BC
    E = scipy.linalg.expm(M * dt)
    np.testing.assert_allclose(A, E[:4, :4], rtol=0, atol=1e-12)
    np.testing.assert_allclose(B, E[:4, 4:], rtol=0, atol=1e-12)
    assert np.max(np.abs(np.linalg.eigvals(A))) > 1.0  # the open loop is unstable


def test_afti16_closed_loop_on_the_oracle():
    wl = W.afti16()
    us, xs, its = oracle_loop(wl, wl["steps"])
    assert np.abs(us).max() <= 25.0 + 1e-9                 # |u_i| <= 25 degrees
    assert np.abs(xs[1:, 1]).max() <= 0.5 + 1e-3            # |y_1| <= 0.5 (z is in the box)
    half = wl["period"] // 2
    for h in range(wl["steps"] // half):
        r = W.afti16_reference(wl, h * half)[3]
        seg = xs[h * half + 1:(h + 1) * half + 1, 3]
        assert np.sign(seg[-1]) == np.sign(r)                 # y_2 follows each reference phase
        assert abs(seg[-1] - r) < abs(seg[0] - r)
    assert 2030 / 3 <= its.mean() <= 2030 * 3, its.mean()
