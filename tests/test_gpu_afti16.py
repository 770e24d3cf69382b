"""AFTI-16 closed loop (the paper's first example) on the GPU against the oracle's loop.

FP64: 200 MPC steps, each solved to c <= 1e-6 from the previous step's iterates; the GPU loop and
the oracle loop run independently and must take the same number of iterations at every step and
apply the same inputs to 1e-8. FP32: the loop stays within the bounds and its inputs stay within
1e-3 (relative to the 25-degree input range) of the oracle loop's.
"""
import numpy as np
import pytest

from afti16_loop import oracle_loop
from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300.closed_loop import afti16_gpu_loop
from paper_2601_14414_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def test_afti16_fp64_loop_matches_the_oracle_loop():
    wl = W.afti16()
    steps = wl["steps"]
    gu, gx, gi, _ = afti16_gpu_loop(wl, steps, pimpc.F64)
    ou, ox, oi = oracle_loop(wl, steps)
    np.testing.assert_array_equal(gi, oi)
    np.testing.assert_allclose(gu, ou, rtol=0, atol=1e-8 * 25.0)
    np.testing.assert_allclose(gx, ox, rtol=0, atol=1e-8 * max(1.0, np.abs(ox).max()))


def test_afti16_fp32_loop_stays_feasible_and_close():
    wl = W.afti16()
    steps = 60
    gu, gx, gi, _ = afti16_gpu_loop(wl, steps, pimpc.F32)
    ou, ox, oi = oracle_loop(wl, steps)
    assert np.abs(gu).max() <= 25.0 + 1e-6
    assert np.abs(gx[1:, 1]).max() <= 0.5 + 1e-3
    assert np.abs(gu - ou).max() <= 1e-3 * 25.0
