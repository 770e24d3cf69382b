"""Sampled parity at the full sizes of the workloads, in the launch configuration of the bench.

The oracle cannot solve thousands of instances in a test, so each test solves the whole batch on
the GPU and compares a sample of instances (chosen by a fixed seed, plus the largest and the
smallest) with the oracle, at the tolerances of the smaller parity tests: FP64 1e-10 and FP32
1e-4 (relative, on u and x) at a fixed iteration count, and for the adjoint the oracle's central
finite differences (FP32 iterations: 1e-4 of max(1, |gradient|) after 150 iterations).
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import configs as C
from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W
from test_gpu_parity import relerr

pytestmark = pytest.mark.gpu


def sample(insts, count, seed=0):
    sizes = [i["N"] * (i["nx"] + i["nu"]) ** 2 for i in insts]
    rng = np.random.default_rng(seed)
    pick = set(rng.choice(len(insts), count, replace=False).tolist())
    pick |= {int(np.argmax(sizes)), int(np.argmin(sizes))}
    return sorted(pick)


@pytest.fixture(scope="module")
def batched():
    cfg = C.BATCHED_UNEVEN
    return W.batched_uneven(seed=cfg["seed"], batch=cfg["batch"])


def test_batched_uneven_full_size_plain(batched):
    s = pimpc.Solver(batched, precision=pimpc.F32, eps=-1.0, max_iters=30, accel=0)
    res = s.solve()
    for j in sample(batched, 8):
        o = oracle.solve(batched[j], eps=-1.0, max_iters=30, accel=0)
        assert relerr(res["u"][j], o["u"]) <= 1e-4, j
        assert relerr(res["x"][j], o["x"]) <= 1e-4, j
    s.close()


def test_batched_uneven_full_size_accelerated(batched):
    """The bench's options (accelerated iteration, rho = 1) for a fixed count, with the oracle's
    restart decisions replayed for the sampled instances."""
    cfg = C.BATCHED_UNEVEN
    K = 40
    picks = sample(batched, 6, seed=1)
    mask = np.ones((len(batched), K), np.uint8)
    ora = {}
    for j in picks:
        ora[j] = oracle.solve(batched[j], eps=-1.0, max_iters=K, accel=1, eta=cfg["eta"],
                              history=True)
        mask[j] = ora[j]["mask"]
    s = pimpc.Solver(batched, precision=pimpc.F32, eps=-1.0, max_iters=K, accel=1, eta=cfg["eta"])
    pimpc.pimpc_set_restart_mask(s.h, np.ascontiguousarray(mask), K)
    res = s.solve()
    for j in picks:
        assert relerr(res["u"][j], ora[j]["u"]) <= 1e-4, j
        assert relerr(res["x"][j], ora[j]["x"]) <= 1e-4, j
    s.close()


def cartpole_dynamics(inst):
    A, B, e = oracle.linearise(W.MODEL_CARTPOLE, inst["params"], inst["dt"], inst["op_x"][None, :],
                               inst["op_u"][None, :])
    return dict(inst, A=A[0], B=B[0], e=e[0])


def test_differentiable_cartpole_full_size():
    """1024 cart-pole instances (N = 100), 150 plain FP32 iterations, checkpoints every 25; the
    model is linearised at the upright equilibrium by the solver's own linearisation."""
    insts = W.cartpole_batch()
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=150, accel=0)
    prm = np.ascontiguousarray(np.concatenate([i["params"] for i in insts]))
    xbar = np.ascontiguousarray(np.concatenate([i["op_x"] for i in insts]))
    ubar = np.ascontiguousarray(np.concatenate([i["op_u"] for i in insts]))
    pimpc.pimpc_linearise(s.h, W.MODEL_CARTPOLE, prm, insts[0]["dt"], xbar, ubar)
    res = s.solve()
    rng = np.random.default_rng(7)
    Wu = [rng.standard_normal((i["N"], i["nu"])) for i in insts]
    Wx = [rng.standard_normal((i["N"], i["nx"])) for i in insts]
    g = s.backward(Wu, Wx, checkpoint_every=25)
    for j in sample(insts, 2, seed=2):
        inst = cartpole_dynamics(insts[j])
        o = oracle.solve(inst, eps=-1.0, max_iters=150, accel=0)
        assert relerr(res["u"][j], o["u"]) <= 1e-4
        for name in ("x0", "q", "r", "umin", "umax", "ref"):
            fd = oracle.fd_gradient(inst, Wu[j], Wx[j], 150, name, h=1e-6)
            if name == "ref":
                fd = fd.sum(axis=0)          # one constant reference per instance
            got = np.asarray(g[name][j]).reshape(fd.shape)
            assert np.max(np.abs(got - fd)) <= 1e-4 * max(1.0, float(np.max(np.abs(fd)))), (j, name)
    s.close()


@pytest.mark.parametrize("precision,tol", [(pimpc.F64, 1e-10), (pimpc.F32, 1e-4)])
def test_large_state_lti_full_size(precision, tol):
    """256 instances with nx = 48, nu = 16 (n = 64, two components per lane) and N = 1000."""
    insts = W.large_lti()
    s = pimpc.Solver(insts, precision=precision, eps=-1.0, max_iters=20, accel=0)
    res = s.solve()
    for j in (0, 97, 255):
        o = oracle.solve(insts[j], eps=-1.0, max_iters=20, accel=0)
        assert relerr(res["u"][j], o["u"]) <= tol, j
        assert relerr(res["x"][j], o["x"]) <= tol, j
    s.close()
