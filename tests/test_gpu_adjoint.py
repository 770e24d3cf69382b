"""Reverse mode of the unrolled iteration (pimpc_backward) against the FP64 oracle.

The oracle side is the central finite difference (h = 1e-6) of the oracle's unrolled map, whose
own pins (tests/test_oracle_gradients.py) tie it to the implicit derivative of the KKT system.
The GPU side is the exact derivative of the same unrolled map, so in FP64 the two agree to the
finite-difference error (about 1e-9 here); the test allows 1e-6 of max(1, |gradient|). FP32
iterations change the unrolled map itself by rounding (unit roundoff 6e-8, amplified over 40
iterations; measured at most 9e-7 of max(1, |gradient|) on these fixtures); the bound there is
1e-5.
The fixtures were chosen with no clamp argument within the finite-difference step of a bound.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W
from test_oracle_pins import tiny_ltv

pytestmark = pytest.mark.gpu

NAMES = ("x0", "q", "r", "ref", "xmin", "xmax", "umin", "umax")


def small_batch():
    insts = [tiny_ltv(3, nx=3, nu=2, N=6, xabs=1.0, uabs=0.3, ref_scale=1.0, x0_abs=0.8),
             tiny_ltv(12, nx=4, nu=2, N=9, xabs=1.2, uabs=0.4, rdu=True, ref_scale=0.5,
                      x0_abs=1.0),
             tiny_ltv(5, nx=3, nu=2, N=6, xabs=1.0, uabs=0.3, rdu=True, ref_scale=1.0, x0_abs=0.8)]
    for inst in insts:      # one solver object has one rho
        inst["rho"] = 1.3
    return insts


def as_oracle_shape(got, ref_fd, name, inst):
    """The GPU returns one gradient per reference entry it was given: a constant reference gets
    the sum over stages of the per-stage finite differences."""
    if name == "ref" and np.ndim(inst["ref"]) == 1:
        return np.asarray(got), ref_fd.sum(axis=0)
    return np.asarray(got).reshape(ref_fd.shape), ref_fd


def loss_weights(insts, seed=0):
    rng = np.random.default_rng(seed)
    return ([rng.standard_normal((i["N"], i["nu"])) for i in insts],
            [rng.standard_normal((i["N"], i["nx"])) for i in insts])


def gpu_gradients(insts, precision, iters, K, Wu, Wx):
    s = pimpc.Solver(insts, precision=precision, eps=-1.0, max_iters=iters, accel=0)
    s.solve()
    g = s.backward(Wu, Wx, checkpoint_every=K)
    s.close()
    return g


def fd(inst, Wu, Wx, iters, name):
    return oracle.fd_gradient(inst, Wu, Wx, iters, name, h=1e-6)


@pytest.mark.parametrize("K", [7])
def test_adjoint_matches_oracle_finite_differences_fp64(K):
    insts = small_batch()
    Wu, Wx = loss_weights(insts)
    iters = 40
    g = gpu_gradients(insts, pimpc.F64, iters, K, Wu, Wx)
    active = set()
    for j, inst in enumerate(insts):
        for name in NAMES:
            ref = fd(inst, Wu[j], Wx[j], iters, name)
            got = np.asarray(g[name][j]).reshape(ref.shape)
            tol = 1e-6 * max(1.0, float(np.max(np.abs(ref))))
            assert np.max(np.abs(got - ref)) <= tol, (j, name, np.max(np.abs(got - ref)))
            if np.max(np.abs(ref)) > 0 and name in ("xmin", "xmax", "umin", "umax"):
                active.add(name)
    assert {"xmin", "xmax", "umin", "umax"} <= active, "fixtures must exercise every bound"


def test_checkpoint_spacing_does_not_change_the_gradient():
    insts = small_batch()
    Wu, Wx = loss_weights(insts, seed=1)
    iters = 40
    base = gpu_gradients(insts, pimpc.F64, iters, 1000, Wu, Wx)
    for K in (1, 3, 13, 40):
        g = gpu_gradients(insts, pimpc.F64, iters, K, Wu, Wx)
        for name in NAMES:
            for a, b in zip(g[name], base[name]):
                assert np.array_equal(a, b), (K, name)


def test_adjoint_fp32_iterations():
    insts = small_batch()
    Wu, Wx = loss_weights(insts, seed=2)
    iters = 40
    g = gpu_gradients(insts, pimpc.F32, iters, 10, Wu, Wx)
    for j, inst in enumerate(insts):
        for name in NAMES:
            ref = fd(inst, Wu[j], Wx[j], iters, name)
            got = np.asarray(g[name][j]).reshape(ref.shape)
            tol = 1e-5 * max(1.0, float(np.max(np.abs(ref))))
            assert np.max(np.abs(got - ref)) <= tol, (j, name, np.max(np.abs(got - ref)))


def test_adjoint_long_horizon_stage_invariant():
    """N = 300 > threads per CTA (every thread handles two stages), constant reference."""
    inst = W.plain_lti(seed=1, nx=4, nu=2, N=300)
    inst["ref"] = np.random.default_rng(9).uniform(-1, 1, 6)
    Wu, Wx = loss_weights([inst], seed=3)
    iters = 30
    g = gpu_gradients([inst], pimpc.F64, iters, 8, Wu, Wx)
    for name in ("x0", "q", "r", "ref", "umax", "umin"):
        got, ref = as_oracle_shape(g[name][0], fd(inst, Wu[0], Wx[0], iters, name), name, inst)
        tol = 1e-6 * max(1.0, float(np.max(np.abs(ref))))
        assert np.max(np.abs(got - ref)) <= tol, (name, np.max(np.abs(got - ref)))


def test_autograd_function_matches_the_host_backward():
    import torch
    from paper_2601_14414_gb300.autograd import unrolled_solve
    insts = small_batch()
    Wu, Wx = loss_weights(insts, seed=4)
    iters = 25
    host = gpu_gradients(insts, pimpc.F64, iters, 6, Wu, Wx)
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=iters, accel=0)
    dev = torch.device("cuda")
    t = lambda a: torch.tensor(np.asarray(a, np.float64), device=dev, requires_grad=True)
    p = s.p
    args = [t(p[k]) for k in ("x0", "ref", "q", "r", "xmin", "xmax", "umin", "umax")]
    u, x = unrolled_solve(s, iters, *args, checkpoint_every=6)
    loss = (torch.tensor(np.concatenate([w.ravel() for w in Wu]), device=dev) * u).sum() + \
           (torch.tensor(np.concatenate([w.ravel() for w in Wx]), device=dev) * x).sum()
    loss.backward()
    for name, a in zip(("x0", "ref", "q", "r", "xmin", "xmax", "umin", "umax"), args):
        want = np.concatenate([np.ravel(v) for v in host[name]])
        assert np.array_equal(a.grad.cpu().numpy(), want), name
    # the forward outputs are the solve's outputs
    r = s.solve()
    assert np.array_equal(u.detach().cpu().numpy(), np.concatenate([v.ravel() for v in r["u"]]))
    s.close()


def test_backward_needs_a_fixed_plain_cold_solve():
    insts = small_batch()[:1]
    Wu, Wx = loss_weights(insts)
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=1e-8, max_iters=50, accel=1)
    with pytest.raises(pimpc.PimpcError) as e:
        s.backward(Wu, Wx)          # no solve yet
    assert e.value.code == pimpc.ESTATE
    s.solve()
    with pytest.raises(pimpc.PimpcError) as e:
        s.backward(Wu, Wx)          # accelerated, tolerance-stopped
    assert e.value.code == pimpc.ESTATE
    s.set_options(-1.0, 20, 0)
    s.solve()
    with pytest.raises(pimpc.PimpcError) as e:
        s.backward(Wu, Wx, checkpoint_every=0)
    assert e.value.code == pimpc.EINVAL
    s.close()
