"""pimpc_solve_static (the entry point that allocates no device memory) against pimpc_solve.

Callers that cannot call cudaMalloc (real-time control loops that forbid allocation after
start-up, controllers certified without dynamic memory, plug-ins whose host owns the device
allocator) use pimpc_solve_static, which keeps its working memory in a fixed device array inside
the library. Its results must equal those of the allocating entry point within the parity
tolerances of the other GPU tests (1e-10 in FP64, 1e-4 on u and x in FP32), on two calls in a
row (the second call reuses the array the first one left behind). This file is collected last.
"""
import numpy as np
import pytest

from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def relerr(a, b):
    return float(np.max(np.abs(a - b)) / max(np.max(np.abs(b)), 1e-12))


def run_static(inst, precision, eps, max_iters, accel):
    import torch
    dev = torch.device("cuda")

    def t(a):
        if a is None:
            return None
        return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float64).ravel()).to(dev)
    nx, nu, N = inst["nx"], inst["nu"], inst["N"]
    u = torch.zeros(N * nu, dtype=torch.float64, device=dev)
    x = torch.zeros(N * nx, dtype=torch.float64, device=dev)
    it = torch.zeros(1, dtype=torch.int32, device=dev)
    c = torch.zeros(1, dtype=torch.float64, device=dev)
    st = torch.zeros(1, dtype=torch.int32, device=dev)
    pimpc.pimpc_solve_static(nx, nu, N, precision, t(inst["A"]), t(inst["B"]), t(inst["e"]),
                             t(inst["q"]), t(inst["r"]), t(inst["xmin"]), t(inst["xmax"]),
                             t(inst["umin"]), t(inst["umax"]), t(inst["x0"]), t(inst["ref"]),
                             inst["rho"], eps, max_iters, accel, 0.999, u, x, it, c, st)
    torch.cuda.synchronize()
    return (u.cpu().numpy().reshape(N, nu), x.cpu().numpy().reshape(N, nx), int(it.item()),
            float(c.item()), int(st.item()))


def run_allocating(inst, precision, eps, max_iters, accel):
    s = pimpc.Solver([inst], precision=precision, eps=eps, max_iters=max_iters, accel=accel)
    r = s.solve()
    s.close()
    return r["u"][0], r["x"][0], int(r["iters"][0]), float(r["c"][0]), int(r["status"][0])


def test_static_entry_point_matches_allocating_one_twice_in_a_row():
    first = W.random_ltv(501, 9, 3, 150)     # two work items: exercises the item halo
    second = W.random_ltv(502, 14, 5, 37)    # different sizes, reusing the same array
    for inst, (eps, iters, accel) in ((first, (1e-7, 3000, 1)), (second, (-1.0, 120, 0))):
        us, xs, its, cs, sts = run_static(inst, pimpc.F64, eps, iters, accel)
        ua, xa, ita, ca, sta = run_allocating(inst, pimpc.F64, eps, iters, accel)
        assert relerr(us, ua) <= 1e-10
        assert relerr(xs, xa) <= 1e-10
        assert its == ita and sts == sta
        assert abs(cs - ca) <= 1e-8 * ca + 1e-24


def test_static_entry_point_rejects_instances_larger_than_its_array():
    inst = W.random_ltv(503, 24, 8, 4000)  # needs far more than PIMPC_STATIC_BYTES
    with pytest.raises(pimpc.PimpcError) as e:
        run_static(inst, pimpc.F64, 1e-6, 10, 1)
    assert e.value.code == pimpc.EINVAL
    assert "static array" in str(e.value)


def test_static_entry_point_fp32_matches_allocating_one_twice_in_a_row():
    # FP32 iterations (one thread per stage on the tiled layout) at a fixed iteration count of
    # the plain iteration, so that no discrete restart decision can differ: a nonzero constant
    # reference, and one call without the affine term e (NULL = 0).
    first = W.random_ltv(511, 8, 3, 100)
    first["ref"] = np.linspace(-0.8, 0.9, first["nx"] + first["nu"])
    second = W.random_ltv(512, 12, 4, 45)
    second["ref"] = np.full(second["nx"] + second["nu"], 0.3)
    second["e"] = None
    for inst in (first, second):
        us, xs, its, _, _ = run_static(inst, pimpc.F32, -1.0, 150, 0)
        alloc = dict(inst)
        if alloc["e"] is None:
            alloc["e"] = np.zeros((inst["N"], inst["nx"]))
        ua, xa, ita, _, _ = run_allocating(alloc, pimpc.F32, -1.0, 150, 0)
        assert its == ita == 150
        assert relerr(us, ua) <= 1e-4
        assert relerr(xs, xa) <= 1e-4
        assert np.max(np.abs(xs)) > 1e-3  # the reference moved the solution away from zero
