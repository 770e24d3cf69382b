"""Schedules of the batched solve (pimpc_set_schedule / pimpc_autotune) against the FP64 oracle.

Every schedule computes the same iteration: the one-thread-per-stage kernel on halo tiles
(family 2) must meet the FP32 tolerances of the lane-group kernel (1e-4 on u, x at a fixed
iteration count, 1e-5 on converged solutions); different item sizes of the lane-group kernel
change only the order of the sums of c. The batches cover tiles of 32 and 16 slots, instances
of one tile, several tiles with a ragged last tile, and N = 1.
"""
import numpy as np
import pytest

import oracle
from paper_2601_14414_gb300 import pimpc
from paper_2601_14414_gb300 import workloads as W
from test_gpu_parity import RAGGED, ragged_batch, relerr, solution_error

pytestmark = pytest.mark.gpu

TILE_DIMS = RAGGED + [(24, 8, 45), (3, 2, 95), (2, 1, 2)]


def tiles_solver(insts, **kw):
    s = pimpc.Solver(insts, precision=pimpc.F32, **kw)
    s.set_schedule(pimpc.FAMILY_TILES)
    assert s.schedule()["family"] == pimpc.FAMILY_TILES
    return s


def test_halo_tiles_plain_fixed_iterations_match_oracle():
    insts = ragged_batch(21, dims=TILE_DIMS)
    s = tiles_solver(insts, eps=-1.0, max_iters=200, accel=0)
    res = s.solve()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=200, accel=0)
    for j, o in enumerate(ora):
        assert relerr(res["u"][j], o["u"]) <= 1e-4, j
        assert relerr(res["x"][j], o["x"]) <= 1e-4, j
        assert res["iters"][j] == 200


def test_halo_tiles_accel_with_replayed_restarts_matches_oracle():
    insts = ragged_batch(22, dims=TILE_DIMS)
    K = 200
    ora = [oracle.solve(i, eps=-1.0, max_iters=K, accel=1, history=True) for i in insts]
    mask = np.ascontiguousarray(np.stack([o["mask"] for o in ora]).astype(np.uint8))
    s = tiles_solver(insts, eps=-1.0, max_iters=K, accel=1)
    pimpc.pimpc_set_restart_mask(s.h, mask, K)
    res = s.solve()
    for j, o in enumerate(ora):
        assert relerr(res["u"][j], o["u"]) <= 1e-4, j
        assert relerr(res["x"][j], o["x"]) <= 1e-4, j


def test_halo_tiles_converged_match_converged_oracle():
    insts = ragged_batch(23, dims=[(4, 2, 37), (14, 2, 19), (12, 4, 33), (6, 2, 1), (24, 8, 45)])
    s = tiles_solver(insts, eps=1e-11, max_iters=20000, accel=1)
    res = s.solve()
    ora = oracle.solve_batch(insts, eps=1e-22, max_iters=200000, accel=1)
    for j, o in enumerate(ora):
        assert o["status"] == oracle.CONVERGED
        assert solution_error(res["u"][j], res["x"][j], o["u"], o["x"]) <= 1e-5, j


@pytest.mark.parametrize("mode", [1, 2])
def test_halo_tiles_warm_start(mode):
    """Warm start reuses (1) or shifts (2) the iterates; the shifted copy must also refresh the
    halo slots of the neighbouring tiles."""
    insts = ragged_batch(24, dims=[(4, 2, 70), (24, 8, 45), (14, 2, 19)])
    s = tiles_solver(insts, eps=-1.0, max_iters=60, accel=0)
    s.solve()
    first = s.iterates()
    res = s.solve(warm_start=mode)
    for j, inst in enumerate(insts):
        warm = {k: first[j][k].copy() for k in ("z", "v", "th", "be", "la")}
        if mode == 2:
            for k in warm:
                warm[k] = np.concatenate([warm[k][1:], warm[k][-1:]], axis=0)
        o = oracle.solve(inst, eps=-1.0, max_iters=60, accel=0, warm=warm)
        assert relerr(res["u"][j], o["u"]) <= 1e-4, j
        assert relerr(res["x"][j], o["x"]) <= 1e-4, j


def test_lane_group_item_sizes_agree():
    insts = ragged_batch(25)
    b = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=120, accel=1)
    b.set_schedule(pimpc.FAMILY_LANES)
    base = b.solve()
    for scale in (1, 3, 40):
        s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=120, accel=1)
        s.set_schedule(pimpc.FAMILY_LANES, 0, scale)
        r = s.solve()
        for j in range(len(insts)):
            assert relerr(r["u"][j], base["u"][j]) <= 1e-5
            assert relerr(r["x"][j], base["x"][j]) <= 1e-5


def test_schedule_errors_keep_the_previous_schedule():
    insts = ragged_batch(26, dims=[(4, 2, 37)])
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=50, accel=0)
    before = s.schedule()
    with pytest.raises(pimpc.PimpcError) as e:
        s.set_schedule(pimpc.FAMILY_TILES)        # halo tiles are FP32 only
    assert e.value.code == pimpc.EINVAL
    assert s.schedule() == before
    with pytest.raises(pimpc.PimpcError):
        s.set_schedule(8)                         # no such family
    with pytest.raises(pimpc.PimpcError):
        s.set_schedule(6)                         # tensor cores: stage-invariant FP32 only
    assert s.schedule() == before
    o = oracle.solve(insts[0], eps=-1.0, max_iters=50, accel=0)
    r = s.solve()
    assert relerr(r["u"][0], o["u"]) <= 1e-10


def test_autotune_picks_a_schedule_that_solves_correctly(tmp_path):
    insts = ragged_batch(27, dims=TILE_DIMS)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=150, accel=0)
    pick = s.autotune(trial_iters=10, cache=str(tmp_path / "tune.json"))
    assert pick["family"] in (pimpc.FAMILY_LANES, pimpc.FAMILY_TILES, pimpc.FAMILY_RESIDENT,
                              pimpc.FAMILY_BLOCKED, pimpc.FAMILY_TEMPORAL) and pick["ms"] > 0
    assert s.schedule()["family"] == pick["family"] and not pick["cached"]
    again = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=150, accel=0)
    assert again.autotune(cache=str(tmp_path / "tune.json"))["cached"]
    res = s.solve()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=150, accel=0)
    for j, o in enumerate(ora):
        assert relerr(res["u"][j], o["u"]) <= 1e-4
        assert relerr(res["x"][j], o["x"]) <= 1e-4


def test_adjoint_on_halo_tiles():
    from test_gpu_adjoint import NAMES, fd, loss_weights, small_batch
    insts = small_batch()
    Wu, Wx = loss_weights(insts, seed=2)
    s = tiles_solver(insts, eps=-1.0, max_iters=40, accel=0)
    s.solve()
    g = s.backward(Wu, Wx, checkpoint_every=10)
    for j, inst in enumerate(insts):
        for name in NAMES:
            ref = fd(inst, Wu[j], Wx[j], 40, name)
            got = np.asarray(g[name][j]).reshape(ref.shape)
            assert np.max(np.abs(got - ref)) <= 1e-5 * max(1.0, float(np.max(np.abs(ref)))), name


# ---- CUDA graphs of device-memory solves ----------------------------------------------------

def device_solve(s, dev_args):
    x0, up, ref, u, x, it, c, st = dev_args
    pimpc.pimpc_solve(s.h, x0, up, ref, s.p["ref_per_stage"], 0, u, x, it, c, st)


def test_graph_replays_give_the_direct_results():
    import torch
    insts = ragged_batch(41)
    dev = torch.device("cuda")
    t = lambda a: None if a is None else torch.from_numpy(np.asarray(a, np.float64)).to(dev)
    eager = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=100, accel=0)
    graph = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=100, accel=0)
    pimpc.pimpc_set_graph(graph.h, 1)
    p = eager.p
    outs = lambda: (torch.zeros(int(np.sum(eager.N * eager.nu)), dtype=torch.float64, device=dev),
                    torch.zeros(int(np.sum(eager.N * eager.nx)), dtype=torch.float64, device=dev),
                    torch.zeros(eager.batch, dtype=torch.int32, device=dev),
                    torch.zeros(eager.batch, dtype=torch.float64, device=dev),
                    torch.zeros(eager.batch, dtype=torch.int32, device=dev))
    ins = (t(p["x0"]), t(p["u_prev"]), t(p["ref"]))
    a = ins + outs()
    g = ins + outs()
    device_solve(eager, a)
    for rep in range(3):
        g[3].zero_()
        device_solve(graph, g)
        torch.cuda.synchronize()
        assert torch.equal(a[3], g[3]) and torch.equal(a[4], g[4]) and torch.equal(a[5], g[5])
    stats = pimpc.pimpc_get_graph_stats(graph.h)
    assert stats["refused"] is None, stats
    assert stats["enabled"] and stats["captures"] == 1 and stats["replays"] == 2
    # new options drop the graph; the next call records a new one
    graph.set_options(-1.0, 60, 0)
    eager.set_options(-1.0, 60, 0)
    device_solve(eager, a)
    device_solve(graph, g)
    torch.cuda.synchronize()
    assert torch.equal(a[3], g[3]) and pimpc.pimpc_get_graph_stats(graph.h)["captures"] == 2


def test_graph_with_polish_and_accel():
    import torch
    insts = ragged_batch(42, dims=[(4, 2, 37), (14, 2, 19), (24, 8, 45)])
    dev = torch.device("cuda")
    t = lambda a: None if a is None else torch.from_numpy(np.asarray(a, np.float64)).to(dev)
    ref = oracle.solve_batch(insts, eps=1e-22, max_iters=200000, accel=1)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=1e-8, max_iters=20000, accel=1)
    s.set_polish(200000, 1e-22)
    pimpc.pimpc_set_graph(s.h, 1)
    p = s.p
    u = torch.zeros(int(np.sum(s.N * s.nu)), dtype=torch.float64, device=dev)
    x = torch.zeros(int(np.sum(s.N * s.nx)), dtype=torch.float64, device=dev)
    st = torch.zeros(s.batch, dtype=torch.int32, device=dev)
    x0d = t(p["x0"])
    for rep in range(2):
        u.zero_()
        x.zero_()
        pimpc.pimpc_solve(s.h, x0d, None, None, False, 0, u, x, None, None, st)
        torch.cuda.synchronize()
        assert (st.cpu().numpy() == pimpc.CONVERGED).all()
        us = pimpc.split(u.cpu().numpy(), s.N * s.nu)
        xs = pimpc.split(x.cpu().numpy(), s.N * s.nx)
        for j, o in enumerate(ref):
            assert solution_error(us[j], xs[j], o["u"], o["x"]) <= 1e-9
    stats = pimpc.pimpc_get_graph_stats(s.h)
    assert stats["refused"] is None and stats["captures"] == 1 and stats["replays"] == 1


# ---- every instance resident on chip (one CTA or a cluster per instance) -------------------

SMALL_DIMS = [(4, 2, 20), (3, 1, 1), (6, 2, 9), (12, 4, 33), (5, 3, 17), (9, 9, 12)]


def resident_solver(insts, precision, cluster=0, **kw):
    s = pimpc.Solver(insts, precision=precision, **kw)
    s.set_schedule(pimpc.FAMILY_RESIDENT, 0, cluster)
    assert s.schedule()["family"] == pimpc.FAMILY_RESIDENT
    return s


@pytest.mark.parametrize("accel", [0, 1])
def test_resident_fp64_matches_oracle(accel):
    insts = ragged_batch(51, dims=SMALL_DIMS)
    s = resident_solver(insts, pimpc.F64, eps=-1.0, max_iters=200, accel=accel)
    res = s.solve()
    its = s.iterates()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=200, accel=accel)
    for j, o in enumerate(ora):
        for key in ("z", "v", "th", "be", "la"):
            assert relerr(its[j][key], o[key]) <= 1e-10, (j, key)
        assert relerr(res["u"][j], o["u"]) <= 1e-10
        assert res["iters"][j] == 200 and res["status"][j] == pimpc.MAXITER
        assert abs(res["c"][j] - o["c"]) <= 1e-8 * o["c"] + 1e-24


@pytest.mark.parametrize("cluster", [2, 4, 8, 16])
def test_resident_clusters_match_oracle(cluster):
    """Instances split over clusters of 2..16 CTAs: the boundary stages cross CTAs through
    distributed shared memory (N not a multiple of the cluster size)."""
    insts = ragged_batch(52 + cluster, dims=[(12, 4, 61), (4, 2, 37), (24, 8, 19), (7, 3, 16)])
    s = resident_solver(insts, pimpc.F64, cluster, eps=-1.0, max_iters=150, accel=1)
    res = s.solve()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=150, accel=1)
    for j, o in enumerate(ora):
        assert relerr(res["u"][j], o["u"]) <= 1e-10, j
        assert relerr(res["x"][j], o["x"]) <= 1e-10, j


def test_resident_fp32_and_converged():
    insts = ragged_batch(53, dims=SMALL_DIMS)
    K = 200
    ora = [oracle.solve(i, eps=-1.0, max_iters=K, accel=1, history=True) for i in insts]
    mask = np.ascontiguousarray(np.stack([o["mask"] for o in ora]).astype(np.uint8))
    s = resident_solver(insts, pimpc.F32, eps=-1.0, max_iters=K, accel=1)
    pimpc.pimpc_set_restart_mask(s.h, mask, K)
    res = s.solve()
    for j, o in enumerate(ora):
        assert relerr(res["u"][j], o["u"]) <= 1e-4, j
        assert relerr(res["x"][j], o["x"]) <= 1e-4, j
    conv = ragged_batch(4, dims=[(4, 2, 37), (14, 2, 19), (12, 4, 33), (6, 2, 1), (9, 9, 17)])
    c = resident_solver(conv, pimpc.F32, eps=1e-11, max_iters=20000, accel=1)
    r = c.solve()
    oc = oracle.solve_batch(conv, eps=1e-22, max_iters=200000, accel=1)
    for j, o in enumerate(oc):
        assert solution_error(r["u"][j], r["x"][j], o["u"], o["x"]) <= 1e-5, j


@pytest.mark.parametrize("mode", [1, 2])
def test_resident_warm_start(mode):
    insts = ragged_batch(54, dims=[(4, 2, 37), (12, 4, 33)])
    s = resident_solver(insts, pimpc.F64, 2, eps=-1.0, max_iters=60, accel=1)
    s.solve()
    first = s.iterates()
    s.solve(warm_start=mode)
    its = s.iterates()
    for j, inst in enumerate(insts):
        warm = {k: first[j][k].copy() for k in ("z", "v", "th", "be", "la")}
        if mode == 2:
            for k in warm:
                warm[k] = np.concatenate([warm[k][1:], warm[k][-1:]], axis=0)
        o = oracle.solve(inst, eps=-1.0, max_iters=60, accel=1, warm=warm)
        for key in ("z", "v", "th", "be", "la"):
            assert relerr(its[j][key], o[key]) <= 1e-10, (j, key)


def test_resident_stage_invariant_n64():
    insts = [W.plain_lti(seed=61 + i, nx=48, nu=16, N=40) for i in range(2)]
    s = resident_solver(insts, pimpc.F64, eps=-1.0, max_iters=80, accel=1)
    res = s.solve()
    for j, inst in enumerate(insts):
        o = oracle.solve(inst, eps=-1.0, max_iters=80, accel=1)
        assert relerr(res["u"][j], o["u"]) <= 1e-10


def test_resident_rejects_what_does_not_fit():
    insts = ragged_batch(55, dims=[(4, 2, 3)])
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=10, accel=0)
    with pytest.raises(pimpc.PimpcError) as e:
        s.set_schedule(pimpc.FAMILY_RESIDENT, 0, 4)   # N = 3 < 4 CTAs
    assert e.value.code == pimpc.EINVAL
    big = [W.random_ltv(56, 24, 8, 3000)]
    s2 = pimpc.Solver(big, precision=pimpc.F64, eps=-1.0, max_iters=10, accel=0)
    with pytest.raises(pimpc.PimpcError):
        s2.set_schedule(pimpc.FAMILY_RESIDENT, 0, 1)  # far more than one CTA's shared memory


def test_resident_graph_and_adjoint():
    import torch
    from test_gpu_adjoint import NAMES, fd, loss_weights, small_batch
    insts = small_batch()
    Wu, Wx = loss_weights(insts, seed=5)
    s = resident_solver(insts, pimpc.F64, eps=-1.0, max_iters=40, accel=0)
    s.solve()
    g = s.backward(Wu, Wx, checkpoint_every=7)
    for j, inst in enumerate(insts):
        for name in NAMES:
            ref = fd(inst, Wu[j], Wx[j], 40, name)
            got = np.asarray(g[name][j]).reshape(ref.shape)
            assert np.max(np.abs(got - ref)) <= 1e-6 * max(1.0, float(np.max(np.abs(ref)))), name
    # cluster launches recorded into a CUDA graph
    pimpc.pimpc_set_graph(s.h, 1)
    dev = torch.device("cuda")
    x0 = torch.from_numpy(s.p["x0"]).to(dev)
    up = torch.from_numpy(s.p["u_prev"]).to(dev)
    ref = torch.from_numpy(s.p["ref"]).to(dev)
    u = torch.zeros(int(np.sum(s.N * s.nu)), dtype=torch.float64, device=dev)
    base = s.solve()
    for _ in range(2):
        pimpc.pimpc_solve(s.h, x0, up, ref, s.p["ref_per_stage"], 0, u, None)
    torch.cuda.synchronize()
    st = pimpc.pimpc_get_graph_stats(s.h)
    assert st["refused"] is None and st["captures"] == 1 and st["replays"] == 1, st
    assert np.array_equal(u.cpu().numpy(), np.concatenate([v.ravel() for v in base["u"]]))


# ---- stage-invariant instances as dense contractions ---------------------------------------

def lti_batch(seed, dims):
    return [W.plain_lti(seed=seed * 100 + i, nx=nx, nu=nu, N=N) for i, (nx, nu, N) in enumerate(dims)]


LTI_DIMS = [(4, 2, 20), (48, 16, 75), (3, 1, 1), (12, 4, 130), (7, 5, 34)]


@pytest.mark.parametrize("accel,items", [(0, 0), (1, 0), (1, 5)])
def test_contraction_fp64_matches_oracle(accel, items):
    insts = lti_batch(71, LTI_DIMS)
    s = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=120, accel=accel)
    s.set_schedule(4, 0, items)
    res = s.solve()
    its = s.iterates()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=120, accel=accel)
    for j, o in enumerate(ora):
        for key in ("z", "v", "th", "be", "la"):
            assert relerr(its[j][key], o[key]) <= 1e-10, (j, key)
        assert relerr(res["u"][j], o["u"]) <= 1e-10


def test_contraction_fp32_and_warm_start():
    insts = lti_batch(72, LTI_DIMS)
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=150, accel=0)
    s.set_schedule(4)
    res = s.solve()
    ora = oracle.solve_batch(insts, eps=-1.0, max_iters=150, accel=0)
    for j, o in enumerate(ora):
        assert relerr(res["u"][j], o["u"]) <= 1e-4, j
        assert relerr(res["x"][j], o["x"]) <= 1e-4, j
    d = pimpc.Solver(insts, precision=pimpc.F64, eps=-1.0, max_iters=40, accel=1)
    d.set_schedule(4, 0, 7)
    d.solve()
    first = d.iterates()
    d.solve(warm_start=2)
    its = d.iterates()
    for j, inst in enumerate(insts):
        warm = {k: np.concatenate([first[j][k][1:], first[j][k][-1:]], axis=0)
                for k in ("z", "v", "th", "be", "la")}
        o = oracle.solve(inst, eps=-1.0, max_iters=40, accel=1, warm=warm)
        assert relerr(its[j]["z"], o["z"]) <= 1e-10, j


def test_contraction_rejects_stage_varying_batches():
    s = pimpc.Solver(ragged_batch(73, dims=[(4, 2, 10)]), precision=pimpc.F32, eps=-1.0,
                     max_iters=5, accel=0)
    with pytest.raises(pimpc.PimpcError) as e:
        s.set_schedule(4)
    assert e.value.code == pimpc.EINVAL
