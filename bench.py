#!/usr/bin/env python
"""Benchmark of the piMPC hot path (arXiv 2601.14414) on GB300: batched uneven NMPC/MPC solves.

Workload (per GPU): 4096 independent random linear time-varying MPC instances, nx ~ U{4..24},
nu ~ U{2..8}, N ~ U{50..500} (1.13M stages), FP32 ADMM iterations of Algorithm 1 (accelerated,
with restart) on an FP64 per-stage factorisation, one persistent launch for the whole batch.

One step = factorise (FP64 cache of Algorithm 1) + solve (all iterations of every instance), cold
start, inputs resident in HBM, the solve replayed from a CUDA graph on the schedule the autotuner
picked for this batch. Iterations stop on c <= 1e-12 or, in FP32, once c has stalled at the
arithmetic's floor. A solve counts when its (u, x) is within 1e-4 (max error over max(1, max|w*|))
of the FP64 solution of the same instance from this GPU's FP64 path run to c <= 1e-20; a sample
of instances is also scored against the converged FP64 CPU oracle. The stage data (~3.5 GB) is
far larger than the 129 MB L2, so no flush is needed.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
Multi-GPU (torchrun): every rank solves its own seeded batch (weak scaling, no collective on the
data path); rank 0 prints one JSON line.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import subprocess
import sys
import tempfile
import time

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, HERE)

METRIC = "batched NMPC solves/s & ADMM iters/s at 1e-4 vs FP64 plain path; % roofline"
REF_STEP_SECONDS = 6.0  # oracle time per reference-arm step (bounded sample of the workload)


def parse_args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--batch", type=int, default=None, help="instances per GPU (default 4096)")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the further rows (polish, adjoint, latency, RTI, large state)")
    ap.add_argument("--profile", action="store_true",
                    help="profiling driver: only the FP32 factorise + solve steps, no reference, "
                         "e2e or CPU legs; prints the algorithmic bytes of the solve launch")
    ap.add_argument("--fixed-iters", type=int, default=None,
                    help="with --profile: run exactly this many iterations (eps < 0)")
    ap.add_argument("--profile-workload", choices=["batched", "large_lti"], default="batched",
                    help="with --profile: the batched uneven workload, or the large-state LTI one "
                         "(plain iterations)")
    ap.add_argument("--family", type=int, default=-1,
                    help="with --profile: the schedule family of the solve (-1: the default)")
    return ap.parse_args()


def rank_seed(seed, rank):
    """Every rank solves its own seeded batch (weak scaling: independent instances)."""
    return seed + 7919 * rank


def combine_ranks(torch, dist, dev, ms, ok, iters, stage_iters):
    """Whole-job figures from every rank's step time and counts: the slowest rank's time and
    the sums of accurate solves, instance-iterations and stage-iterations (no collective on the
    data path; one gather of four numbers after the timed region)."""
    if dist is None:
        return ms, float(ok), float(iters), float(stage_iters)
    t = torch.tensor([ms, float(ok), iters, stage_iters], dtype=torch.float64, device=dev)
    allt = [torch.zeros_like(t) for _ in range(dist.get_world_size())]
    dist.all_gather(allt, t)
    allt = torch.stack(allt).cpu().numpy()
    return (float(allt[:, 0].max()), float(allt[:, 1].sum()), float(allt[:, 2].sum()),
            float(allt[:, 3].sum()))


def dist_env():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


# ---------------------------------------------------------------------------------------------
# Clock sampling during the timed region.
# ---------------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_id):
        self.gpu_id = gpu_id
        self.proc = None
        self.path = None

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if self.gpu_id is not None:
            cmd += ["-i", str(self.gpu_id)]
        try:
            self.proc = subprocess.Popen(cmd, stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = []
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                rows.append(dict(sm=float(parts[1]), smax=float(parts[2]), hw=parts[5], hwt=parts[6],
                                 swt=parts[7], pcap=parts[8]))
            except ValueError:
                continue
        os.unlink(self.path)
        if not rows:
            return None
        reasons = []
        for key, name in (("hw", "hw_slowdown"), ("hwt", "hw_thermal_slowdown"),
                          ("swt", "sw_thermal_slowdown"), ("pcap", "sw_power_cap")):
            if any(r[key].lower().startswith("active") for r in rows):
                reasons.append(name)
        return dict(sm_mhz=float(np.median([r["sm"] for r in rows])),
                    sm_max_mhz=float(max(r["smax"] for r in rows)), reasons=reasons,
                    samples=len(rows))


def gpu_uuid(torch):
    try:
        u = str(torch.cuda.get_device_properties(torch.cuda.current_device()).uuid)
        return u if u.startswith("GPU-") else "GPU-" + u
    except Exception:
        return None


# ---------------------------------------------------------------------------------------------
# Algorithmic work per stage-iteration: the stage matrices (packed symmetric H and M) and the
# iterates read and written.
# ---------------------------------------------------------------------------------------------

def matrix_words(nx, nu):
    n = nx + nu
    return nx * n + nx + n * (n + 1) // 2 + nu * (nu + 1) // 2


def algorithmic_bytes(nx, nu, N, iters, momentum, word):
    """Minimum HBM traffic of the solve: per stage and iteration the stage matrices (G_k, e_k,
    packed H_k and M_k) plus the iterates: read z, v, theta, beta, lambda (5n), write them (5n),
    and read the previous iterate too (5n) on iterations that use the momentum step."""
    n = nx + nu
    per_stage = matrix_words(nx, nu) + 10 * n
    return float(np.sum(N * (iters * per_stage + momentum * 5 * n)) * word)


def load_peaks():
    path = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        d = json.load(open(path))
        return float(d["hbm_gbs"]), "measured"
    return 6800.0, "fallback"


# The solve kernel of each schedule family: (kernel name, source file, committed ncu summary).
SOLVE_KERNELS = {
    0: ("admm_kernel<float>", "admm.cu", "admm_kernel_f32_batched_512x30.md"),
    5: ("blk_kernel<float>", "admm_blk.cu", "blk_kernel_f32_batched_512x30.md"),
}
def kernel_files(source):
    """The kernel's source file and the library headers it includes, directly or through another
    header (a change in any of them changes the compiled kernel)."""
    csrc = os.path.join(HERE, "paper_2601_14414_gb300", "csrc")
    seen, todo = set(), [source]
    while todo:
        name = todo.pop()
        path = os.path.join(csrc, name)
        if name in seen or not os.path.exists(path):
            continue
        seen.add(name)
        todo += re.findall(r'^\s*#include\s+"([^"]+)"', open(path).read(), re.M)
    return [source] + sorted(seen - {source})


def kernel_source_hash(source):
    h = hashlib.sha256()
    for name in kernel_files(source):
        h.update(open(os.path.join(HERE, "paper_2601_14414_gb300", "csrc", name), "rb").read())
    return h.hexdigest()[:16]


def profiled_traffic(family):
    """DRAM bytes per algorithmic byte of the solve kernel from the committed ncu summary (a
    smaller case of the same workload; traffic grows in proportion to the stage-iterations), if
    it was taken on the current kernel source (the summary's source hash matches); else None."""
    if family not in SOLVE_KERNELS:
        return None
    _, source, profile_name = SOLVE_KERNELS[family]
    path = os.path.join(HERE, "profiles", profile_name)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m_hash = re.search(re.escape(source) + r" sha256\[:16\]:\s*([0-9a-f]{16})", text)
    m_traffic = re.search(r"traffic_per_algorithmic_byte:\s*([0-9.eE+-]+)", text)
    if not m_hash or not m_traffic or m_hash.group(1) != kernel_source_hash(source):
        return None
    return float(m_traffic.group(1))


# ---------------------------------------------------------------------------------------------
# The reference arm: the FP64 CPU oracle on the host cores.
# ---------------------------------------------------------------------------------------------

def oracle_sample(insts, cfg, seconds_hint, rng_seed=0, keep=False):
    """The FP64 oracle (Algorithm 1, same eps and iteration cap) on random instances of the
    workload, all host cores, grown until about `seconds_hint` seconds. Returns (count, seconds,
    threads, indices[, results])."""
    import oracle
    threads = os.cpu_count() or 1
    rng = np.random.default_rng(rng_seed)
    order = rng.permutation(len(insts))
    take = max(threads, 8)
    done = 0
    results = []
    t0 = time.perf_counter()
    while True:
        chunk = [insts[i] for i in order[done:done + take]]
        if not chunk:
            break
        r = oracle.solve_batch(chunk, threads=threads, eps=cfg["eps"], max_iters=cfg["max_iters"],
                               accel=cfg["accel"], eta=cfg["eta"])
        if keep:
            results += r
        done += len(chunk)
        if time.perf_counter() - t0 >= seconds_hint:
            break
    dt = time.perf_counter() - t0
    if keep:
        return done, dt, threads, order[:done], results
    return done, dt, threads, order[:done]


def oracle_converged(insts, idx):
    """Converged FP64 oracle solutions (c <= 1e-22) of insts[idx], all host cores (untimed)."""
    import oracle
    r = oracle.solve_batch([insts[i] for i in idx], threads=os.cpu_count() or 1, eps=1e-22,
                           max_iters=60000, accel=1, eta=0.999)
    return [np.concatenate([a["u"].ravel(), a["x"].ravel()]) for a in r]


def rel_err(w, ws):
    return float(np.max(np.abs(w - ws)) / max(1.0, np.max(np.abs(ws))))


# ---------------------------------------------------------------------------------------------
# Further rows measured on the same GPU (rank 0): each returns a dict, or an error entry.
# ---------------------------------------------------------------------------------------------

def extra(fn, *a, **kw):
    try:
        return fn(*a, **kw)
    except Exception as ex:  # one failing extra must not lose the benchmark line
        return dict(error=f"{type(ex).__name__}: {ex}")


def accuracy_count(u, x, u_ref, x_ref, ou, ox, tol):
    err = np.array([np.max(np.abs(np.concatenate([u[ou[j]:ou[j + 1]], x[ox[j]:ox[j + 1]]]) -
                                  np.concatenate([u_ref[ou[j]:ou[j + 1]], x_ref[ox[j]:ox[j + 1]]])))
                    / max(1.0, np.max(np.abs(np.concatenate([u_ref[ou[j]:ou[j + 1]],
                                                             x_ref[ox[j]:ox[j + 1]]]))))
                    for j in range(len(ou) - 1)])
    return int(np.sum(err <= tol)), err


def bench_polish(torch, pimpc, make, d, p, cfg, tot_u, tot_x, refs, ou, ox):
    """The headline workload with the FP64 polish: FP32 iterations to eps, then FP64 iterations
    (FP64 cache) to polish_eps; every step refreshes the dynamics, so both caches are rebuilt."""
    stream = torch.cuda.current_stream()
    h = make(pimpc.F32, cfg["eps"], cfg["max_iters"])
    pimpc.pimpc_set_polish(h, cfg["polish_iters"], cfg["polish_eps"])
    dev = d["x0"].device
    u = torch.zeros(tot_u, dtype=torch.float64, device=dev)
    x = torch.zeros(tot_x, dtype=torch.float64, device=dev)

    def step():
        pimpc.pimpc_set_dynamics(h, d["A"], d["B"], d["e"])
        pimpc.pimpc_factorise(h, stream.cuda_stream)
        pimpc.pimpc_solve(h, d["x0"], None, d["ref"], p["ref_per_stage"], 0, u, x)

    step()
    torch.cuda.synchronize()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    step()
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    ok, err = accuracy_count(u.cpu().numpy(), x.cpu().numpy(), refs[0], refs[1], ou, ox,
                             cfg["accuracy"])
    iters = np.zeros(len(ou) - 1, np.int32)
    pimpc.pimpc_get_stats(h, iters, None, None, None)
    pimpc.pimpc_destroy(h)
    return dict(value=ok / (ms / 1e3), unit="solves/s", ms_per_step=ms, ok=ok, of=len(ou) - 1,
                median_err=float(np.median(err)), polish_iters=cfg["polish_iters"],
                polish_eps=cfg["polish_eps"], mean_iters_fp32_plus_fp64=float(np.mean(iters)),
                steps=1, warmup=1)


def fp32_peak_tflops():
    """FP32 CUDA-core peak of the part from its unit counts and clock: 152 SMs x 128 FP32 lanes x
    2 flops per fused multiply-add x the SM clock (the measured maximum in MEASURED_PEAKS.json,
    else 2070 MHz)."""
    mhz = 2070.0
    path = os.path.join(HERE, "MEASURED_PEAKS.json")
    if os.path.exists(path):
        mhz = float(json.load(open(path)).get("sm_max_mhz", mhz))
    return 152 * 128 * 2 * mhz * 1e6 / 1e12


def bench_cartpole(torch, pimpc, W, steps, family=None):
    """Differentiable MPC: 1024 cart-pole instances (N = 100), 150 plain FP32 iterations,
    forward solve + reverse sweep with checkpoints every 25 iterations, device memory.
    ``family``: the forward solve's schedule (None: the default). The roofline is the FP32 ALU
    one: forward flops per stage-iteration 2 n^2 + 4 nx n + 4 nx nu + 2 nu^2 + 40 n (the
    products and the elementwise steps, n = nx + nu)."""
    insts = W.cartpole_batch()
    iters, K = 150, 25
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=iters, accel=0)
    if family is not None:
        s.set_schedule(family)
    prm = np.ascontiguousarray(np.concatenate([i["params"] for i in insts]))
    xb = np.ascontiguousarray(np.concatenate([i["op_x"] for i in insts]))
    ub = np.ascontiguousarray(np.concatenate([i["op_u"] for i in insts]))
    pimpc.pimpc_linearise(s.h, W.MODEL_CARTPOLE, prm, insts[0]["dt"], xb, ub)
    dev = torch.device("cuda", torch.cuda.current_device())
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev)
    x0, ref = t(s.p["x0"]), t(s.p["ref"])
    tu, tx = int(np.sum(s.N * s.nu)), int(np.sum(s.N * s.nx))
    u = torch.zeros(tu, dtype=torch.float64, device=dev)
    x = torch.zeros(tx, dtype=torch.float64, device=dev)
    rng = np.random.default_rng(4)
    gu, gx = t(rng.standard_normal(tu)), t(rng.standard_normal(tx))
    outs = [torch.zeros(n, dtype=torch.float64, device=dev)
            for n in (int(np.sum(s.nx)), int(np.sum(s.nx + s.nu)), int(np.sum(s.nx)),
                      int(np.sum(s.nu)), int(np.sum(s.nx)), int(np.sum(s.nx)),
                      int(np.sum(s.nu)), int(np.sum(s.nu)))]
    stream = torch.cuda.current_stream()

    def fwd():
        pimpc.pimpc_solve(s.h, x0, None, ref, False, 0, u, x)

    def bwd():
        pimpc.pimpc_backward(s.h, gu, gx, *outs, checkpoint_every=K)

    for _ in range(2):
        fwd()
        bwd()
    torch.cuda.synchronize()
    ev = [torch.cuda.Event(enable_timing=True) for _ in range(3 * steps)]
    for k in range(steps):
        ev[3 * k].record(stream)
        fwd()
        ev[3 * k + 1].record(stream)
        bwd()
        ev[3 * k + 2].record(stream)
    torch.cuda.synchronize()
    f_ms = float(np.mean([ev[3 * k].elapsed_time(ev[3 * k + 1]) for k in range(steps)]))
    b_ms = float(np.mean([ev[3 * k + 1].elapsed_time(ev[3 * k + 2]) for k in range(steps)]))
    fam = s.schedule()["family"]
    s.close()
    nx, nu, n = 4, 1, 5
    flops = float(len(insts) * 100 * iters * (2 * n * n + 4 * nx * n + 4 * nx * nu + 2 * nu * nu + 40 * n))
    peak = fp32_peak_tflops()
    fwd_tf = flops / (f_ms / 1e3) / 1e12
    return dict(value=len(insts) / ((f_ms + b_ms) / 1e3), unit="forward+backward solves/s",
                forward_ms=f_ms, backward_ms=b_ms, instances=len(insts), N=100, iterations=iters,
                checkpoint_every=K, dtype="f32", steps=steps, warmup=2, forward_family=fam,
                roofline=dict(bound="alu", achieved=fwd_tf, peak=peak, unit="TFLOP/s",
                              frac=fwd_tf / peak, forward_flops=flops,
                              peak_kind="derived: 152 SMs x 128 FP32 lanes x 2 x SM clock",
                              note="forward solve; the backward sweep is about three forward "
                                   "passes per iteration (recompute and reverse)"),
                forward_plus_backward_frac=(4 * flops / ((f_ms + b_ms) / 1e3) / 1e12) / peak)


def bench_temporal_blocking(torch, pimpc, W, cfg, iters=64):
    """Plain iterations (accel = 0, fixed count) on the batched workload: the blocked lane groups
    (family 5, one pass over the stage data per iteration) against temporal blocking (family 7,
    one pass per T iterations), and the one-pass roofline bound (algorithmic bytes of one plain
    iteration over the measured HBM peak)."""
    insts = W.batched_uneven(seed=cfg["seed"], batch=cfg["batch"])
    p = pimpc.pack(insts)
    nx, nu, N = p["nx"].astype(np.int64), p["nu"].astype(np.int64), p["N"].astype(np.int64)
    peak, _ = load_peaks()
    one = algorithmic_bytes(nx, nu, N, np.ones(len(insts), np.int64), np.zeros(len(insts), np.int64), 4)
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    x0, ref = torch.from_numpy(p["x0"]).to(dev), torch.from_numpy(p["ref"]).to(dev)
    res = dict(iterations=iters, one_pass_bound_ms_per_iteration=one / peak / 1e6,
               one_pass_bytes_per_iteration=one)
    for name, fam, T in (("blocked_lanes", 5, 0), ("temporal_T4", 7, 4), ("temporal_T8", 7, 8)):
        s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=iters, accel=0)
        s.set_schedule(fam, 0, T)
        u = torch.zeros(int(np.sum(N * nu)), dtype=torch.float64, device=dev)
        x = torch.zeros(int(np.sum(N * nx)), dtype=torch.float64, device=dev)
        pimpc.pimpc_solve(s.h, x0, None, ref, False, 0, u, x)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        pimpc.pimpc_solve(s.h, x0, None, ref, False, 0, u, x)
        b.record(stream)
        torch.cuda.synchronize()
        res[name + "_ms_per_iteration"] = a.elapsed_time(b) / iters
        s.close()
    return res


def bench_latency(torch, pimpc, W, reps=50):
    """One plain LTI instance (nx 4, nu 2, N 20), FP64, 200 iterations: time per solve with
    direct launches and with the solve replayed from a CUDA graph (device memory)."""
    inst = W.plain_lti()
    dev = torch.device("cuda", torch.cuda.current_device())
    out = {}
    for mode in ("direct", "graph", "resident", "resident_graph"):
        s = pimpc.Solver([inst], precision=pimpc.F64, eps=-1.0, max_iters=200, accel=0)
        if mode.startswith("resident"):
            s.set_schedule(pimpc.FAMILY_RESIDENT)
        if mode.endswith("graph"):
            pimpc.pimpc_set_graph(s.h, 1)
        t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev)
        x0, ref = t(s.p["x0"]), t(s.p["ref"])
        u = torch.zeros(40, dtype=torch.float64, device=dev)
        x = torch.zeros(80, dtype=torch.float64, device=dev)
        for _ in range(10):
            pimpc.pimpc_solve(s.h, x0, None, ref, False, 0, u, x)
        torch.cuda.synchronize()
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record()
        for _ in range(reps):
            pimpc.pimpc_solve(s.h, x0, None, ref, False, 0, u, x)
        b.record()
        torch.cuda.synchronize()
        out[mode + "_us_per_solve"] = 1e3 * a.elapsed_time(b) / reps
        if mode.endswith("graph"):
            out[mode + "_stats"] = pimpc.pimpc_get_graph_stats(s.h)
        s.close()
    out["us_per_iteration_resident_graph"] = out["resident_graph_us_per_solve"] / 200
    out.update(workload="plain LTI nx 4, nu 2, N 20, FP64, 200 iterations", reps=reps)
    return out


def bench_rti(torch, pimpc, W, precision, steps=50, family=None):
    """Quadrotor NMPC by real-time iteration (N = 200, 100 iterations per sample, warm start):
    per sample linearise along the shifted previous solution, factorise, solve, plant step; all
    on device memory. ``family``: the solve's schedule (None: the default)."""
    wl = W.quadrotor_rti()
    nx, nu, N = wl["nx"], wl["nu"], wl["N"]
    inst = {k: wl[k] for k in ("nx", "nu", "N", "q", "r", "rdu", "xmin", "xmax", "umin", "umax",
                               "u_prev", "rho")}
    inst.update(lti=False, x0=wl["x0"], ref=W.quadrotor_reference(wl, 0))
    s = pimpc.Solver([inst], precision=precision, eps=-1.0, max_iters=wl["iters"], accel=1)
    if family is not None:
        s.set_schedule(family)
    dev = torch.device("cuda", torch.cuda.current_device())
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev)
    prm = t(wl["params"])
    refs = [t(W.quadrotor_reference(wl, k)) for k in range(steps)]
    x = t(wl["x0"])
    u = torch.zeros(N * nu, dtype=torch.float64, device=dev)
    xs = torch.zeros(N * nx, dtype=torch.float64, device=dev)
    xn = torch.zeros(nx, dtype=torch.float64, device=dev)
    xbar = x.repeat(N)
    ubar = t(wl["hover_u"]).repeat(N)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(steps):
        pimpc.pimpc_linearise(s.h, wl["model"], prm, wl["dt"], xbar, ubar)
        pimpc.pimpc_solve(s.h, x, None, refs[k], False, 1 if k else 0, u, xs)
        pimpc.pimpc_plant_step(s.h, wl["model"], prm, wl["dt"], x, u[:nu].contiguous(), xn)
        x.copy_(xn)
        xbar = torch.cat([x, xs[nx:]])
        ubar = torch.cat([u[nu:], u[-nu:]])
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    sched = s.schedule()
    s.close()
    return dict(value=steps / (ms / 1e3), unit="RTI samples/s", ms_per_sample=ms / steps,
                us_per_iteration=1e3 * ms / steps / wl["iters"], samples=steps, N=N,
                iterations_per_sample=wl["iters"],
                dtype="f64" if precision == pimpc.F64 else "f32",
                schedule=dict(family=sched["family"], item_scale=sched["item_scale"]),
                final_position=x[:3].cpu().numpy().tolist())


def bench_cstr(torch, pimpc, W, precision, steps=400, family=None):
    """The paper's CSTR NMPC at its size: N = 5000, 1000 iterations per sample (warm start),
    W_du = 0.1 with u_prev = the applied coolant temperature, inlet temperature varying with
    time; per sample linearise along the shifted previous solution, factorise, solve, plant
    step, all on device memory. The paper's figure for this loop is context only (another GPU)."""
    wl = W.cstr_nmpc()
    nx, nu, N = wl["nx"], wl["nu"], wl["N"]
    iters = 1000
    inst = {k: wl[k] for k in ("nx", "nu", "N", "q", "r", "rdu", "xmin", "xmax", "umin", "umax",
                               "u_prev", "rho")}
    inst.update(lti=False, x0=wl["x0"], ref=wl["ref"])
    s = pimpc.Solver([inst], precision=precision, eps=-1.0, max_iters=iters, accel=1)
    if family is not None:
        s.set_schedule(family)
    dev = torch.device("cuda", torch.cuda.current_device())
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a, np.float64)).to(dev)
    prms = [t(np.append(wl["params"], W.cstr_inlet_temperature(k * wl["dt"])))
            for k in range(steps)]
    ref = t(wl["ref"])
    x = t(wl["x0"])
    up = t(wl["u_prev"])
    u = torch.zeros(N * nu, dtype=torch.float64, device=dev)
    xs = torch.zeros(N * nx, dtype=torch.float64, device=dev)
    xn = torch.zeros(nx, dtype=torch.float64, device=dev)
    xbar = x.repeat(N)
    ubar = up.repeat(N)
    stream = torch.cuda.current_stream()
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    for k in range(steps):
        pimpc.pimpc_linearise(s.h, wl["model"], prms[k], wl["dt"], xbar, ubar)
        pimpc.pimpc_solve(s.h, x, up, ref, False, 1 if k else 0, u, xs)
        up = u[:nu].contiguous()
        pimpc.pimpc_plant_step(s.h, wl["model"], prms[k], wl["dt"], x, up, xn)
        x.copy_(xn)
        xbar = torch.cat([x, xs[nx:]])
        ubar = torch.cat([u[nu:], u[-nu:]])
    b.record(stream)
    torch.cuda.synchronize()
    ms = a.elapsed_time(b)
    sched = s.schedule()
    s.close()
    return dict(value=ms / 1e3 / steps, unit="s per MPC step", ms_per_step=ms / steps,
                us_per_iteration=1e3 * ms / steps / iters, steps=steps, N=N,
                iterations_per_step=iters, dtype="f64" if precision == pimpc.F64 else "f32",
                schedule=dict(family=sched["family"], item_scale=sched["item_scale"]),
                final_state=x.cpu().numpy().tolist(),
                paper_context="0.526 s per step median (RTX 3080, Julia; Table II)")


def bench_afti16(pimpc, W, precision, family=None):
    """The paper's AFTI-16 example: 200 closed-loop MPC steps (N = 5), each solved to
    c <= 1e-6 from the previous iterates; mean iterations per step (the paper's is 2030 with
    its own unstated rho and reference) and wall time per step of the host-memory solves."""
    from paper_2601_14414_gb300.closed_loop import afti16_gpu_loop
    wl = W.afti16()
    afti16_gpu_loop(wl, 5, precision, family=family)  # warm-up of the library and the GPU
    us, xs, its, secs = afti16_gpu_loop(wl, wl["steps"], precision, family=family)
    return dict(mean_iterations=float(np.mean(its)), max_iterations=int(np.max(its)),
                ms_per_step=1e3 * secs / wl["steps"],
                us_per_iteration=1e6 * secs / max(1, int(np.sum(its))), steps=wl["steps"],
                rho=wl["rho"], dtype="f64" if precision == pimpc.F64 else "f32",
                max_abs_y1=float(np.abs(xs[1:, 1]).max()), paper_mean_iterations=2030)


def bench_large_lti(torch, pimpc, W, iters=200):
    """256 LTI instances, nx 48, nu 16, N 1000 (bounds active on about a fifth of the inputs).
    (1) A fixed number of iterations (plain and accelerated) of the tensor-core schedule
    (family 6, FP32), of the blocked lane groups (family 5, FP32) and of the plain lane groups
    in FP64 (family 0): time per iteration, iterate traffic against the measured HBM peak.
    (2) Solved to c <= 1e-5 (accelerated, at most 20000 iterations) in FP32 on the tensor cores:
    seconds per solve and iterations; the FP64 time to the same tolerance is its iterations
    times its measured time per accelerated iteration (running it takes minutes). Device-memory
    solves timed with CUDA events."""
    insts = W.large_lti()
    peak, _ = load_peaks()
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()
    p = pimpc.pack(insts)
    x0 = torch.from_numpy(p["x0"]).to(dev)
    ref = torch.from_numpy(p["ref"]).to(dev)
    tu = int(np.sum(p["N"] * p["nu"]))
    tx = int(np.sum(p["N"] * p["nx"]))
    n = 64

    def timed(s, reps=2):
        u = torch.zeros(tu, dtype=torch.float64, device=dev)
        x = torch.zeros(tx, dtype=torch.float64, device=dev)
        pimpc.pimpc_solve(s.h, x0, None, ref, False, 0, u, x)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(reps):
            pimpc.pimpc_solve(s.h, x0, None, ref, False, 0, u, x)
        b.record(stream)
        torch.cuda.synchronize()
        its = np.zeros(len(insts), np.int32)
        mom = np.zeros(len(insts), np.int32)
        pimpc.pimpc_get_stats(s.h, its, None, None, mom)
        return a.elapsed_time(b) / reps, its, mom, u.cpu().numpy(), x.cpu().numpy()

    res = dict(instances=len(insts), N=1000, nx=48, nu=16, fixed_iterations=iters)
    for name, prec, fam, word in (("f32_tensor_cores", pimpc.F32, 6, 4),
                                  ("f32_blocked_lanes", pimpc.F32, 5, 4),
                                  ("f64_lanes", pimpc.F64, 0, 8)):
        row = {}
        its_fixed = iters if prec == pimpc.F32 else iters // 4
        for accel in (0, 1):
            s = pimpc.Solver(insts, precision=prec, eps=-1.0, max_iters=its_fixed, accel=accel)
            s.set_schedule(fam)
            ms, its, mom, _, _ = timed(s, reps=2 if prec == pimpc.F32 else 1)
            alg = float(np.sum(1000 * (its.astype(np.int64) * 10 * n + mom * 5 * n))) * word
            row["plain" if accel == 0 else "accel"] = dict(
                ms_per_iteration=ms / its_fixed, iterate_gb_per_s=alg / (ms / 1e3) / 1e9,
                frac_of_measured_hbm=alg / (ms / 1e3) / 1e9 / peak)
            s.close()
        res[name] = row
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=1e-5, max_iters=20000, accel=1)
    s.set_schedule(6)
    ms, its, _, _, _ = timed(s, reps=1)
    st = np.zeros(len(insts), np.int32)
    pimpc.pimpc_get_stats(s.h, None, None, st, None)
    s.close()
    res["f32_tensor_cores_to_1e-5"] = dict(
        seconds_per_solve=ms / 1e3, mean_iterations=float(np.mean(its)),
        converged=int(np.sum(st == pimpc.CONVERGED)), max_iterations=20000)
    res["f64_lanes_to_1e-5_estimate_s"] = float(
        np.sum(its) / len(insts) * res["f64_lanes"]["accel"]["ms_per_iteration"] / 1e3)
    res["note"] = ("iterate traffic: per stage-iteration 10 n words (read, write) plus 5 n on "
                   "momentum iterations; the stage matrices are shared by all stages")
    return res


def profile_large_lti(args, torch, pimpc, W):
    """Profiling driver on the large-state LTI workload (nx 48, nu 16, N 1000; --batch
    instances, default 256): FP32, plain iterations, --fixed-iters of them, the schedule of
    --family; warm-up + steps solves from device memory. Prints the algorithmic bytes of one
    solve (iterates only: the stage matrices are shared by every stage)."""
    insts = W.large_lti(batch=args.batch or 256)
    iters = args.fixed_iters or 10
    s = pimpc.Solver(insts, precision=pimpc.F32, eps=-1.0, max_iters=iters, accel=0)
    if args.family >= 0:
        s.set_schedule(args.family)
    dev = torch.device("cuda", torch.cuda.current_device())
    x0 = torch.from_numpy(s.p["x0"]).to(dev)
    ref = torch.from_numpy(s.p["ref"]).to(dev)
    u = torch.zeros(int(np.sum(s.N * s.nu)), dtype=torch.float64, device=dev)
    x = torch.zeros(int(np.sum(s.N * s.nx)), dtype=torch.float64, device=dev)
    for _ in range(args.warmup + args.steps):
        pimpc.pimpc_solve(s.h, x0, None, ref, False, 0, u, x)
    torch.cuda.synchronize()
    n = 64
    alg = float(len(insts) * 1000 * iters * 10 * n * 4)
    print(json.dumps(dict(profile=True, workload="large_lti", instances=len(insts),
                          family=s.schedule()["family"], iterations=iters,
                          algorithmic_bytes_per_solve=alg)), flush=True)
    s.close()
    return 0


def run_reference(args):
    """The reference arm: the FP64 CPU oracle (Algorithm 1, same eps, iteration cap and restart
    rule as our arm) on the host cores. Each step solves a random sample of the workload for
    about REF_STEP_SECONDS; warm-up steps solve one chunk each. The solves of the first step's
    first instances are scored against converged oracle solutions (untimed), and the rate
    counts only the fraction of solves that meet the accuracy threshold there."""
    world, rank, _ = dist_env()
    if rank != 0:
        return 0
    from paper_2601_14414_gb300 import configs, workloads as W
    cfg = configs.BATCHED_UNEVEN
    batch = args.batch or cfg["batch"]
    insts = W.batched_uneven(seed=cfg["seed"], batch=batch)
    for k in range(args.warmup):
        oracle_sample(insts, cfg, 0.0, rng_seed=1000 + k)  # one chunk of real solves
    times, counts, threads, scored = [], [], 1, None
    for k in range(args.steps):
        n, dt, threads, idx, res = oracle_sample(insts, cfg, REF_STEP_SECONDS, rng_seed=k,
                                                 keep=(k == 0))
        times.append(dt)
        counts.append(n)
        if k == 0:
            m = min(len(idx), cfg["oracle_score_sample"])
            wo = oracle_converged(insts, idx[:m])
            errs = [rel_err(np.concatenate([r["u"].ravel(), r["x"].ravel()]), w)
                    for r, w in zip(res[:m], wo)]
            scored = dict(ok=int(np.sum(np.array(errs) <= cfg["accuracy"])), of=m,
                          max_err=float(np.max(errs)), threshold=cfg["accuracy"])
    frac_ok = scored["ok"] / scored["of"] if scored else 1.0
    value = float(np.sum(counts) / np.sum(times)) * frac_ok
    sample = (f"{int(np.mean(counts))} random instances of the {batch}-instance workload per "
              f"step, about {REF_STEP_SECONDS:.0f} s each")
    line = dict(impl="reference", metric=METRIC, value=value, unit="solves/s", n_gpus=args.gpus,
                steps=args.steps, warmup=args.warmup,
                ms_per_step=1e3 * float(np.mean(times)), higher_is_better=True, scaling="weak",
                vs_baseline=None, dtype="f64", data="synthetic",
                config=dict(workload=cfg["name"], instances=batch, eps=cfg["eps"],
                            accel=cfg["accel"], max_iters=cfg["max_iters"]),
                accuracy=scored,
                cpu_baseline=dict(value=value, unit="solves/s", cores=threads, kind="oracle",
                                  sample=sample),
                e2e=dict(value=value, unit="solves/s", h2d_bytes_per_step=0, d2h_bytes_per_step=0))
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------------------------------------
# Our arm.
# ---------------------------------------------------------------------------------------------

def run_ours(args):
    import torch
    world, rank, local = dist_env()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        dist = None
    from paper_2601_14414_gb300 import configs, pimpc, workloads as W
    cfg = configs.BATCHED_UNEVEN
    batch = args.batch or cfg["batch"]
    dev = torch.device("cuda", torch.cuda.current_device())
    stream = torch.cuda.current_stream()

    insts = W.batched_uneven(seed=rank_seed(cfg["seed"], rank), batch=batch)
    p = pimpc.pack(insts)
    nx, nu, N = p["nx"].astype(np.int64), p["nu"].astype(np.int64), p["N"].astype(np.int64)
    d = {k: torch.from_numpy(p[k]).to(dev) for k in ("A", "B", "e", "x0", "ref")}
    tot_u, tot_x = int(np.sum(N * nu)), int(np.sum(N * nx))

    def make(prec, eps, iters, stall=True):
        h = pimpc.pimpc_create(p["nx"], p["nu"], p["N"], 0, prec, device=dev.index)
        pimpc.pimpc_set_weights(h, p["q"], p["r"], p["rdu"])
        pimpc.pimpc_set_bounds(h, p["xmin"], p["xmax"], p["umin"], p["umax"])
        pimpc.pimpc_set_options(h, cfg["rho"], eps, iters, cfg["accel"], cfg["eta"])
        pimpc.pimpc_set_dynamics(h, d["A"], d["B"], d["e"])
        if stall and prec == pimpc.F32:
            pimpc.pimpc_set_stall(h, cfg["stall_window"], cfg["stall_factor"], cfg["stall_below"],
                                  cfg["stall_rel"])
        return h

    if args.profile and args.profile_workload == "large_lti":
        return profile_large_lti(args, torch, pimpc, W)
    if args.profile:
        eps = -1.0 if args.fixed_iters else cfg["eps"]
        iters_cap = args.fixed_iters or cfg["max_iters"]
        h = make(pimpc.F32, eps, iters_cap)
        if args.family >= 0:
            pimpc.pimpc_set_schedule(h, args.family, 0, 0)
        u = torch.zeros(tot_u, dtype=torch.float64, device=dev)
        x = torch.zeros(tot_x, dtype=torch.float64, device=dev)
        for _ in range(args.warmup + args.steps):
            pimpc.pimpc_factorise(h, stream.cuda_stream)
            pimpc.pimpc_solve(h, d["x0"], None, d["ref"], p["ref_per_stage"], 0, u, x)
        torch.cuda.synchronize()
        iters = np.zeros(batch, np.int32)
        mom = np.zeros(batch, np.int32)
        pimpc.pimpc_get_stats(h, iters, None, None, mom)
        alg = algorithmic_bytes(nx, nu, N, iters.astype(np.int64), mom.astype(np.int64), 4)
        if rank == 0:
            print(json.dumps(dict(profile=True, instances=batch, stages=int(np.sum(N)),
                                  stage_iterations=int(np.sum(iters * N)),
                                  algorithmic_bytes_per_solve=alg)), flush=True)
        pimpc.pimpc_destroy(h)
        return 0

    # FP64 reference solution on this GPU (untimed), scored against in every step.
    href = make(pimpc.F64, cfg["ref_eps"], cfg["ref_max_iters"])
    u_ref = torch.zeros(tot_u, dtype=torch.float64, device=dev)
    x_ref = torch.zeros(tot_x, dtype=torch.float64, device=dev)
    pimpc.pimpc_solve(href, d["x0"], None, d["ref"], p["ref_per_stage"], 0, u_ref, x_ref)
    torch.cuda.synchronize()
    pimpc.pimpc_destroy(href)

    h = make(pimpc.F32, cfg["eps"], cfg["max_iters"])
    # Schedule from the autotuner on this batch (untimed), then the solve as a CUDA graph.
    tuned = pimpc.pimpc_autotune(h, 20)
    pimpc.pimpc_set_graph(h, 1)
    u = torch.zeros(tot_u, dtype=torch.float64, device=dev)
    x = torch.zeros(tot_x, dtype=torch.float64, device=dev)

    def step(ev_a=None, ev_b=None, ev_c=None):
        if ev_a is not None:
            ev_a.record(stream)
        pimpc.pimpc_factorise(h, stream.cuda_stream)
        if ev_b is not None:
            ev_b.record(stream)
        pimpc.pimpc_solve(h, d["x0"], None, d["ref"], p["ref_per_stage"], 0, u, x)
        if ev_c is not None:
            ev_c.record(stream)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()

    clocks = ClockSampler(gpu_uuid(torch))
    evs = [[torch.cuda.Event(enable_timing=True) for _ in range(3)] for _ in range(args.steps)]
    t_start = torch.cuda.Event(enable_timing=True)
    t_end = torch.cuda.Event(enable_timing=True)
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    t_start.record(stream)
    for k in range(args.steps):
        step(*evs[k])
    t_end.record(stream)
    torch.cuda.synchronize()
    clk = clocks.stop()
    if dist is not None:
        dist.barrier()
    total_ms = t_start.elapsed_time(t_end)
    fact_ms = [a.elapsed_time(b) for a, b, _ in evs]
    solve_ms = [b.elapsed_time(c) for _, b, c in evs]

    # Per-instance results of the last step.
    iters = np.zeros(batch, np.int32)
    cvals = np.zeros(batch)
    status = np.zeros(batch, np.int32)
    mom = np.zeros(batch, np.int32)
    pimpc.pimpc_get_stats(h, iters, cvals, status, mom)
    uu, xx, ur, xr = (t.cpu().numpy() for t in (u, x, u_ref, x_ref))
    ou = np.concatenate([[0], np.cumsum(N * nu)])
    ox = np.concatenate([[0], np.cumsum(N * nx)])
    err = np.zeros(batch)
    for j in range(batch):
        w = np.concatenate([uu[ou[j]:ou[j + 1]], xx[ox[j]:ox[j + 1]]])
        ws = np.concatenate([ur[ou[j]:ou[j + 1]], xr[ox[j]:ox[j + 1]]])
        err[j] = np.max(np.abs(w - ws)) / max(1.0, np.max(np.abs(ws)))
    ok = int(np.sum(err <= cfg["accuracy"]))
    graph_stats = pimpc.pimpc_get_graph_stats(h)

    ms_step = total_ms / args.steps
    ms_max, ok_all, it_all, stit_all = combine_ranks(
        torch, dist, dev, ms_step, ok, float(np.sum(iters)), float(np.sum(iters * N)))
    value = ok_all / (ms_max / 1e3)

    # Roofline of the dominant kernel (the ADMM solve), bytes per launch / launch time.
    alg = algorithmic_bytes(nx, nu, N, iters.astype(np.int64), mom.astype(np.int64), 4)
    solve_s = float(np.mean(solve_ms)) / 1e3
    peak, peak_kind = load_peaks()
    achieved = alg / solve_s / 1e9
    family = pimpc.pimpc_get_schedule(h)["family"]
    ratio = profiled_traffic(family)
    traffic = None if ratio is None else ratio * alg
    kernel_name = SOLVE_KERNELS.get(family, ("family %d" % family,))[0]

    line = None
    if rank == 0:
        # e2e: the same step through the C ABI with host buffers (pinned), copies inside.
        e2e = None
        if not args.no_e2e:
            pinned = {k: torch.from_numpy(p[k]).pin_memory() for k in ("A", "B", "e", "x0", "ref")}
            hp = {k: v.numpy() for k, v in pinned.items()}
            hu = torch.zeros(tot_u, dtype=torch.float64).pin_memory().numpy()
            hx = torch.zeros(tot_x, dtype=torch.float64).pin_memory().numpy()
            hit = np.zeros(batch, np.int32)
            hst = np.zeros(batch, np.int32)
            he = make(pimpc.F32, cfg["eps"], cfg["max_iters"])

            def host_step():
                pimpc.pimpc_set_dynamics(he, hp["A"], hp["B"], hp["e"])
                pimpc.pimpc_solve(he, hp["x0"], None, hp["ref"], p["ref_per_stage"], 0, hu, hx,
                                  hit, None, hst)

            for _ in range(max(1, min(args.warmup, 2))):
                host_step()
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            for _ in range(args.steps):
                host_step()
            torch.cuda.synchronize()
            e2e_s = (time.perf_counter() - t0) / args.steps
            w_all = np.concatenate([hu, hx])
            same = np.array_equal(hu, uu) and np.array_equal(hx, xx)
            h2d = sum(hp[k].nbytes for k in ("A", "B", "e", "x0", "ref"))
            d2h = hu.nbytes + hx.nbytes + hit.nbytes + hst.nbytes
            e2e = dict(value=ok / e2e_s, unit="solves/s", h2d_bytes_per_step=int(h2d),
                       d2h_bytes_per_step=int(d2h), ms_per_step=1e3 * e2e_s,
                       same_result_as_device_path=bool(same))
            pimpc.pimpc_destroy(he)
            del w_all

        # The plain single-instance FP64 GPU path on a sample of the same instances.
        rng = np.random.default_rng(0)
        sample = rng.choice(batch, size=16, replace=False)
        t_single = 0.0
        ok_single = 0
        for j in sample:
            inst = insts[j]
            s1 = pimpc.Solver([inst], precision=pimpc.F64, eps=cfg["eps"],
                              max_iters=cfg["max_iters"], accel=cfg["accel"], eta=cfg["eta"])
            s1.solve()  # warm-up of this object
            torch.cuda.synchronize()
            t0 = time.perf_counter()
            r1 = s1.solve()
            t_single += time.perf_counter() - t0
            w = np.concatenate([r1["u"][0].ravel(), r1["x"][0].ravel()])
            ws = np.concatenate([ur[ou[j]:ou[j + 1]], xr[ox[j]:ox[j + 1]]])
            ok_single += int(np.max(np.abs(w - ws)) / max(1.0, np.max(np.abs(ws))) <= cfg["accuracy"])
            s1.close()
        single = dict(value=ok_single / t_single, unit="solves/s", sample=int(len(sample)),
                      note="one FP64 instance per solver object and launch, same eps, accel")

        cpu = None
        oracle_score = None
        if not args.no_cpu_baseline:
            n_cpu, dt_cpu, cores, idx_cpu = oracle_sample(insts, cfg, 20.0)
            cpu = dict(value=n_cpu / dt_cpu, unit="solves/s", cores=cores, kind="oracle",
                       sample=f"{n_cpu} random instances of the {batch}-instance workload "
                              f"(all iterations to the same eps), {dt_cpu:.1f} s")
            # Accuracy against the converged oracle on the first instances of that sample.
            t0 = time.perf_counter()
            idx_s = idx_cpu[:cfg["oracle_score_sample"]]
            wo = oracle_converged(insts, idx_s)
            e32 = [rel_err(np.concatenate([uu[ou[j]:ou[j + 1]], xx[ox[j]:ox[j + 1]]]), w)
                   for j, w in zip(idx_s, wo)]
            e64 = [rel_err(np.concatenate([ur[ou[j]:ou[j + 1]], xr[ox[j]:ox[j + 1]]]), w)
                   for j, w in zip(idx_s, wo)]
            oracle_score = dict(ok=int(np.sum(np.array(e32) <= cfg["accuracy"])), of=len(idx_s),
                                max_err=float(np.max(e32)),
                                fp64_reference_max_err=float(np.max(e64)),
                                seconds=time.perf_counter() - t0,
                                oracle="FP64 CPU oracle run to c <= 1e-22")

        extras = dict(
            fp64_polish=extra(bench_polish, torch, pimpc, make, d, p, cfg, tot_u, tot_x, (ur, xr),
                              ou, ox),
            differentiable_cartpole=extra(bench_cartpole, torch, pimpc, W, args.steps),
            differentiable_cartpole_resident=extra(bench_cartpole, torch, pimpc, W, args.steps,
                                                   family=pimpc.FAMILY_RESIDENT),
            single_instance_latency=extra(bench_latency, torch, pimpc, W),
            temporal_blocking_plain=extra(bench_temporal_blocking, torch, pimpc, W, cfg),
            quadrotor_rti_f64=extra(bench_rti, torch, pimpc, W, pimpc.F64),
            quadrotor_rti_f32=extra(bench_rti, torch, pimpc, W, pimpc.F32),
            quadrotor_rti_f64_resident=extra(bench_rti, torch, pimpc, W, pimpc.F64,
                                             family=pimpc.FAMILY_RESIDENT),
            quadrotor_rti_f32_resident=extra(bench_rti, torch, pimpc, W, pimpc.F32,
                                             family=pimpc.FAMILY_RESIDENT),
            large_state_lti=extra(bench_large_lti, torch, pimpc, W),
            cstr_nmpc_f64_resident=extra(bench_cstr, torch, pimpc, W, pimpc.F64,
                                         family=pimpc.FAMILY_RESIDENT),
            cstr_nmpc_f32_resident=extra(bench_cstr, torch, pimpc, W, pimpc.F32,
                                         family=pimpc.FAMILY_RESIDENT),
            afti16_f64=extra(bench_afti16, pimpc, W, pimpc.F64, family=pimpc.FAMILY_RESIDENT),
        ) if not args.no_extras else None

        n_stages = int(np.sum(N))
        stage_bytes = float(np.sum(N * (matrix_words(nx, nu) + 10 * (nx + nu)))) * 4
        line = dict(
            metric=METRIC, value=value, unit="solves/s", n_gpus=world, steps=args.steps,
            warmup=args.warmup, ms_per_step=ms_max, higher_is_better=True, scaling="weak",
            vs_baseline=None, dtype="f32", data="synthetic",
            config=dict(workload=cfg["name"], instances_per_gpu=batch, stages_per_gpu=n_stages,
                        nx="4..24", nu="2..8", N="50..500", eps=cfg["eps"], accel=cfg["accel"],
                        stall=dict(window=cfg["stall_window"], factor=cfg["stall_factor"]),
                        max_iters=cfg["max_iters"], factorisation="fp64",
                        l2="no flush: stage data %.1f GB per GPU >> 129 MB L2" % (stage_bytes / 1e9),
                        parallelism=f"replicas x{world}" if world > 1 else "single GPU"),
            iters_per_s=it_all / (ms_max / 1e3),
            stage_iters_per_s=stit_all / (ms_max / 1e3),
            accuracy=dict(ok=ok, of=batch, threshold=cfg["accuracy"],
                          median_err=float(np.median(err)), max_err=float(np.max(err)),
                          converged=int(np.sum(status == pimpc.CONVERGED)),
                          stalled=int(np.sum(status == pimpc.STALLED)),
                          mean_iters=float(np.mean(iters)),
                          reference="this GPU's FP64 path, c <= %g" % cfg["ref_eps"],
                          against_oracle=oracle_score),
            schedule=dict(pimpc.pimpc_get_schedule(h), autotuned=tuned, graph=graph_stats),
            breakdown_ms=dict(factorise=float(np.mean(fact_ms)), solve=float(np.mean(solve_ms))),
            roofline=dict(bound="hbm", achieved=achieved, peak=peak, unit="GB/s",
                          frac=achieved / peak, traffic=traffic,
                          traffic_source=None if traffic is None else
                          "DRAM bytes per algorithmic byte of an ncu capture of the same kernel "
                          "source (profiles/), times this launch's algorithmic bytes",
                          kernel=kernel_name, peak_kind=peak_kind,
                          algorithmic_bytes_per_launch=alg),
            fp64_single_instance_gpu=single,
            cpu_baseline=cpu,
            e2e=e2e,
            gpu_launches=8 * args.steps,
            clocks=clk,
            extras=extras,
        )
        print(json.dumps(line), flush=True)
    pimpc.pimpc_destroy(h)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def main():
    args = parse_args()
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
