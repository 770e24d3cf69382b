"""Thin Python binding of the C ABI in ``include/pimpc.h`` (argument marshalling only).

Every function named ``pimpc_*`` here calls the C entry point of the same name in the in-tree
``libpimpc.so``; nothing in this module computes any part of the solver. Arrays may be numpy
arrays (host memory) or CUDA torch tensors (device memory, passed by ``data_ptr()`` together with
the current torch stream); all arrays of one call must live in the same memory space. Missing
library -> ImportError/RuntimeError: there is no CPU fallback.

``Solver`` wraps one solver object and packs per-instance dicts (the format of
``paper_2601_14414_gb300.workloads``) into the concatenated FP64 layout the C ABI expects.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from . import build as _build

OK, EINVAL, ENOMEM, ECUDA, ESTATE = 0, 1, 2, 3, 4
CONVERGED, MAXITER, NONFINITE, TIMEOUT, FACTOR_FAILED, STALLED = 0, 1, 2, 3, 4, 5
USET_BOX, USET_BALL2, USET_BALL1, USET_HALFSPACE, USET_SOC = 0, 1, 2, 3, 4
F32, F64 = 0, 1
HOST, DEVICE = 0, 1
MODEL_QUADROTOR, MODEL_CARTPOLE, MODEL_CSTR = 0, 1, 2
MAX_N_LTV, MAX_N_LTI = 32, 64

_lib = None
_VP = ctypes.c_void_p
_I = ctypes.c_int
_D = ctypes.c_double

_SIGS = {
    "pimpc_create": (_I, [_I, _VP, _VP, _VP, _I, _I, _I, ctypes.POINTER(_VP)]),
    "pimpc_destroy": (None, [_VP]),
    "pimpc_last_error": (ctypes.c_char_p, [_VP]),
    "pimpc_set_weights": (_I, [_VP, _VP, _VP, _VP, _I, _VP]),
    "pimpc_set_bounds": (_I, [_VP, _VP, _VP, _VP, _VP, _I, _VP]),
    "pimpc_set_options": (_I, [_VP, _D, _D, _I, _I, _D]),
    "pimpc_set_dynamics": (_I, [_VP, _VP, _VP, _VP, _I, _VP]),
    "pimpc_linearise": (_I, [_VP, _I, _VP, _D, _VP, _VP, _I, _VP]),
    "pimpc_get_dynamics": (_I, [_VP, _VP, _VP, _VP, _I, _VP]),
    "pimpc_factorise": (_I, [_VP, _VP]),
    "pimpc_solve": (_I, [_VP, _VP, _VP, _VP, _I, _I, _VP, _VP, _VP, _VP, _VP, _I, _VP]),
    "pimpc_get_iterates": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _I, _VP]),
    "pimpc_get_stats": (_I, [_VP, _VP, _VP, _VP, _VP, _I, _VP]),
    "pimpc_set_restart_mask": (_I, [_VP, _VP, _I, _I, _VP]),
    "pimpc_set_wait_limit": (_I, [_VP, _I]),
    "pimpc_set_stall": (_I, [_VP, _I, _D, _D, _D]),
    "pimpc_set_input_set": (_I, [_VP, _VP, _VP, _VP, _I, _VP]),
    "pimpc_plant_step": (_I, [_VP, _I, _VP, _D, _VP, _VP, _VP, _I, _VP]),
    "pimpc_backward": (_I, [_VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _VP, _I, _I, _VP]),
    "pimpc_solve_static": (_I, [_I, _I, _I, _I] + [_VP] * 11 + [_D, _D, _I, _I, _D] + [_VP] * 6),
    "pimpc_set_schedule": (_I, [_VP, _I, _I, _I]),
    "pimpc_set_polish": (_I, [_VP, _I, _D]),
    "pimpc_set_graph": (_I, [_VP, _I]),
    "pimpc_get_graph_stats": (_I, [_VP] * 5),
    "pimpc_get_schedule": (_I, [_VP] * 7),
    "pimpc_autotune": (_I, [_VP, _I, _VP, _VP, _VP, _VP, _VP]),
}

EXPORTED = tuple(_SIGS)


def library_path() -> str:
    return _build.LIB


def load(build_if_stale: bool = True):
    """Load libpimpc.so (compiling it first if it is missing or older than its sources)."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_stale:
        _build.build()
    if not os.path.exists(_build.LIB):
        raise RuntimeError(f"libpimpc.so not found at {_build.LIB}; run the build first")
    lib = ctypes.CDLL(_build.LIB)
    for name, (res, args) in _SIGS.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


class PimpcError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"pimpc error {code}: {msg}")
        self.code = code


def _is_torch(x):
    return type(x).__module__.startswith("torch")


def _arg(x, mem_seen):
    """(pointer, mem) of an array argument; None -> NULL."""
    if x is None:
        return None, mem_seen
    if _is_torch(x):
        assert x.is_cuda and x.is_contiguous(), "device arrays must be contiguous CUDA tensors"
        mem = DEVICE
        p = x.data_ptr()
    else:
        assert isinstance(x, np.ndarray) and x.flags.c_contiguous
        mem = HOST
        p = x.ctypes.data
    if mem_seen is not None and mem != mem_seen:
        raise ValueError("all arrays of one call must be in the same memory space")
    return p, mem


def _marshal(*arrays):
    mem = None
    ptrs = []
    for a in arrays:
        p, mem = _arg(a, mem)
        ptrs.append(p)
    if mem is None:
        mem = HOST
    stream = None
    if mem == DEVICE:
        import torch
        stream = torch.cuda.current_stream().cuda_stream
    return ptrs, mem, stream


def _check(h, rc):
    if rc != OK:
        msg = load().pimpc_last_error(h)
        raise PimpcError(rc, msg.decode() if msg else "")


# ---- one Python function per C entry point ------------------------------------------------

def pimpc_create(nx, nu, N, lti, precision, device=0):
    lib = load()
    nx = np.ascontiguousarray(nx, dtype=np.int32)
    nu = np.ascontiguousarray(nu, dtype=np.int32)
    N = np.ascontiguousarray(N, dtype=np.int32)
    h = _VP()
    rc = lib.pimpc_create(len(nx), nx.ctypes.data, nu.ctypes.data, N.ctypes.data, int(lti),
                          int(precision), int(device), ctypes.byref(h))
    _check(None, rc)
    return h


def pimpc_destroy(h):
    load().pimpc_destroy(h)


def pimpc_set_weights(h, q, r, rdu=None):
    (pq, pr, prdu), mem, st = _marshal(q, r, rdu)
    _check(h, load().pimpc_set_weights(h, pq, pr, prdu, mem, st))


def pimpc_set_bounds(h, xmin, xmax, umin, umax):
    p, mem, st = _marshal(xmin, xmax, umin, umax)
    _check(h, load().pimpc_set_bounds(h, *p, mem, st))


def pimpc_set_options(h, rho, eps, max_iters, accel, eta=0.999):
    _check(h, load().pimpc_set_options(h, float(rho), float(eps), int(max_iters), int(accel),
                                       float(eta)))


def pimpc_set_dynamics(h, A, B, e=None):
    p, mem, st = _marshal(A, B, e)
    _check(h, load().pimpc_set_dynamics(h, *p, mem, st))


def pimpc_linearise(h, model, params, dt, xbar, ubar):
    (pp, px, pu), mem, st = _marshal(params, xbar, ubar)
    _check(h, load().pimpc_linearise(h, int(model), pp, float(dt), px, pu, mem, st))


def pimpc_get_dynamics(h, A=None, B=None, e=None):
    p, mem, st = _marshal(A, B, e)
    _check(h, load().pimpc_get_dynamics(h, *p, mem, st))


def pimpc_factorise(h, stream=None):
    _check(h, load().pimpc_factorise(h, stream))


def pimpc_solve(h, x0, u_prev=None, ref=None, ref_per_stage=False, warm_start=0, u_out=None,
                x_out=None, iters=None, c=None, status=None):
    p, mem, st = _marshal(x0, u_prev, ref, None, None)
    px0, pup, pref = p[0], p[1], p[2]
    outs, mem2, _ = _marshal(u_out, x_out, iters, c, status)
    if any(o is not None for o in (u_out, x_out, iters, c, status)) and mem2 != mem:
        raise ValueError("inputs and outputs must be in the same memory space")
    _check(h, load().pimpc_solve(h, px0, pup, pref, int(bool(ref_per_stage)), int(warm_start),
                                 *outs, mem, st))


def pimpc_get_iterates(h, z=None, v=None, theta=None, beta=None, lam=None):
    p, mem, st = _marshal(z, v, theta, beta, lam)
    _check(h, load().pimpc_get_iterates(h, *p, mem, st))


def pimpc_get_stats(h, iters=None, c=None, status=None, momentum_iters=None):
    p, mem, st = _marshal(iters, c, status, momentum_iters)
    _check(h, load().pimpc_get_stats(h, *p, mem, st))


def pimpc_set_input_set(h, kind, r, a=None):
    """kind: int [batch] (numpy host array or int32 CUDA tensor), r [batch], a [sum nu] or None."""
    if not _is_torch(kind):
        kind = np.ascontiguousarray(kind, dtype=np.int32)
    p, mem, st = _marshal(kind, r, a)
    _check(h, load().pimpc_set_input_set(h, *p, mem, st))


def pimpc_set_stall(h, window, factor=0.5, below=1e-9, rel=0.0):
    _check(h, load().pimpc_set_stall(h, int(window), float(factor), float(below), float(rel)))


def pimpc_set_wait_limit(h, polls):
    _check(h, load().pimpc_set_wait_limit(h, int(polls)))


def pimpc_set_restart_mask(h, mask, length):
    if mask is None:
        _check(h, load().pimpc_set_restart_mask(h, None, 0, HOST, None))
        return
    (pm,), mem, st = _marshal(mask)
    _check(h, load().pimpc_set_restart_mask(h, pm, int(length), mem, st))


def pimpc_plant_step(h, model, params, dt, x, u, x_next):
    p, mem, st = _marshal(params, x, u, x_next)
    _check(h, load().pimpc_plant_step(h, int(model), p[0], float(dt), p[1], p[2], p[3], mem, st))


def pimpc_backward(h, dL_du, dL_dx, g_x0=None, g_ref=None, g_q=None, g_r=None, g_xmin=None,
                   g_xmax=None, g_umin=None, g_umax=None, checkpoint_every=25):
    p, mem, st = _marshal(dL_du, dL_dx, g_x0, g_ref, g_q, g_r, g_xmin, g_xmax, g_umin, g_umax)
    _check(h, load().pimpc_backward(h, *p, int(checkpoint_every), mem, st))


def pimpc_solve_static(nx, nu, N, precision, A, B, e, q, r, xmin, xmax, umin, umax, x0, ref,
                       rho, eps, max_iters, accel, eta, u_out=None, x_out=None, iters=None,
                       c=None, status=None):
    """Single-instance solve that allocates nothing; every array is a CUDA tensor."""
    p, mem, st = _marshal(A, B, e, q, r, xmin, xmax, umin, umax, x0, ref, u_out, x_out, iters,
                          c, status)
    if mem != DEVICE:
        raise ValueError("pimpc_solve_static takes device arrays only")
    _check(None, load().pimpc_solve_static(int(nx), int(nu), int(N), int(precision), *p[:11],
                                           float(rho), float(eps), int(max_iters), int(accel),
                                           float(eta), *p[11:], st))


FAMILY_LANES, FAMILY_TILES, FAMILY_RESIDENT, FAMILY_CONTRACTION, FAMILY_BLOCKED = 0, 2, 3, 4, 5
FAMILY_TENSOR, FAMILY_TEMPORAL = 6, 7


def pimpc_set_graph(h, enable):
    _check(h, load().pimpc_set_graph(h, int(bool(enable))))


def pimpc_get_graph_stats(h):
    en, cap, rep = ctypes.c_int(), ctypes.c_longlong(), ctypes.c_longlong()
    why = ctypes.c_char_p()
    _check(h, load().pimpc_get_graph_stats(h, ctypes.byref(en), ctypes.byref(cap),
                                           ctypes.byref(rep), ctypes.byref(why)))
    return dict(enabled=bool(en.value), captures=cap.value, replays=rep.value,
                refused=why.value.decode() if why.value else None)


def pimpc_set_polish(h, polish_iters, polish_eps=0.0):
    _check(h, load().pimpc_set_polish(h, int(polish_iters), float(polish_eps)))


def pimpc_set_schedule(h, family, ctas_per_sm=0, item_scale=0):
    _check(h, load().pimpc_set_schedule(h, int(family), int(ctas_per_sm), int(item_scale)))


def pimpc_get_schedule(h):
    vals = [ctypes.c_int() for _ in range(6)]
    _check(h, load().pimpc_get_schedule(h, *[ctypes.byref(v) for v in vals]))
    keys = ("family", "ctas_per_sm", "item_scale", "grid", "threads", "items")
    return {k: v.value for k, v in zip(keys, vals)}


def pimpc_autotune(h, trial_iters=20):
    fam, cps, scale = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
    ms = ctypes.c_double()
    stream = None
    if load() is not None:
        try:
            import torch
            if torch.cuda.is_available():
                stream = torch.cuda.current_stream().cuda_stream
        except ImportError:
            pass
    _check(h, load().pimpc_autotune(h, int(trial_iters), ctypes.byref(fam), ctypes.byref(cps),
                                    ctypes.byref(scale), ctypes.byref(ms), stream))
    return dict(family=fam.value, ctas_per_sm=cps.value, item_scale=scale.value, ms=ms.value)


# ---- packing of per-instance dicts ----------------------------------------------------------

def _cat(parts):
    return np.ascontiguousarray(np.concatenate([np.asarray(p, np.float64).ravel() for p in parts]))


def pack(instances):
    """Concatenate instance dicts into the FP64 arrays of the C ABI (batch order, stage-major)."""
    out = {}
    out["nx"] = np.array([i["nx"] for i in instances], np.int32)
    out["nu"] = np.array([i["nu"] for i in instances], np.int32)
    out["N"] = np.array([i["N"] for i in instances], np.int32)
    lti = bool(instances[0].get("lti", False))
    assert all(bool(i.get("lti", False)) == lti for i in instances), "mixed lti flags"
    out["lti"] = lti
    if all("A" in i for i in instances):
        out["A"] = _cat([i["A"] for i in instances])
        out["B"] = _cat([i["B"] for i in instances])
        out["e"] = _cat([i["e"] for i in instances])
    for key in ("q", "r", "xmin", "xmax", "umin", "umax", "x0"):
        out[key] = _cat([i[key] for i in instances])
    out["rdu"] = None if all(i.get("rdu") is None for i in instances) else _cat(
        [np.zeros(i["nu"]) if i.get("rdu") is None else i["rdu"] for i in instances])
    out["u_prev"] = None if all(i.get("u_prev") is None for i in instances) else _cat(
        [np.zeros(i["nu"]) if i.get("u_prev") is None else i["u_prev"] for i in instances])
    per_stage = any(np.ndim(i["ref"]) == 2 for i in instances)
    if per_stage:
        out["ref"] = _cat([np.broadcast_to(np.asarray(i["ref"], np.float64),
                                           (i["N"], i["nx"] + i["nu"])) for i in instances])
    else:
        out["ref"] = _cat([i["ref"] for i in instances])
    out["ref_per_stage"] = per_stage
    out["rho"] = float(instances[0]["rho"])
    if any(i.get("uset") is not None for i in instances):
        us = [i.get("uset") or dict(kind=USET_BOX, r=0.0) for i in instances]
        out["uset_kind"] = np.array([u["kind"] for u in us], np.int32)
        out["uset_r"] = np.array([float(u.get("r", 0.0)) for u in us])
        out["uset_a"] = _cat([np.zeros(i["nu"]) if u.get("a") is None else u["a"]
                              for i, u in zip(instances, us)])
    return out


def split(flat, sizes):
    """Split a concatenated array into per-instance pieces of the given lengths."""
    offs = np.concatenate([[0], np.cumsum(sizes)])
    return [flat[offs[i]:offs[i + 1]] for i in range(len(sizes))]


class Solver:
    """One solver object for a batch of instances (see ``pack`` for the instance format)."""

    def __init__(self, instances, precision=F32, device=0, eps=1e-6, max_iters=1000, accel=1,
                 eta=0.999):
        self.p = pack(instances)
        self.batch = len(instances)
        self.lti = self.p["lti"]
        self.precision = precision
        self.h = pimpc_create(self.p["nx"], self.p["nu"], self.p["N"], self.lti, precision, device)
        self.nx, self.nu, self.N = self.p["nx"], self.p["nu"], self.p["N"]
        pimpc_set_weights(self.h, self.p["q"], self.p["r"], self.p["rdu"])
        pimpc_set_bounds(self.h, self.p["xmin"], self.p["xmax"], self.p["umin"], self.p["umax"])
        pimpc_set_options(self.h, self.p["rho"], eps, max_iters, accel, eta)
        if "A" in self.p:
            pimpc_set_dynamics(self.h, self.p["A"], self.p["B"], self.p["e"])
        if "uset_kind" in self.p:
            pimpc_set_input_set(self.h, self.p["uset_kind"], self.p["uset_r"], self.p["uset_a"])

    def close(self):
        if self.h is not None:
            pimpc_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def set_polish(self, polish_iters, polish_eps=0.0):
        pimpc_set_polish(self.h, polish_iters, polish_eps)

    def set_schedule(self, family, ctas_per_sm=0, item_scale=0):
        pimpc_set_schedule(self.h, family, ctas_per_sm, item_scale)

    def schedule(self):
        return pimpc_get_schedule(self.h)

    def autotune(self, trial_iters=20, cache=None):
        """Pick the fastest schedule for this batch (pimpc_autotune). With ``cache`` (a path
        to a JSON file) a batch with the same signature reuses the stored choice."""
        key = self.signature()
        if cache is not None:
            import json
            store = json.load(open(cache)) if os.path.exists(cache) else {}
            if key in store:
                c = store[key]
                self.set_schedule(c["family"], c["ctas_per_sm"], c["item_scale"])
                return dict(c, cached=True)
        res = pimpc_autotune(self.h, trial_iters)
        if cache is not None:
            store[key] = res
            with open(cache, "w") as f:
                json.dump(store, f, indent=1, sort_keys=True)
        return dict(res, cached=False)

    def signature(self):
        """Autotuner cache key: precision, stage kind, and the multiset of (nx, nu, N bucket)."""
        import hashlib
        buckets = sorted(zip(self.nx.tolist(), self.nu.tolist(), (self.N // 64).tolist()))
        h = hashlib.sha256(repr(buckets).encode()).hexdigest()[:16]
        return f"p{self.precision}-lti{int(self.lti)}-b{self.batch}-{h}"

    def set_options(self, eps, max_iters, accel, eta=0.999, rho=None):
        pimpc_set_options(self.h, self.p["rho"] if rho is None else rho, eps, max_iters, accel, eta)

    def solve(self, x0=None, warm_start=0):
        """Host-memory solve; returns per-instance lists of u [N, nu], x [N, nx] plus arrays
        iters, c, status."""
        x0 = self.p["x0"] if x0 is None else np.ascontiguousarray(x0, np.float64)
        tot_u = int(np.sum(self.N * self.nu))
        tot_x = int(np.sum(self.N * self.nx))
        u = np.zeros(tot_u)
        x = np.zeros(tot_x)
        it = np.zeros(self.batch, np.int32)
        c = np.zeros(self.batch)
        st = np.zeros(self.batch, np.int32)
        pimpc_solve(self.h, x0, self.p["u_prev"], self.p["ref"], self.p["ref_per_stage"],
                    warm_start, u, x, it, c, st)
        us = [a.reshape(n, m) for a, n, m in zip(split(u, self.N * self.nu), self.N, self.nu)]
        xs = [a.reshape(n, m) for a, n, m in zip(split(x, self.N * self.nx), self.N, self.nx)]
        return dict(u=us, x=xs, iters=it, c=c, status=st)

    def backward(self, dL_du, dL_dx, checkpoint_every=25):
        """Gradients of L w.r.t. the inputs of the last solve (host memory), given per-instance
        dL/du [N, nu] and dL/dx [N, nx]; the last solve must have run a fixed number of plain
        iterations from the zero start (eps < 0, accel = 0, warm_start = 0). Returns per-instance
        lists x0, q, r, xmin, xmax, umin, umax and ref ([N, n] or [n], like the reference)."""
        gu = _cat([np.asarray(a, np.float64) for a in dL_du])
        gx = _cat([np.asarray(a, np.float64) for a in dL_dx])
        n = self.nx + self.nu
        per_stage = self.p["ref_per_stage"]
        out = dict(x0=np.zeros(int(np.sum(self.nx))), q=np.zeros(int(np.sum(self.nx))),
                   r=np.zeros(int(np.sum(self.nu))), xmin=np.zeros(int(np.sum(self.nx))),
                   xmax=np.zeros(int(np.sum(self.nx))), umin=np.zeros(int(np.sum(self.nu))),
                   umax=np.zeros(int(np.sum(self.nu))),
                   ref=np.zeros(int(np.sum(self.N * n)) if per_stage else int(np.sum(n))))
        pimpc_backward(self.h, gu, gx, out["x0"], out["ref"], out["q"], out["r"], out["xmin"],
                       out["xmax"], out["umin"], out["umax"], checkpoint_every)
        res = {}
        for key in ("x0", "q", "xmin", "xmax"):
            res[key] = split(out[key], self.nx)
        for key in ("r", "umin", "umax"):
            res[key] = split(out[key], self.nu)
        if per_stage:
            res["ref"] = [a.reshape(m, k) for a, m, k in zip(split(out["ref"], self.N * n), self.N, n)]
        else:
            res["ref"] = split(out["ref"], n)
        return res

    def iterates(self):
        tot = int(np.sum(self.N * (self.nx + self.nu)))
        arrs = [np.zeros(tot) for _ in range(5)]
        pimpc_get_iterates(self.h, *arrs)
        sizes = self.N * (self.nx + self.nu)
        out = []
        for j in range(self.batch):
            n = int(self.nx[j] + self.nu[j])
            d = {}
            for key, a in zip(("z", "v", "th", "be", "la"), arrs):
                d[key] = split(a, sizes)[j].reshape(int(self.N[j]), n)
            out.append(d)
        return out
