"""Plain FP64 CPU oracle for the piMPC hot path (arXiv 2601.14414) -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference leg may
import this package. The CUDA library never imports, links or calls it, and the two share no code:
the C source here (``pimpc_oracle.c``) is a separate, slow, dense restatement of Algorithm 1 of the
paper, and this module only marshals numpy arrays into it.

Instances are plain dicts (built by ``paper_2601_14414_gb300.workloads``):
``nx, nu, N, A, B, e, q, r, rdu, xmin, xmax, umin, umax, x0, u_prev, ref, rho`` and ``lti``.
With ``lti`` true, ``A`` is ``[nx, nx]``, ``B`` is ``[nx, nu]`` and ``e`` is ``[nx]`` for every stage;
otherwise they carry a leading stage axis of length ``N``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from concurrent.futures import ThreadPoolExecutor

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "pimpc_oracle.c")
_HDR = os.path.join(_HERE, "pimpc_oracle.h")
_BUILD = os.path.join(_HERE, "_build")
_SO = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

CONVERGED, MAXITER, NONFINITE = 0, 1, 2
USET_BOX, USET_BALL2, USET_BALL1, USET_HALFSPACE, USET_SOC = 0, 1, 2, 3, 4
MODEL_QUADROTOR, MODEL_CARTPOLE, MODEL_CSTR = 0, 1, 2

_dp = ctypes.POINTER(ctypes.c_double)
_ip = ctypes.POINTER(ctypes.c_int)
_up = ctypes.POINTER(ctypes.c_ubyte)


class _Problem(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("nu", ctypes.c_int), ("N", ctypes.c_int),
                ("A", _dp), ("B", _dp), ("e", _dp), ("q", _dp), ("r", _dp), ("rdu", _dp),
                ("xmin", _dp), ("xmax", _dp), ("umin", _dp), ("umax", _dp),
                ("x0", _dp), ("u_prev", _dp), ("ref", _dp), ("rho", ctypes.c_double),
                ("uset", ctypes.c_int), ("uset_r", ctypes.c_double), ("uset_a", _dp)]


class _Options(ctypes.Structure):
    _fields_ = [("eps", ctypes.c_double), ("max_iters", ctypes.c_int), ("accel", ctypes.c_int),
                ("eta", ctypes.c_double), ("force_mask", _up)]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (FP64, no FMA contraction). Returns the library path."""
    with _lock:
        stale = (not os.path.exists(_SO) or
                 os.path.getmtime(_SO) < max(os.path.getmtime(_SRC), os.path.getmtime(_HDR)))
        if force or stale:
            os.makedirs(_BUILD, exist_ok=True)
            tmp = _SO + f".tmp{os.getpid()}"
            subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math",
                                   "-fPIC", "-shared", "-o", tmp, _SRC, "-lm"])
            os.replace(tmp, _SO)
    return _SO


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_SO)
        P = ctypes.POINTER(_Problem)
        lib.orc_cache.argtypes = [P, _dp, _dp]
        lib.orc_iteration.argtypes = [P, _dp, _dp] + [_dp] * 5 + [_dp] * 7 + [_dp]
        lib.orc_solve.argtypes = [P, ctypes.POINTER(_Options)] + [_dp] * 7 + [_ip, _dp, _ip, _dp, _up]
        lib.orc_project_u.argtypes = [P, _dp, _dp]
        lib.orc_model_dims.argtypes = [ctypes.c_int, _ip, _ip]
        lib.orc_model_f.argtypes = [ctypes.c_int, _dp, _dp, _dp, _dp]
        lib.orc_linearise.argtypes = [ctypes.c_int, _dp, ctypes.c_double, ctypes.c_int, _dp, _dp,
                                      _dp, _dp, _dp]
        lib.orc_plant_step.argtypes = [ctypes.c_int, _dp, ctypes.c_double, _dp, _dp, _dp]
        _lib = lib
    return _lib


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def stage_arrays(inst):
    """Per-stage (A, B, e) of an instance as contiguous FP64 arrays, materialising LTI data."""
    N, nx, nu = inst["N"], inst["nx"], inst["nu"]
    if inst.get("lti", False):
        A = np.broadcast_to(np.asarray(inst["A"], np.float64), (N, nx, nx))
        B = np.broadcast_to(np.asarray(inst["B"], np.float64), (N, nx, nu))
        e = np.broadcast_to(np.asarray(inst["e"], np.float64), (N, nx))
        return _f64(A), _f64(B), _f64(e)
    return _f64(inst["A"]), _f64(inst["B"]), _f64(inst["e"])


def reference(inst):
    """The [N, n] reference for xbar_{k+1}, broadcasting a constant reference."""
    N, n = inst["N"], inst["nx"] + inst["nu"]
    return _f64(np.broadcast_to(np.asarray(inst["ref"], np.float64), (N, n)))


class _Bound:
    """Keeps the numpy buffers behind a ctypes problem struct alive."""

    def __init__(self, inst):
        A, B, e = stage_arrays(inst)
        self.keep = dict(A=A, B=B, e=e, q=_f64(inst["q"]), r=_f64(inst["r"]),
                         rdu=None if inst.get("rdu") is None else _f64(inst["rdu"]),
                         xmin=_f64(inst["xmin"]), xmax=_f64(inst["xmax"]),
                         umin=_f64(inst["umin"]), umax=_f64(inst["umax"]),
                         x0=_f64(inst["x0"]),
                         u_prev=None if inst.get("u_prev") is None else _f64(inst["u_prev"]),
                         ref=reference(inst))
        us = inst.get("uset") or dict(kind=USET_BOX, r=0.0, a=None)
        self.keep["uset_a"] = None if us.get("a") is None else _f64(us["a"])
        k = self.keep
        self.s = _Problem(inst["nx"], inst["nu"], inst["N"], _ptr(k["A"]), _ptr(k["B"]),
                          _ptr(k["e"]), _ptr(k["q"]), _ptr(k["r"]), _ptr(k["rdu"]),
                          _ptr(k["xmin"]), _ptr(k["xmax"]), _ptr(k["umin"]), _ptr(k["umax"]),
                          _ptr(k["x0"]), _ptr(k["u_prev"]), _ptr(k["ref"]), float(inst["rho"]),
                          int(us["kind"]), float(us.get("r", 0.0)), _ptr(k["uset_a"]))


def project_u(inst, y):
    """Euclidean projection of y [nu] onto the instance's input set."""
    lib = _load()
    pb = _Bound(inst)
    y = _f64(y)
    out = np.zeros(inst["nu"])
    if lib.orc_project_u(ctypes.byref(pb.s), _ptr(y), _ptr(out)):
        raise RuntimeError("oracle: unknown input set")
    return out


def cache(inst):
    """Explicit H[N, n, n] and J[N, nu, n] (Algorithm 1, 'cache')."""
    lib = _load()
    N, nx, nu = inst["N"], inst["nx"], inst["nu"]
    n = nx + nu
    pb = _Bound(inst)
    H = np.zeros((N, n, n))
    J = np.zeros((N, nu, n))
    if lib.orc_cache(ctypes.byref(pb.s), _ptr(H), _ptr(J)):
        raise RuntimeError("oracle: singular cache matrix")
    return H, J


def iteration(inst, H, J, hats):
    """One pass of Algorithm 1 steps 1-4 from hats = dict(z, v, th, be, la)."""
    lib = _load()
    N, nx, nu = inst["N"], inst["nx"], inst["nu"]
    n = nx + nu
    pb = _Bound(inst)
    H, J = _f64(H), _f64(J)
    hz, hv, hth, hbe, hla = (_f64(hats[k]) for k in ("z", "v", "th", "be", "la"))
    out = {k: np.zeros((N, n)) for k in ("z", "v", "th", "be", "la", "xb")}
    out["du"] = np.zeros((N, nu))
    c = ctypes.c_double()
    if lib.orc_iteration(ctypes.byref(pb.s), _ptr(H), _ptr(J), _ptr(hz), _ptr(hv), _ptr(hth),
                         _ptr(hbe), _ptr(hla), _ptr(out["du"]), _ptr(out["xb"]), _ptr(out["z"]),
                         _ptr(out["v"]), _ptr(out["th"]), _ptr(out["be"]), _ptr(out["la"]),
                         ctypes.byref(c)):
        raise RuntimeError("oracle: iteration failed")
    out["c"] = c.value
    return out


def solve(inst, eps=0.0, max_iters=200, accel=0, eta=0.999, force_mask=None, warm=None,
          history=False):
    """Algorithm 1 on one instance. Returns dict(z, v, th, be, la, du, xb, iters, c, status, u, x)
    plus c_hist / mask when ``history``. ``warm`` = dict(z, v, th, be, la) or None (cold start)."""
    lib = _load()
    N, nx, nu = inst["N"], inst["nx"], inst["nu"]
    n = nx + nu
    pb = _Bound(inst)
    st = {k: (np.zeros((N, n)) if warm is None else _f64(warm[k]).copy())
          for k in ("z", "v", "th", "be", "la")}
    du = np.zeros((N, nu))
    xb = np.zeros((N, n))
    fm = None
    if force_mask is not None:
        fm = np.ascontiguousarray(force_mask, dtype=np.uint8)
        assert fm.size >= max_iters
    opts = _Options(float(eps), int(max_iters), int(accel), float(eta),
                    None if fm is None else fm.ctypes.data_as(_up))
    it, cf, status = ctypes.c_int(), ctypes.c_double(), ctypes.c_int()
    ch = np.zeros(max(max_iters, 1)) if history else None
    mk = np.zeros(max(max_iters, 1), np.uint8) if history else None
    rc = lib.orc_solve(ctypes.byref(pb.s), ctypes.byref(opts), _ptr(st["z"]), _ptr(st["v"]),
                       _ptr(st["th"]), _ptr(st["be"]), _ptr(st["la"]), _ptr(du), _ptr(xb),
                       ctypes.byref(it), ctypes.byref(cf), ctypes.byref(status),
                       None if ch is None else _ptr(ch),
                       None if mk is None else mk.ctypes.data_as(_up))
    if rc:
        raise RuntimeError("oracle: solve failed (singular cache matrix or out of memory)")
    res = dict(st, du=du, xb=xb, iters=it.value, c=cf.value, status=status.value)
    res["x"] = st["z"][:, :nx].copy()
    res["u"] = st["z"][:, nx:].copy()
    if history:
        res["c_hist"] = ch[: it.value].copy()
        res["mask"] = mk[: it.value].copy()
    return res


def solve_batch(instances, threads=None, **opts):
    """Solve independent instances on a thread pool (the C call releases the GIL)."""
    threads = threads or os.cpu_count() or 1
    if threads == 1 or len(instances) == 1:
        return [solve(inst, **opts) for inst in instances]
    with ThreadPoolExecutor(max_workers=threads) as ex:
        return list(ex.map(lambda inst: solve(inst, **opts), instances))


def model_dims(model):
    lib = _load()
    nx, nu = ctypes.c_int(), ctypes.c_int()
    if lib.orc_model_dims(int(model), ctypes.byref(nx), ctypes.byref(nu)):
        raise ValueError(f"unknown model {model}")
    return nx.value, nu.value


def model_f(model, params, x, u):
    lib = _load()
    nx, _ = model_dims(model)
    p, x, u = _f64(params), _f64(x), _f64(u)
    f = np.zeros(nx)
    if lib.orc_model_f(int(model), _ptr(p), _ptr(x), _ptr(u), _ptr(f)):
        raise ValueError("oracle: model_f failed")
    return f


def plant_step(model, params, dt, x, u):
    lib = _load()
    nx, _ = model_dims(model)
    p, x, u = _f64(params), _f64(x), _f64(u)
    xn = np.zeros(nx)
    if lib.orc_plant_step(int(model), _ptr(p), float(dt), _ptr(x), _ptr(u), _ptr(xn)):
        raise ValueError("oracle: plant_step failed")
    return xn


def linearise(model, params, dt, xbar, ubar):
    """Explicit-Euler linearisation along xbar[N, nx], ubar[N, nu] -> A[N,nx,nx], B[N,nx,nu], e[N,nx]."""
    lib = _load()
    nx, nu = model_dims(model)
    xbar, ubar, p = _f64(xbar), _f64(ubar), _f64(params)
    N = xbar.shape[0]
    A = np.zeros((N, nx, nx))
    B = np.zeros((N, nx, nu))
    e = np.zeros((N, nx))
    if lib.orc_linearise(int(model), _ptr(p), float(dt), N, _ptr(xbar), _ptr(ubar), _ptr(A),
                         _ptr(B), _ptr(e)):
        raise ValueError("oracle: linearise failed")
    return A, B, e


def with_params(inst, **changes):
    """A shallow copy of an instance with some entries replaced (for finite differences)."""
    out = dict(inst)
    out.update(changes)
    return out


def unrolled_loss(inst, W_u, W_x, iters, accel=0, **kw):
    """L = <W_u, u> + <W_x, x> after exactly ``iters`` cold-started iterations (eps = -1)."""
    res = solve(inst, eps=-1.0, max_iters=iters, accel=accel, **kw)
    return float(np.sum(W_u * res["u"]) + np.sum(W_x * res["x"]))


def fd_gradient(inst, W_u, W_x, iters, name, h=1e-6, index=None):
    """Central finite difference dL/d(inst[name]) of the unrolled loss, in FP64.

    ``name`` is one of x0, ref, q, r, xmin, xmax, umin, umax. With ``index`` None the full
    gradient array is returned (one pair of solves per entry)."""
    base = np.array(inst[name], dtype=np.float64)
    if name == "ref":
        base = reference(inst).copy()
    grad = np.zeros_like(base)
    idxs = [index] if index is not None else list(np.ndindex(base.shape))
    for idx in idxs:
        p = base.copy(); p[idx] += h
        m = base.copy(); m[idx] -= h
        lp = unrolled_loss(with_params(inst, **{name: p}), W_u, W_x, iters)
        lm = unrolled_loss(with_params(inst, **{name: m}), W_u, W_x, iters)
        grad[idx] = (lp - lm) / (2 * h)
    return grad if index is None else grad[index]
