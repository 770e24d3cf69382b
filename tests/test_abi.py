"""The C-ABI library builds for sm_103a, loads, and exports every entry point include/pimpc.h
declares; argument validation that needs no GPU rejects bad calls (CPU only)."""
import ctypes
import os
import re

import numpy as np

from paper_2601_14414_gb300 import build, pimpc

HEADER = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))), "include",
                      "pimpc.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(pimpc_[a-z_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    syms = declared_symbols()
    for name in ("pimpc_create", "pimpc_destroy", "pimpc_last_error", "pimpc_set_weights",
                 "pimpc_set_bounds", "pimpc_set_options", "pimpc_set_dynamics",
                 "pimpc_linearise", "pimpc_get_dynamics", "pimpc_factorise", "pimpc_solve", "pimpc_get_iterates", "pimpc_get_stats",
                 "pimpc_set_restart_mask", "pimpc_plant_step", "pimpc_backward"):
        assert name in syms


def test_library_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    assert set(pimpc.EXPORTED) == set(declared_symbols())


def test_create_rejects_bad_sizes_before_touching_a_device():
    lib = pimpc.load()
    h = ctypes.c_void_p()
    nx = np.array([4, 30], np.int32)
    nu = np.array([2, 8], np.int32)  # 30 + 8 > 32 for stage-varying data
    N = np.array([10, 10], np.int32)
    rc = lib.pimpc_create(2, nx.ctypes.data, nu.ctypes.data, N.ctypes.data, 0, 0, 0, ctypes.byref(h))
    assert rc == pimpc.EINVAL and not h.value
    assert b"nx + nu" in lib.pimpc_last_error(None)
    rc = lib.pimpc_create(0, nx.ctypes.data, nu.ctypes.data, N.ctypes.data, 0, 0, 0, ctypes.byref(h))
    assert rc == pimpc.EINVAL
    rc = lib.pimpc_create(1, nx.ctypes.data, nu.ctypes.data, N.ctypes.data, 0, 7, 0, ctypes.byref(h))
    assert rc == pimpc.EINVAL
    # stage-invariant data allows n = nx + nu up to 64, but nu stays within one warp's lanes
    nx1, nu1, N1 = (np.array([v], np.int32) for v in (20, 33, 10))
    rc = lib.pimpc_create(1, nx1.ctypes.data, nu1.ctypes.data, N1.ctypes.data, 1, 0, 0, ctypes.byref(h))
    assert rc == pimpc.EINVAL and not h.value
    assert b"nu <= 32" in lib.pimpc_last_error(None)


def test_pack_layout_is_batch_then_stage_major():
    from paper_2601_14414_gb300 import workloads as W
    insts = [W.random_ltv(s, nx, nu, N) for s, (nx, nu, N) in enumerate([(3, 1, 4), (5, 2, 2)])]
    p = pimpc.pack(insts)
    assert p["A"].size == 4 * 9 + 2 * 25
    np.testing.assert_array_equal(p["A"][:36], insts[0]["A"].ravel())
    np.testing.assert_array_equal(p["A"][36:], insts[1]["A"].ravel())
    assert p["x0"].size == 3 + 5 and p["umax"].size == 1 + 2


def test_static_entry_point_checks_options_like_set_options():
    # Rejected before any device is touched (no GPU needed): the pointers are never read.
    lib = pimpc.load()
    buf = np.zeros(64)
    ptr = ctypes.c_void_p(buf.ctypes.data)
    inf, nan = float("inf"), float("nan")
    for rho, eps, eta in ((inf, 1e-6, 0.999), (0.0, 1e-6, 0.999), (1.0, nan, 0.999),
                          (1.0, 1e-6, -0.5), (1.0, 1e-6, nan), (1.0, 1e-6, inf)):
        rc = lib.pimpc_solve_static(2, 1, 4, 0, *([ptr] * 11), ctypes.c_double(rho),
                                    ctypes.c_double(eps), 10, 1, ctypes.c_double(eta),
                                    *([None] * 5), None)
        assert rc == pimpc.EINVAL, (rho, eps, eta)
