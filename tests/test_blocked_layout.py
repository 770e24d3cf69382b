"""The blocked stage-block layout (schedule family 5) checked on the CPU against the mathematics.

The layout helpers of `csrc/pimpc_internal.cuh` and `csrc/bl_slot.cuh` are host-callable: a small
C++ program compiled here with g++ includes them and prints, for every matrix size m = 1..64,
the block count, the number of stored block diagonals, the storage size, the storage index of
every (block diagonal d, block row I, row a, column b) slot and the slot decode of every storage
word, plus the G strides and block offsets. The test then checks what the solve kernel and the
factorisation rely on:
  * the storage index is injective into [0, bl_sym_words(m)) and leaves only the padding of the
    diagonal-block region unused, and the slot decode the factorisation writes through inverts
    it; the slots are exactly the upper triangles of the diagonal blocks, the blocks
    S_{I,(I+d) mod nb} for 0 < d < nb/2 and, for d = nb/2, the block rows I below nb/2 of an
    even nb (every element of a symmetric matrix once, up to symmetry); the diagonal blocks'
    pairs and every other block row are aligned for the kernel's vector reads;
  * storing those blocks holds every element of a symmetric m x m matrix;
  * the per-lane product the kernel runs (the diagonal block rebuilt from its upper triangle;
    per further full block diagonal: block (I, I+d) against h_{I+d}, the transpose of block
    (I-d, I) against h_{I-d}; the middle diagonal of an even nb: block (I, I+nb/2) for
    I < nb/2, else the transpose of block (I-nb/2, I)) reproduces S h;
  * G rows start 16-byte aligned; the FP32 row products (lane l reads row l, in a rotated block
    order for block counts 4 and 8) and 8 consecutive FP64 rows hit distinct 16-byte bank
    groups; every offset inside a block is 16-byte aligned.
"""
import os
import shutil
import subprocess

import numpy as np
import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(os.path.dirname(HERE), "paper_2601_14414_gb300", "csrc")
CUDA_INC = "/usr/local/cuda/include"

HARNESS = r"""
#include <cstdio>
#include "bl_slot.cuh"
using namespace pimpc;
int main() {
  for (int m = 1; m <= 64; ++m) {
    const int nb = bl_nb(m), D = bl_diags(nb);
    std::printf("M %d %d %d %d %d %d\n", m, nb, D, bl_sym_words(m), bl_ldg(m, 4), bl_ldg(m, 8));
    for (int d = 0; d < D; ++d)
      for (int I = 0; I < nb; ++I)
        for (int a = 0; a < 4; ++a)
          for (int b = 0; b < 4; ++b)
            if (bl_sym_stored(nb, d, I, a, b))
              std::printf("S %d %d %d %d %d\n", d, I, a, b, bl_sym_index(nb, d, I, a, b));
    for (int w = 0; w < bl_sym_words(m); ++w) {
      int d, I, a, b;
      const bool held = bl_sym_slot(nb, w, d, I, a, b);
      std::printf("W %d %d %d %d %d %d\n", w, held ? 1 : 0, d, I, a, b);
    }
  }
  for (int nx = 1; nx <= 40; ++nx)
    for (int nu = 1; nu <= 24; ++nu)
      for (int ts : {4, 8})
        std::printf("B %d %d %d %d %d %d %d %d\n", nx, nu, ts, bl_oE(nx, nu, ts), bl_oH(nx, nu, ts),
                    bl_oM(nx, nu, ts), bl_block_words(nx, nu, ts), bl_rec(nx + nu));
  return 0;
}
"""


@pytest.fixture(scope="module")
def layout(tmp_path_factory):
    gxx = shutil.which("g++")
    if gxx is None or not os.path.isdir(CUDA_INC):
        pytest.skip("g++ or the CUDA headers are not available")
    d = tmp_path_factory.mktemp("bl")
    src = d / "h.cpp"
    exe = d / "h"
    src.write_text(HARNESS)
    subprocess.run([gxx, "-std=c++17", "-O1", "-I", CSRC, "-I", CUDA_INC, str(src), "-o", str(exe)],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout
    mats, blocks, cur = {}, [], None
    for line in out.splitlines():
        f = line.split()
        if f[0] == "M":
            m, nb, D, words, ld4, ld8 = map(int, f[1:])
            cur = dict(nb=nb, D=D, words=words, ld4=ld4, ld8=ld8, idx={})
            mats[m] = cur
        elif f[0] == "S":
            dd, I, a, b, k = map(int, f[1:])
            cur["idx"][(dd, I, a, b)] = k
        elif f[0] == "W":
            w, held, dd, I, a, b = map(int, f[1:])
            cur.setdefault("slot", {})[w] = (dd, I, a, b) if held else None
        else:
            blocks.append(tuple(map(int, f[1:])))
    return mats, blocks


def test_storage_index_is_a_bijection(layout):
    mats, _ = layout
    for m, L in mats.items():
        nb = L["nb"]
        assert nb == (m + 3) // 4 and L["D"] == nb // 2 + 1
        vals = sorted(L["idx"].values())
        assert len(set(vals)) == len(vals), m
        d0w = (10 * nb + 3) // 4 * 4
        unused = set(range(L["words"])) - set(vals)
        assert unused == set(range(10 * nb, d0w)), m  # only the diagonal region's padding
        slots = {(d, I) for (d, I, a, b) in L["idx"]}
        want = {(d, I) for d in range(nb // 2 + 1) for I in range(nb)
                if 2 * d < nb or (2 * d == nb and I < nb // 2) or nb == 1}
        assert slots == want, m
        # one slot per block of the upper block triangle (I <= J) of the padded matrix
        assert len(slots) == nb * (nb + 1) // 2, m
        # the diagonal blocks hold exactly their upper triangles, at 10 I, read as aligned pairs
        for I in range(nb):
            tri = sorted(k for (d, J, a, b), k in L["idx"].items() if d == 0 and J == I)
            assert tri == list(range(10 * I, 10 * I + 10)), (m, I)
            assert {(a, b) for (d, J, a, b) in L["idx"] if d == 0 and J == I} == \
                {(a, b) for a in range(4) for b in range(a, 4)}, (m, I)
        # rows of the other blocks start 16-byte aligned (FP32 words) and run over 4 slots
        for (d, I, a, b), k in L["idx"].items():
            if d > 0:
                assert (k - b) % 4 == 0 and L["idx"][(d, I, a, 0)] + b == k, (m, d, I, a, b)


def test_slot_decode_inverts_the_storage_index(layout):
    # bl_sym_slot (the factorisation writes every slot through it) returns, for each slot, the
    # element whose storage index it is, and reports only the diagonal region's padding as empty
    mats, _ = layout
    for m, L in mats.items():
        inv = {k: key for key, k in L["idx"].items()}
        assert sorted(L["slot"]) == list(range(L["words"])), m
        for w, key in L["slot"].items():
            assert key == inv.get(w), (m, w, key)


def stored(L, S):
    """The storage array of the symmetric matrix S (zero-padded to 4 nb) in the blocked layout."""
    nb, D = L["nb"], L["D"]
    P = np.zeros((4 * nb, 4 * nb))
    P[:S.shape[0], :S.shape[0]] = S
    H = np.zeros(L["words"])
    for (d, I, a, b), k in L["idx"].items():
        H[k] = P[4 * I + a, 4 * ((I + d) % nb) + b]
    return H


def test_every_element_is_held_and_the_lane_products_give_S_h(layout):
    mats, _ = layout
    rng = np.random.default_rng(0)
    for m, L in mats.items():
        nb, D, idx = L["nb"], L["D"], L["idx"]
        A = rng.standard_normal((m, m))
        S = A + A.T
        H = stored(L, S)
        # every element, read back through the block diagonal that holds it (or its transpose)
        for r in range(m):
            for c in range(m):
                I, a, J, b = r // 4, r % 4, c // 4, c % 4
                d = (J - I) % nb
                if 2 * d > nb or (2 * d == nb and I >= nb // 2 and nb > 1) or (d == 0 and a > b):
                    d, I, J, a, b = (nb - d) % nb, J, I, b, a
                assert H[idx[(d, I, a, b)]] == S[r, c]
        # the lane products of the solve kernel
        h = np.zeros(4 * nb)
        h[:m] = rng.standard_normal(m)
        y = np.zeros(4 * nb)
        def block(d, I):
            return np.array([[H[idx[(d, I, a, b)]] for b in range(4)] for a in range(4)])

        def diag_block(I):
            t = [H[10 * I + q] for q in range(10)]  # s00 s01 s02 s03 s11 s12 s13 s22 s23 s33
            return np.array([[t[0], t[1], t[2], t[3]], [t[1], t[4], t[5], t[6]],
                             [t[2], t[5], t[7], t[8]], [t[3], t[6], t[8], t[9]]])
        Df = (nb + 1) // 2
        for I in range(nb):
            y[4 * I:4 * I + 4] += diag_block(I) @ h[4 * I:4 * I + 4]
            for d in range(1, Df):
                Jp = (I + d) % nb
                y[4 * I:4 * I + 4] += block(d, I) @ h[4 * Jp:4 * Jp + 4]
                Jm = (I - d) % nb
                y[4 * I:4 * I + 4] += block(d, Jm).T @ h[4 * Jm:4 * Jm + 4]
            if nb % 2 == 0:
                hb = nb // 2
                if I < hb:
                    y[4 * I:4 * I + 4] += block(hb, I) @ h[4 * (I + hb):4 * (I + hb) + 4]
                else:
                    y[4 * I:4 * I + 4] += block(hb, I - hb).T @ h[4 * (I - hb):4 * (I - hb) + 4]
        np.testing.assert_allclose(y[:m], S @ h[:m], rtol=1e-12, atol=1e-12)
        assert np.all(y[m:] == 0)


def test_g_stride_and_offsets(layout):
    mats, blocks = layout
    for m, L in mats.items():
        nb = L["nb"]
        for ld, word in ((L["ld4"], 4), (L["ld8"], 8)):
            assert ld >= 4 * nb and (ld * word) % 16 == 0
        # FP64: 8 consecutive rows start in 8 distinct 16-byte bank groups
        units = L["ld8"] * 8 // 16
        assert len({(r * units) % 8 for r in range(8)}) == 8, m
        # FP32: the row products (lane l of a group of g lanes reads row l, at step J block J,
        # or block (J + l) mod nb for nb = 4 and 8) put the lanes of a quarter warp
        # that belong to one group on distinct 16-byte bank groups at every step
        units = L["ld4"] * 4 // 16
        g = 4 if m <= 16 else (8 if m <= 32 else 16)
        rot = nb in (4, 8)
        assert L["ld4"] == 4 * nb or L["ld4"] == 4 * (nb + 1), m
        for J in range(nb):
            for q0 in range(0, g, 8):
                lanes = range(q0, min(g, q0 + 8))
                banks = [(l * units + ((J + l) % nb if rot else J)) % 8 for l in lanes]
                assert len(set(banks)) == len(banks), (m, J)
    for nx, nu, ts, oE, oH, oM, W, rec in blocks:
        n = nx + nu
        ld = mats[n]["ld4"] if ts == 4 else mats[n]["ld8"]
        assert oE == nx * ld and oH == oE + (nx + 3) // 4 * 4
        assert oM == oH + mats[n]["words"] and W >= oM + nu * (nu + 1) // 2
        for off in (oE, oH, oM, W, rec):
            assert (off * ts) % 16 == 0, (nx, nu, ts, off)
        assert rec == 5 * ((n + 3) // 4 * 4)
