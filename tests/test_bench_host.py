"""Host logic of the roofline figures `bench.py` reports (no GPU).

* The algorithmic bytes of a solve: per stage-iteration the stage matrices (G, e, packed H and M)
  and the iterates read and written, plus the previous iterate on momentum iterations — checked
  against the sum written out by hand for small sizes.
* The profiled traffic: the DRAM bytes per algorithmic byte of the committed ncu summary are used
  only while the summary's source hash matches the kernel source and the headers compiled into
  it; a stale summary gives None.
"""
import hashlib
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def test_algorithmic_bytes_by_hand():
    nx, nu, N = np.array([2, 3]), np.array([1, 2]), np.array([4, 5])
    iters, mom = np.array([10, 7]), np.array([6, 0])
    total = 0
    for a, b, k, it, m in zip(nx, nu, N, iters, mom):
        n = a + b
        mats = a * n + a + n * (n + 1) // 2 + b * (b + 1) // 2   # G, e, packed H, packed M
        total += k * (it * (mats + 10 * n) + m * 5 * n)          # read + write 5n, prev 5n
    assert bench.algorithmic_bytes(nx, nu, N, iters, mom, 4) == 4.0 * total
    assert bench.algorithmic_bytes(nx, nu, N, iters, mom, 8) == 8.0 * total


def test_profiled_traffic_follows_the_source_hash(tmp_path, monkeypatch):
    csrc = tmp_path / "paper_2601_14414_gb300" / "csrc"
    csrc.mkdir(parents=True)
    (tmp_path / "profiles").mkdir()
    src = csrc / "admm_blk.cu"
    src.write_text('// kernel source\n#include "lockstep.cuh"\n#include <math.h>\n')
    (csrc / "lockstep.cuh").write_text('// lockstep.cuh\n#include "launch.h"\n')
    (csrc / "launch.h").write_text("// launch.h\n")
    (csrc / "tc.cuh").write_text("// tc.cuh\n")                # not included by the kernel
    monkeypatch.setattr(bench, "HERE", str(tmp_path))
    assert bench.kernel_files("admm_blk.cu") == ["admm_blk.cu", "launch.h", "lockstep.cuh"]
    h = hashlib.sha256()
    for name in ("admm_blk.cu", "launch.h", "lockstep.cuh"):
        h.update((csrc / name).read_bytes())
    digest = h.hexdigest()[:16]
    prof = tmp_path / "profiles" / "blk_kernel_f32_batched_512x30.md"
    prof.write_text(f"traffic_per_algorithmic_byte: 1.2345\n\nadmm_blk.cu sha256[:16]: {digest} (x)\n")
    assert bench.profiled_traffic(5) == 1.2345
    assert bench.profiled_traffic(7) is None            # no summary for that family
    (csrc / "tc.cuh").write_text("// changed\n")          # a header the kernel does not include
    assert bench.profiled_traffic(5) == 1.2345
    (csrc / "launch.h").write_text("// changed\n")        # an included header (through another)
    assert bench.profiled_traffic(5) is None
    (csrc / "launch.h").write_text("// launch.h\n")
    assert bench.profiled_traffic(5) == 1.2345
    src.write_text('// kernel source, changed\n#include "lockstep.cuh"\n#include <math.h>\n')
    assert bench.profiled_traffic(5) is None            # the kernel changed since the capture


def test_committed_summaries_name_their_source_and_ratio():
    for family, (_, source, name) in bench.SOLVE_KERNELS.items():
        text = open(os.path.join(ROOT, "profiles", name)).read()
        assert f"{source} sha256[:16]:" in text, name
        assert "traffic_per_algorithmic_byte:" in text, name
