"""The chunk-stream buffers are sized n (256 + 12 c) bytes per factor, c the longest row
(factor-row or expanded-row capacity): checks, with the kernels' own size functions compiled
for the host, that every chunk the packing can form -- any number of rows r >= 1, segments
1..min(r, kMaxSeg), entries e up to r c -- stays within 256 r + 12 e bytes in both stream forms
and both precisions, so the rows' share of the buffer always covers their chunks; and that one
row of the largest allowed expanded-row capacity fits the smallest ring slot."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1008_5113_gb300", "csrc")

PROG = r"""
#include <cstdio>
#include "vmc_device.cuh"
using namespace vmc;
int main() {
  long bad = 0, checked = 0;
  for (int tsz = 4; tsz <= 8; tsz += 4)
    for (int r = 1; r <= 96; ++r)
      for (int ns = 1; ns <= r && ns <= kMaxSeg; ++ns)
        for (int e = 0; e <= r * 160; e += (e < 64 ? 1 : 7)) {
          const long lim = 256L * r + 12L * e;
          for (int up = 0; up < 2; ++up) {
            ++checked;
            if (chunk_bytes(ns, r, e, tsz, up != 0) > lim) ++bad;
          }
          ++checked;
          if (chunk_bytes_grouped(ns, r, e, tsz) > lim) ++bad;
          if (chunk_bytes_grouped(ns, r, e, tsz) % 16 || chunk_bytes(ns, r, e, tsz, true) % 16) ++bad;
        }
  // one row at the largest expanded-row capacity (480 entries, rounded to 484) in the smallest slot
  const int one = chunk_bytes_grouped(1, 1, 484, 8) > chunk_bytes(1, 1, 484, 8, true)
                      ? chunk_bytes_grouped(1, 1, 484, 8) : chunk_bytes(1, 1, 484, 8, true);
  std::printf("%ld %ld %d %d\n", checked, bad, one, kSlotBytes);
  return 0;
}
"""


def test_stream_chunks_fit_their_rows_share(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "cap.cu"
    src.write_text(PROG)
    exe = tmp_path / "cap"
    subprocess.run([nvcc, "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-I", CSRC,
                    "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    checked, bad, one, slot = map(int, subprocess.run([str(exe)], check=True, capture_output=True,
                                                      text=True).stdout.split())
    assert checked > 100000 and bad == 0
    assert one <= slot
