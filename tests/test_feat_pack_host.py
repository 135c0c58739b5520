"""The packed feature-row format of the flow path's kd build, pinned on the host.

`pack_feat_row` (paper_1508_05151_gb300/csrc/ff_internal.cuh) is compiled into a
small host program that packs rows of values, including the extremes a WHT feature
of radius 8 can take (+-289 * 255 = +-73,695) and the limits of the 18-bit field
(-2^17 .. 2^17 - 1). The program decodes each row with its own code written from
the documented layout (value j, biased by 2^17, at bits [18 j, 18 j + 18) of 16
little-endian 32-bit words; bits 486..511 zero), not with the library's unpacker.
No GPU is needed."""
import os
import shutil
import subprocess

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1508_05151_gb300", "csrc")

PROGRAM = r"""
#include <cstdio>
#include <cstdint>
#include "ff_internal.cuh"
int main() {
  int32_t v[28];
  uint32_t w[ff::FEAT_PACKED_WORDS];
  while (true) {
    for (int j = 0; j < 27; j++)
      if (scanf("%d", &v[j]) != 1) return 0;
    v[27] = 0;
    ff::pack_feat_row(v, w);
    for (int j = 0; j < 27; j++) {
      const int bit = 18 * j;
      unsigned long long two = w[bit / 32];
      if (bit / 32 + 1 < 16) two |= (unsigned long long)w[bit / 32 + 1] << 32;
      const int u = (int)((two >> (bit % 32)) & 0x3ffffu);
      printf("%d ", u - (1 << 17));
    }
    printf("%u\n", w[15] >> (486 - 480));  // bits 486..511 must stay zero
  }
}
"""


def test_packed_rows_round_trip_and_bounds(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(nvcc):
        pytest.skip("nvcc not available")
    src = tmp_path / "pack.cu"
    src.write_text(PROGRAM)
    exe = tmp_path / "pack"
    subprocess.run([nvcc, "-std=c++17", "-I", CSRC, "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe)], check=True, capture_output=True, timeout=600)
    rng = np.random.default_rng(3)
    rows = [rng.integers(-73695, 73696, size=27) for _ in range(300)]
    rows.append(np.full(27, -73695))
    rows.append(np.full(27, 73695))
    rows.append(np.full(27, -(1 << 17)))
    rows.append(np.full(27, (1 << 17) - 1))
    rows.append(np.arange(27) * 4099 - 50000)
    inp = "\n".join(" ".join(str(int(x)) for x in r) for r in rows) + "\n"
    out = subprocess.run([str(exe)], input=inp, capture_output=True, text=True, check=True,
                         timeout=120).stdout.split("\n")
    for r, line in zip(rows, out):
        got = [int(x) for x in line.split()]
        assert got[:27] == [int(x) for x in r]
        assert got[27] == 0
