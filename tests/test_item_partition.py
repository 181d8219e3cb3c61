"""Host-side checks of the work-item arithmetic shared by the central-list scan and the query
kernel (include of the library's internal header, compiled for the host with nvcc; no GPU).

The scan splits the centrals of a cell into full items of 32 / lanes_per_central centrals and
one remainder; the query derives each item's lanes per central from its count alone
(item_lanes).  Both must agree, every lane group must fit in a warp, and the "very heavy" rule
must order items by the work per lane."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

HARNESS = r"""
#include <cstdio>
#include "ps_internal.cuh"
using namespace ps;
int main() {
  int bad = 0;
  // item_lanes: a power of two <= 8 with cnt * L <= 32, and the largest such (or 8)
  for (uint32_t cnt = 4; cnt <= 32; ++cnt) {
    const uint32_t L = item_lanes(cnt);
    const bool pow2 = L == 1 || L == 2 || L == 4 || L == 8;
    if (!pow2 || cnt * L > 32 || (L < 8 && cnt * 2 * L <= 32)) { printf("item_lanes(%u) = %u\n", cnt, L); ++bad; }
  }
  // a full item of a cell split by lanes_per_central (32 / Lx centrals) gets Lx back
  for (uint32_t Lx = 1; Lx <= 4; Lx *= 2)
    if (item_lanes(32 / Lx) != Lx) { printf("full item of %u lanes\n", Lx); ++bad; }
  // lanes_per_central: 1, 2 or 4, nondecreasing in the candidate count
  for (int st = 1; st <= 2; ++st) {
    uint32_t prev = 1;
    for (uint32_t cand = 0; cand <= 200000; cand += 7) {
      const uint32_t L = lanes_per_central(cand, 1000, 100, st);
      if (!(L == 1 || L == 2 || L == 4) || L < prev) { printf("lanes_per_central(%u) = %u\n", cand, L); ++bad; }
      prev = L;
    }
    // the thresholds: 16x and 32x the mean stencil population (w * n_nbr / n_cells)
    const uint32_t w = (2 * st + 1) * (2 * st + 1) * (2 * st + 1), mean = w * 1000 / 100;
    if (lanes_per_central(16 * mean - 1, 1000, 100, st) != 1 || lanes_per_central(16 * mean, 1000, 100, st) != 2 ||
        lanes_per_central(32 * mean - 1, 1000, 100, st) != 2 || lanes_per_central(32 * mean, 1000, 100, st) != 4) {
      printf("lanes_per_central thresholds, stencil %d\n", st);
      ++bad;
    }
    // very_heavy: each lane tests >= 8x the mean population; more lanes make an item lighter
    for (uint32_t L = 1; L <= 8; L *= 2) {
      if (very_heavy(8 * mean * L - 1, L, 1000, 100, st) || !very_heavy(8 * mean * L, L, 1000, 100, st)) {
        printf("very_heavy threshold, L = %u, stencil %d\n", L, st);
        ++bad;
      }
    }
  }
  // no overflow at the largest sizes (2^32 - 1 candidates, 2^31 cells)
  if (!very_heavy(0xFFFFFFFFu, 1, 1u << 31, 1u << 31, 1) || lanes_per_central(0xFFFFFFFFu, 0xFFFFFFFFu, 1u << 31, 2) != 4) {
    printf("overflow\n");
    ++bad;
  }
  printf(bad ? "FAIL %d\n" : "OK\n", bad);
  return bad ? 1 : 0;
}
"""


def test_work_item_arithmetic(tmp_path):
    nvcc = shutil.which("nvcc") or ("/usr/local/cuda/bin/nvcc" if os.path.exists("/usr/local/cuda/bin/nvcc") else None)
    if nvcc is None:
        pytest.skip("nvcc not found")
    src = tmp_path / "items.cu"
    src.write_text(HARNESS)
    exe = tmp_path / "items"
    subprocess.check_call([nvcc, "-std=c++17", "-I", os.path.join(ROOT, "paper_2004_05188_gb300", "csrc"),
                           "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(src)])
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip().endswith("OK"), r.stdout
