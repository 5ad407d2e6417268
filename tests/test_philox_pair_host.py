"""The walks' hoisted Philox evaluations equal Philox4x32-10 itself: the R^3
walk's two-block and one-block forms (per-walk and per-step parts hoisted out of
rounds 0..2) on counters (0, k, i, p) and (1, k, i, p), and the R^n FP32 walk's
block form on counters (k, j, i, p) with j = 256 v + b; the device header's
functions compiled as host code by nvcc and run over random and structured
(seed, i, p, k, j)."""
import os
import subprocess
import tempfile

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")

SRC = r'''
#include <cstdio>
#include <random>
#include "dev_common.cuh"
using namespace mpwos;
int main() {
  std::mt19937_64 g(7);
  long bad = 0;
  for (int t = 0; t < 100000; ++t) {
    uint64_t seed = g(); uint32_t i = g(), p = g(), k = g();
    if (t % 3 == 0) { i = t; p = t / 5; k = t % 700; seed = t % 11; }
    const PhiloxKeys K = philox_keys((uint32_t)seed, (uint32_t)(seed >> 32));
    const PhiloxWalk w = philox_walk(i, p, K);
    U4 a, b;
    philox_step_pair(w, k, K, a, b);
    const U4 ra = philox4x32_10(0u, k, i, p, K), rb = philox4x32_10(1u, k, i, p, K);
    const U4 o = philox_step_one(w, k, K);
    bad += a.x != ra.x || a.y != ra.y || a.z != ra.z || a.w != ra.w ||
           b.x != rb.x || b.y != rb.y || b.z != rb.z || b.w != rb.w ||
           o.x != ra.x || o.y != ra.y || o.z != ra.z || o.w != ra.w;
    const Philox32Walk pw = philox32_walk(i, K);
    const Philox32Step st = philox32_step(pw, k, p, K);
    for (int q = 0; q < 4; ++q) {
      const uint32_t j = (q == 0) ? 0u : (q == 1) ? 255u : (q == 2) ? (uint32_t)(256 * (1 + t % 64) + (g() & 255)) : (uint32_t)g();
      const U4 h = philox32_block(pw.A0 ^ j, st, K);
      const U4 rh = philox4x32_10(k, j, i, p, K);
      bad += h.x != rh.x || h.y != rh.y || h.z != rh.z || h.w != rh.w;
    }
  }
  std::printf("%ld\n", bad);
  return bad != 0;
}
'''


@pytest.mark.skipif(not os.path.exists(NVCC), reason="nvcc not found")
def test_philox_step_pair_equals_generic():
    with tempfile.TemporaryDirectory() as d:
        src = os.path.join(d, "pair.cu")
        exe = os.path.join(d, "pair")
        with open(src, "w") as fh:
            fh.write(SRC)
        inc = os.path.join(ROOT, "paper_2606_21883_b300", "csrc")
        subprocess.run([NVCC, "-std=c++17", "-O2", "-I", inc, "-I", os.path.join(ROOT, "include"), src, "-o", exe],
                       check=True, capture_output=True)
        out = subprocess.run([exe], capture_output=True, text=True)
        assert out.returncode == 0 and out.stdout.strip() == "0", out.stdout
