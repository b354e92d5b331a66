"""The kernels' division by a run-time invariant divisor (multiply-high method) equals
integer division: checked on the CPU by compiling the same header code for the host."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1508_02960_gb300", "csrc")

SRC = r"""
#include <cstdio>
#include <cstdint>
#include "lbm_device.cuh"
using namespace lbm;
int main() {
  uint64_t bad = 0, checked = 0;
  uint32_t ds[] = {1u, 2u, 3u, 5u, 7u, 18u, 20u, 24u, 31u, 32u, 33u, 48u, 96u, 127u, 128u, 160u, 255u,
                   256u, 257u, 511u, 512u, 1000u, 4095u, 16384u, 65535u, 65536u, 1u << 20, (1u << 31) - 1u,
                   1u << 31, 0xFFFFFFFFu};
  for (uint32_t d : ds) {
    FastDiv f = make_fastdiv(d);
    // all n below 2^20, a sweep up to 2^32, and the neighbourhood of every multiple edge
    for (uint64_t n = 0; n < (1u << 20); ++n) { ++checked; if (fast_div((uint32_t)n, f) != (uint32_t)n / d) ++bad; }
    for (uint64_t n = 0; n <= 0xFFFFFFFFull; n += 65521ull) { ++checked; if (fast_div((uint32_t)n, f) != (uint32_t)n / d) ++bad; }
    for (uint64_t q = 1; q * d <= 0xFFFFFFFFull && q < 100000; q = q * 3 + 1)
      for (int o = -2; o <= 2; ++o) { uint64_t n = q * d + o; if (n > 0xFFFFFFFFull) continue;
        ++checked; if (fast_div((uint32_t)n, f) != (uint32_t)n / d) ++bad; }
    uint32_t n = 0xFFFFFFFFu; ++checked; if (fast_div(n, f) != n / d) ++bad;
  }
  printf("%llu %llu\n", (unsigned long long)checked, (unsigned long long)bad);
  return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"),
                    reason="needs nvcc")
def test_fast_div_matches_integer_division(tmp_path):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    src = tmp_path / "fd.cu"
    src.write_text(SRC)
    exe = tmp_path / "fd"
    subprocess.run([nvcc, "-std=c++17", "-O2", "--expt-relaxed-constexpr", "-I", CSRC, str(src), "-o", str(exe)],
                   check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    checked, bad = map(int, out.stdout.split())
    assert checked > 10_000_000
    assert bad == 0 and out.returncode == 0
