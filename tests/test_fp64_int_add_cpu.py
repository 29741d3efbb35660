"""The integer-pipe binary64 addition (fp64_int.cuh), compiled for the host
and checked against the host's IEEE 754 adder (round to nearest even, no
flush of subnormals) on random operand pairs of every class: the same
source the FP64 sweep kernels use for part of the star / heat neighbour
sum.  NaN results only have to be NaNs."""
import os
import shutil
import subprocess

import pytest

HDR = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                   "paper_1207_1746_b300", "csrc", "fp64_int.cuh")

HARNESS = r"""
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#include "fp64_int.cuh"
static uint64_t bits(double x) { uint64_t u; std::memcpy(&u, &x, 8); return u; }
static double dbl(uint64_t u) { double x; std::memcpy(&x, &u, 8); return x; }
static bool is_nan(uint64_t u) { return ((u >> 52) & 0x7ff) == 0x7ff && (u & 0xfffffffffffffull); }
int main(int argc, char **argv) {
  const long long n = atoll(argv[1]);
  std::mt19937_64 g(20240601);
  const uint64_t sp[] = {0ull, 1ull << 63, 0x7ffull << 52, 0xfffull << 52, 0x7ff8ull << 48, 0x7ff0000000000001ull,
                         1ull, 0x800fffffffffffffull, 0x7fefffffffffffffull, 0xffefffffffffffffull, 0x0010000000000000ull};
  long long bad = 0;
  for (long long i = 0; i < n; ++i) {
    uint64_t a = g(), b = g();
    switch (i % 9) {
      case 0: break;                                                          // any bits
      case 1: b = (a & 0xfff0000000000000ull) | (b & 0x000fffffffffffffull); break;  // same exponent and sign
      case 2: b = ((a ^ (1ull << 63)) & 0xfff0000000000000ull) | (b & 0x000fffffffffffffull); break;  // cancellation
      case 3: { uint64_t ea = (a >> 52) & 0x7ff, k = b % 64, eb = ea > k ? ea - k : 0;  // alignment shifts
                b = (b & 0x800fffffffffffffull) | (eb << 52); } break;
      case 4: b = (a ^ (1ull << 63)) + (g() % 5) - 2; break;                  // near-exact cancellation
      case 5: a &= 0x800fffffffffffffull; a |= (g() % 3) << 52;              // subnormal and tiny
              b &= 0x800fffffffffffffull; b |= (g() % 3) << 52; break;
      case 6: a = (a & 0x800fffffffffffffull) | ((2044 + g() % 4) << 52);    // near overflow, inf, NaN
              b = (b & 0x800fffffffffffffull) | ((2040 + g() % 8) << 52); break;
      case 7: a = sp[g() % 11]; if (g() & 1) b = sp[g() % 11]; break;        // special values
      default: { uint64_t ea = 1023 + g() % 64, k = 52 + g() % 5;            // ties at the rounding boundary
                 a = (a & 0x800fffffffffffffull) | (ea << 52);
                 b = (b & 0x8000000000000000ull) | ((ea - k) << 52) | ((g() & 1) ? 0 : (b & 0xfffffffffffffull)); }
    }
    for (int o = 0; o < 2; ++o) {
      const uint64_t x = o ? b : a, y = o ? a : b;
      const uint64_t r = gscl::fp64_add_int_bits(x, y), h = bits(dbl(x) + dbl(y));
      if (r != h && !(is_nan(r) && is_nan(h))) {
        if (bad < 5) std::printf("%016llx + %016llx: %016llx, IEEE %016llx\n", (unsigned long long)x,
                                 (unsigned long long)y, (unsigned long long)r, (unsigned long long)h);
        ++bad;
      }
    }
  }
  std::printf("mismatches %lld\n", bad);
  return bad != 0;
}
"""


@pytest.mark.skipif(shutil.which("g++") is None, reason="needs g++")
def test_integer_add_matches_ieee_on_the_host(tmp_path):
    src = tmp_path / "harness.cpp"
    src.write_text(HARNESS)
    exe = tmp_path / "harness"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-D__host__=", "-D__device__=",
                           "-D__forceinline__=inline", "-I", os.path.dirname(HDR), "-o", str(exe), str(src)])
    out = subprocess.run([str(exe), "3000000"], capture_output=True, text=True, timeout=300)
    assert out.returncode == 0, out.stdout[-2000:]
    assert "mismatches 0" in out.stdout
