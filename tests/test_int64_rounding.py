"""The split kernels' int64-to-double rounding, checked on the host.

The split form assembles every C element as an exact 64-bit integer T and a
power of two, and rounds T * 2^e2 to a double with integer operations only
(`scaled_i64_fast`, exact general path `scaled_i64_to_double`, both in
csrc/split.cu).  This test compiles those two device functions as host C++
(with host versions of the three CUDA intrinsics they call) and compares
them with `long double` arithmetic, whose 64-bit significand holds T exactly,
so that casting to double is one round-to-nearest-even: the IEEE result.
Random T of every magnitude up to 2^62, exponents over the whole normal range
and past it, halfway cases and powers of two; where the fast path reports
that it stays in range its bits must equal both the general path's and the
long double result's.
"""

from __future__ import annotations

import pathlib
import shutil
import subprocess

import pytest

SRC = pathlib.Path(__file__).resolve().parents[1] / "paper_2011_11762_gb300" / "csrc" / "split.cu"

SHIMS = r"""
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <random>
#define __device__
#define __forceinline__ inline
static inline int __clzll(long long x) { return x == 0 ? 64 : __builtin_clzll((unsigned long long)x); }
static inline int __clz(int x) { return x == 0 ? 32 : __builtin_clz((unsigned)x); }
static inline uint32_t __funnelshift_l(uint32_t lo, uint32_t hi, int sh) {
  sh &= 31; unsigned long long w = ((unsigned long long)hi << 32) | lo; return (uint32_t)((w << sh) >> 32); }
static inline uint32_t __funnelshift_r(uint32_t lo, uint32_t hi, int sh) {
  sh &= 31; unsigned long long w = ((unsigned long long)hi << 32) | lo; return (uint32_t)(w >> sh); }
static inline double __longlong_as_double(long long b) { double d; std::memcpy(&d, &b, 8); return d; }
"""

MAIN = r"""
static int check(long long v, int e2, long long *fast_used) {
  bool ok;
  const double a = scaled_i64_fast(v, e2, &ok);
  const double r = scaled_i64_to_double(v, e2);
  const double l = (double)std::ldexp((long double)v, e2);
  if (std::memcmp(&r, &l, 8) && std::isnormal(l)) return 1;   // general path vs IEEE
  if (!ok) return 0;
  ++*fast_used;
  if (!std::isnormal(a) && a != 0.0) return 2;
  if (std::memcmp(&a, &r, 8) || std::memcmp(&a, &l, 8)) return 3;
  return 0;
}
int main() {
  std::mt19937_64 g(20111762);
  long long fast = 0, bad = 0, n = 0;
  for (int it = 0; it < 2000000; ++it) {
    const int bits = (int)(g() % 63);
    long long v = bits ? (long long)(g() >> (63 - bits)) : (long long)(g() % 3);
    if (it % 5 == 0) v = (long long)(1ULL << (g() % 62)) + (long long)(g() % 5) - 2;  // near powers
    if (it % 7 == 0) v = (long long)(((g() >> 12) | 1ULL) << 10) | 0x400;        // exact halves
    if (g() & 1) v = -v;
    int e2 = (int)(g() % 2300) - 1150;
    if (it % 3) e2 = (int)(g() % 240) - 120;
    const int c = check(v, e2, &fast);
    ++n;
    if (c) { if (bad < 5) std::printf("case %d: v=%lld e2=%d\n", c, v, e2); ++bad; }
  }
  std::printf("n=%lld fast=%lld bad=%lld\n", n, fast, bad);
  return bad != 0 || fast < n / 2;
}
"""


def _functions() -> str:
    src = SRC.read_text()
    a = src.index("__device__ inline double scaled_i64_to_double")
    b = src.index("// ------------------------------------------------------------ pre-kernels --")
    return src[a:b]


def test_int64_rounding_matches_ieee(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    cpp = tmp_path / "round.cpp"
    cpp.write_text(SHIMS + _functions() + MAIN)
    exe = tmp_path / "round"
    subprocess.run([gxx, "-O2", "-std=c++17", str(cpp), "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stdout + r.stderr
