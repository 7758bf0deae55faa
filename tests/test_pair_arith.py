"""The pair-of-floats arithmetic of the batched FP64 contributions
(csrc/mc_df64.cuh), compiled for the host with g++ and checked against
long-double references: the integer conversions double <-> pair (with the
power-of-two scale in the exponent), products, a*b - c*d, sums and the
reciprocal square root (an FP32 estimate deliberately 2 ulp off, refined by
the two Newton steps) stay within 2^-45 relative; zero and values below the
float range flush to zero; values with at most 48 significant bits (small
integers, 12345 x 2^980 scaled into range and back) are exact.  No GPU.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_2006_16622_gb300", "csrc", "mc_df64.cuh")

HARNESS = r"""
#include <cmath>
#include <cstdio>
#include <cstring>
#include <cstdint>
#include <random>
#define __device__
#define __forceinline__ inline
static inline long long __double_as_longlong(double x) { long long r; std::memcpy(&r, &x, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; std::memcpy(&r, &x, 8); return r; }
static inline float __int_as_float(int x) { float r; std::memcpy(&r, &x, 4); return r; }
static inline int __float_as_int(float x) { int r; std::memcpy(&r, &x, 4); return r; }
static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x) * (1.0f + 2.4e-7f); }
#define __shfl_up_sync(m, v, d, w) (v)
#define __shfl_sync(m, v, s, w) (v)
#include "HEADER"

static long double val(f2 a) { return (long double)a.h + (long double)a.l; }

int main() {
  std::mt19937_64 g(7);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  double e_conv = 0, e_back = 0, e_mul = 0, e_ms = 0, e_add = 0, e_rs = 0;
  for (int it = 0; it < 200000; it++) {
    const double x = U(g) * std::ldexp(1.0, (int)(g() % 60) - 30);
    const double y = U(g) * std::ldexp(1.0, (int)(g() % 20) - 10);
    const int e = (int)(g() % 21) - 10;
    const f2 a = f2_from_double(x, e);
    const long double ex = (long double)x * std::ldexp(1.0L, e);
    if (x != 0) e_conv = std::fmax(e_conv, (double)(std::fabs(val(a) - ex) / std::fabs(ex)));
    if (x != 0) e_back = std::fmax(e_back, std::fabs(f2_to_double(a, -e) - x) / std::fabs(x));
    const f2 b = f2_from_double(y, 0);
    const long double pm = val(a) * val(b);
    if (x != 0 && y != 0) e_mul = std::fmax(e_mul, (double)(std::fabs(val(f2_mul(a, b)) - pm) / std::fabs(pm)));
    const f2 c = f2_from_double(U(g), 0), d = f2_from_double(U(g), 0);
    const long double ms = val(a) * val(b) - val(c) * val(d);
    const long double sc = std::fabs(val(a) * val(b)) + std::fabs(val(c) * val(d));
    if (sc > 0) e_ms = std::fmax(e_ms, (double)(std::fabs(val(f2_mul_sub(a, b, c, d)) - ms) / sc));
    const long double sm = val(c) + val(d);
    e_add = std::fmax(e_add, (double)(std::fabs(val(f2_add(c, d)) - sm) / (std::fabs(val(c)) + std::fabs(val(d)))));
    const f2 r2 = f2_from_double(std::fabs(y) + 0.01, 0);
    const long double rr = 1.0L / std::sqrt(val(r2));
    e_rs = std::fmax(e_rs, (double)(std::fabs(val(f2_rsqrt(r2)) - rr) / rr));
  }
  const f2 z = f2_from_double(0.0, 5), tiny = f2_from_double(1e-45, 0), three = f2_from_double(-3.0, -2);
  const int special = (z.h == 0.0f && z.l == 0.0f && f2_to_double(z, 9) == 0.0 && tiny.h == 0.0f &&
                       three.h == -0.75f && three.l == 0.0f && f2_to_double(three, 2) == -3.0 &&
                       f2_to_double(f2_from_double(std::ldexp(12345.0, 980), -985), 985) == std::ldexp(12345.0, 980)) ? 1 : 0;
  std::printf("%.6g %.6g %.6g %.6g %.6g %.6g %d\n", e_conv, e_back, e_mul, e_ms, e_add, e_rs, special);
  return 0;
}
"""


def test_pair_arithmetic_error_bounds(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "pair.cpp"
    src.write_text(HARNESS.replace("HEADER", os.path.abspath(HEADER)))
    exe = tmp_path / "pair"
    subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe), str(src), "-lm"],
                   check=True, capture_output=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split()
    e_conv, e_back, e_mul, e_ms, e_add, e_rs = (float(v) for v in out[:6])
    bound = 2.0 ** -45
    assert e_conv <= bound and e_back <= bound, (e_conv, e_back)
    assert e_mul <= bound and e_ms <= bound and e_add <= bound, (e_mul, e_ms, e_add)
    assert e_rs <= bound, e_rs
    assert out[6] == "1"
