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
static inline unsigned __float_as_uint(float x) { unsigned r; std::memcpy(&r, &x, 4); return r; }
static inline float __uint_as_float(unsigned x) { float r; std::memcpy(&r, &x, 4); return r; }
static inline double __hiloint2double(int hi, int lo) {
  const unsigned long long b = ((unsigned long long)(unsigned)hi << 32) | (unsigned)lo;
  double r; std::memcpy(&r, &b, 8); return r;
}
static inline int __double2hiint(double x) { unsigned long long b; std::memcpy(&b, &x, 8); return (int)(b >> 32); }
static inline int __double2loint(double x) { unsigned long long b; std::memcpy(&b, &x, 8); return (int)(unsigned)b; }
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


GROUP_HARNESS = r"""
#include <cmath>
#include <complex>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <random>
#include <thread>
#include <vector>
#define __device__
#define __forceinline__ inline
static inline long long __double_as_longlong(double x) { long long r; std::memcpy(&r, &x, 8); return r; }
static inline double __longlong_as_double(long long x) { double r; std::memcpy(&r, &x, 8); return r; }
static inline float __int_as_float(int x) { float r; std::memcpy(&r, &x, 4); return r; }
static inline int __float_as_int(float x) { int r; std::memcpy(&r, &x, 4); return r; }
static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
static inline unsigned __float_as_uint(float x) { unsigned r; std::memcpy(&r, &x, 4); return r; }
static inline float __uint_as_float(unsigned x) { float r; std::memcpy(&r, &x, 4); return r; }
static inline double __hiloint2double(int hi, int lo) {
  const unsigned long long b = ((unsigned long long)(unsigned)hi << 32) | (unsigned)lo;
  double r; std::memcpy(&r, &b, 8); return r;
}
static inline int __double2hiint(double x) { unsigned long long b; std::memcpy(&b, &x, 8); return (int)(b >> 32); }
static inline int __double2loint(double x) { unsigned long long b; std::memcpy(&b, &x, 8); return (int)(unsigned)b; }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }

// eight host threads stand for the eight lanes of one group; a shuffle is a
// barrier, a store of each lane's value and a read of the source lane's
struct Barrier {
  std::mutex mu;
  std::condition_variable cv;
  int count = 0, gen = 0;
  void wait() {
    std::unique_lock<std::mutex> lk(mu);
    const int g = gen;
    if (++count == 8) { count = 0; gen++; cv.notify_all(); }
    else cv.wait(lk, [&] { return gen != g; });
  }
};
static Barrier g_bar;
static float g_slot[8];
thread_local unsigned t_lane;
struct Dim { unsigned x; };
#define threadIdx (Dim{t_lane})
static float emu_exchange(float v, int src) {
  g_bar.wait();
  g_slot[t_lane] = v;
  g_bar.wait();
  return g_slot[src];
}
static float __shfl_up_sync(unsigned, float v, int d, int) {
  const int l = (int)(t_lane & 7);
  return emu_exchange(v, l >= d ? l - d : l);
}
static float __shfl_sync(unsigned, float v, int s, int) { return emu_exchange(v, s & 7); }
#include "HEADER"

typedef long double LD;
typedef std::complex<LD> CX;

int main() {
  f2 A2[16], W2[16][16];
  for (int k = 0; k < 16; k++) A2[k] = f2_from_double(k ? 2.0 * k - 1.0 : 0.0, 0);
  for (int n = 0; n < 16; n++)
    for (int m = 0; m < 16; m++)
      W2[n][m] = f2_from_double(n >= m + 2 ? ((double)(n - 1) * (n - 1) - (double)m * m) /
                                                 ((2.0 * n - 1.0) * (2.0 * n - 3.0)) : 0.0, 0);
  std::mt19937_64 rng(11);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  double worst = 0.0;
  int bad_cover = 0;
  const int ps[4] = {6, 10, 12, 15};
  for (int c = 0; c < 48; c++) {
    const int p = ps[c % 4];
    const int k = (int)(rng() % 9) - 3;  // unit 2^k
    double d[3];
    double r;
    do {
      for (double& v : d) v = U(rng) * 8.0;
      r = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    } while (r < 1.5 || r > 13.0);
    for (double& v : d) v = std::ldexp(v, k);  // displacement in box units
    const double s = (c & 1) ? 1.0 : -0.25;
    // device-order evaluation: 8 lanes, inputs in units of 2^k
    std::vector<CX> out(16 * 16, CX(0, 0));
    std::vector<int> hits(16 * 16, 0);
    std::mutex omu;
    std::vector<std::thread> th;
    for (unsigned lane = 0; lane < 8; lane++) {
      th.emplace_back([&, lane] {
        t_lane = lane;
        irregular_group_w2(A2, W2, p, f2_from_double(d[0], -k), f2_from_double(d[1], -k),
                           f2_from_double(d[2], -k), f2_from_double(s, 0),
                           [&](int t, int n, int m, bool v, f2 vr, f2 vi) {
                             if (!v) return;
                             const int e = -k * (n + 1);
                             std::lock_guard<std::mutex> g(omu);
                             out[n * 16 + m] = CX(f2_to_double(vr, e), f2_to_double(vi, e));
                             hits[n * 16 + m]++;
                           });
      });
    }
    for (auto& t : th) t.join();
    // reference: the unscaled two-term recurrence (A = 2n - 1,
    // B = (n + m - 1)(n - m - 1)) in long double, divided by P_n^m
    const LD x = d[0], y = d[1], z = d[2];
    const LD r2 = x * x + y * y + z * z, ir = 1.0L / std::sqrt(r2), Q = ir * ir;
    const CX XY(x * Q, y * Q);
    const LD Z = z * Q;
    CX diag = CX(ir * (LD)s, 0);
    for (int m = 0; m <= p; m++) {
      if (m > 0) diag *= (LD)(2 * m - 1) * XY;
      std::vector<CX> I(p + 1);
      LD colmax = 0;
      for (int n = m; n <= p; n++) {
        if (n == m) I[n] = diag;
        else if (n == m + 1) I[n] = (LD)(2 * n - 1) * Z * I[n - 1];
        else I[n] = (LD)(2 * n - 1) * Z * I[n - 1] - Q * (LD)((n + m - 1) * (n - m - 1)) * I[n - 2];
      }
      std::vector<CX> w(p + 1);
      for (int n = m; n <= p; n++) {
        LD P = 1;
        for (int j = m + 1; j <= n; j++) P *= (LD)(2 * j - 1);
        w[n] = I[n] / P;
        colmax = std::max(colmax, std::abs(w[n]));
      }
      for (int n = m; n <= p; n++) {
        if (hits[n * 16 + m] != 1) bad_cover++;
        const LD err = std::abs(CX(out[n * 16 + m]) - w[n]) / colmax;
        worst = std::max(worst, (double)err);
      }
    }
    for (int n = 0; n < 16; n++)
      for (int m = 0; m < 16; m++)
        if ((m > n || n > p) && hits[n * 16 + m] != 0) bad_cover++;
  }
  std::printf("%.6g %d\n", worst, bad_cover);
  return 0;
}
"""


def test_pair_harmonic_group_matches_long_double_recurrence(tmp_path):
    """irregular_group_w2 run as on the device by 8 emulated lanes (host
    threads, shuffles through a barrier): every (n, m) with m <= n <= p made
    exactly once, and within 1e-12 of its column's largest value against the
    unscaled two-term recurrence in long double divided by P_n^m, over
    random displacements with |x| in [1.5, 13] cell units, units 2^-3..2^5
    and p = 6, 10, 12, 15."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    header = os.path.join(HERE, "..", "paper_2006_16622_gb300", "csrc", "mc_pair_harm.cuh")
    src = tmp_path / "group.cpp"
    src.write_text(GROUP_HARNESS.replace("HEADER", os.path.abspath(header)))
    exe = tmp_path / "group"
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-pthread", "-o", str(exe), str(src), "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=120).stdout.split()
    worst, bad_cover = float(out[0]), int(out[1])
    assert bad_cover == 0
    assert worst <= 1e-12, worst


CONV_HARNESS = r"""
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
static inline unsigned __float_as_uint(float x) { unsigned r; std::memcpy(&r, &x, 4); return r; }
static inline float __uint_as_float(unsigned x) { float r; std::memcpy(&r, &x, 4); return r; }
static inline double __hiloint2double(int hi, int lo) {
  const unsigned long long b = ((unsigned long long)(unsigned)hi << 32) | (unsigned)lo;
  return __longlong_as_double((long long)b);
}
static inline int __double2hiint(double x) { return (int)((unsigned long long)__double_as_longlong(x) >> 32); }
static inline int __double2loint(double x) { return (int)(unsigned)(unsigned long long)__double_as_longlong(x); }
static inline int __clz(unsigned x) { return x ? __builtin_clz(x) : 32; }
static inline float rsqrtf(float x) { return 1.0f / std::sqrt(x); }
#define __shfl_up_sync(m, v, d, w) (v)
#define __shfl_sync(m, v, s, w) (v)
#include "HEADER"

static bool same_bits(float a, float b) { return __float_as_uint(a) == __float_as_uint(b); }
static bool same_bits(double a, double b) { return __double_as_longlong(a) == __double_as_longlong(b); }

int main() {
  std::mt19937_64 g(3);
  int bad_f2d = 0, bad_d2f = 0;
  for (int it = 0; it < 1000000; it++) {
    // float -> double: exact for normal floats, subnormals to signed zero
    const unsigned fb = (unsigned)g();
    const float f = __uint_as_float(fb);
    const unsigned ef = (fb >> 23) & 0xffu;
    if (ef != 0xffu) {
      const double want = ef ? (double)f : std::copysign(0.0, (double)f);
      if (!same_bits(f2d_int(f), want)) bad_f2d++;
    }
    // double -> float rounded to nearest even (the host's IEEE conversion),
    // flushed below 2^-126, +-inf from 2^128; every third input sits exactly
    // half-way between two floats (the ties-to-even case)
    double x = std::ldexp((double)((int64_t)g()) / 9.3e18, (int)(g() % 300) - 150);
    if (it % 3 == 0) {
      const long long b = __double_as_longlong(x);
      x = __longlong_as_double((b & ~0x1fffffffLL) | 0x10000000LL);
    }
    float want = (float)x;
    if (std::fabs(x) < std::ldexp(1.0, -126)) want = std::copysign(0.0f, (float)x);
    if (std::fabs(x) >= std::ldexp(1.0, 128)) want = std::copysign(INFINITY, (float)x);
    if (!same_bits(d2f_int(x), want)) bad_d2f++;
  }
  std::printf("%d %d\n", bad_f2d, bad_d2f);
  return 0;
}
"""


def test_integer_pipe_conversions(tmp_path):
    """f2d_int is exact for every normal float (subnormals become signed
    zero); d2f_int rounds to nearest even, flushes below 2^-126 and saturates to
    +-inf from 2^128, bit for bit against the host's IEEE conversions."""
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "conv.cpp"
    src.write_text(CONV_HARNESS.replace("HEADER", os.path.abspath(HEADER)))
    exe = tmp_path / "conv"
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-o", str(exe), str(src), "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-3000:]
    bad_f2d, bad_d2f = (int(v) for v in subprocess.run([str(exe)], check=True, capture_output=True,
                                                        text=True).stdout.split())
    assert bad_f2d == 0 and bad_d2f == 0, (bad_f2d, bad_d2f)
