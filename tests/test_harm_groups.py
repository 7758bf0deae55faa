"""The GPU path's solid-harmonic groups (csrc/mc_harm.cuh) on the CPU.

The device code is compiled for the host with g++ and run by 8 emulated
lanes (host threads; every warp shuffle goes through a barrier), exactly as
one group of a warp runs it.  Each set is checked against the closed forms
of the scaled harmonics, written with the associated Legendre functions of
the C++ library (no Condon-Shortley phase, as the method reads Y_n^m):

    regular    Rt_n^m(x) = r^n P_n^m(cos t) e^{i m phi} / (n + m)!
    irregular  It_n^m(x) = (n - m)! P_n^m(cos t) e^{i m phi} / r^(n + 1)
    column-scaled irregular  It_n^m / prod_{k=m+1..n} (2k - 1)

for the per-coefficient sets (regular_group, irregular_group, the factor
forms regular_group_s / irregular_group_s, irregular_group_w) and the column
factorisation (regular_group_q, irregular_group_q: diagonal value times the
real polynomial), in FP64 (within 1e-13 of each column's largest value) and
FP32 (within 1e-4), for p = 4, 8, 12, 15.  Every (n, m), m <= n <= p, must
come out exactly once.  No GPU.
"""
import os
import shutil
import subprocess

import pytest

HERE = os.path.dirname(os.path.abspath(__file__))
HEADER = os.path.join(HERE, "..", "paper_2006_16622_gb300", "csrc", "mc_harm.cuh")

HARNESS = r"""
#include <cmath>
#include <complex>
#include <condition_variable>
#include <cstdio>
#include <cstring>
#include <functional>
#include <mutex>
#include <random>
#include <thread>
#include <vector>
#define __device__
#define __forceinline__ inline
#define MC_PMAX 15
#define MC_MAXLEV 8
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
static inline double rsqrt(double x) { return 1.0 / std::sqrt(x); }

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
static double g_slot[8];
thread_local unsigned t_lane = 0;
struct Dim { unsigned x; };
#define threadIdx (Dim{t_lane})
#define blockDim (Dim{1u})
template <typename T> static T emu_exchange(T v, int src) {
  g_bar.wait();
  g_slot[t_lane] = (double)v;
  g_bar.wait();
  return (T)g_slot[src];
}
template <typename T> static T __shfl_up_sync(unsigned, T v, int d, int) {
  const int l = (int)(t_lane & 7);
  return emu_exchange(v, l >= d ? l - d : l);
}
template <typename T> static T __shfl_sync(unsigned, T v, int s, int) { return emu_exchange(v, s & 7); }
template <typename T> static T __shfl_xor_sync(unsigned, T v, int o, int = 32) {
  return emu_exchange(v, (int)((t_lane ^ o) & 7));
}
#include "HEADER"

typedef std::complex<double> CX;

static double fact(int n) { double f = 1; for (int k = 2; k <= n; k++) f *= k; return f; }

// closed forms (kind 0 regular, 1 irregular, 2 column-scaled irregular)
static CX closed(int kind, int n, int m, double x, double y, double z) {
  const double r = std::sqrt(x * x + y * y + z * z), ct = z / r, phi = std::atan2(y, x);
  const double P = std::assoc_legendre(n, m, ct);
  const CX e = std::polar(1.0, m * phi);
  if (kind == 0) return std::pow(r, n) * P * e / fact(n + m);
  CX v = fact(n - m) * P * e / std::pow(r, n + 1);
  if (kind == 2) { double pp = 1; for (int k = m + 1; k <= n; k++) pp *= 2 * k - 1; v /= pp; }
  return v;
}

template <typename T>
static void run_case(int form, int p, const double d[3], double s, std::vector<CX>& out, std::vector<int>& hits,
                     const HarmTabs<T>* tabs, const T (*W)[16]) {
  std::mutex omu;
  std::vector<std::thread> th;
  for (unsigned lane = 0; lane < 8; lane++) {
    th.emplace_back([&, lane] {
      t_lane = lane;
      const T x = (T)d[0], y = (T)d[1], z = (T)d[2];
      auto put = [&](int n, int m, bool v, double re, double im) {
        if (!v) return;
        std::lock_guard<std::mutex> g(omu);
        out[n * 16 + m] = CX(re, im);
        hits[n * 16 + m]++;
      };
      auto use = [&](int, int n, int m, bool v, T vr, T vi) { put(n, m, v, (double)vr, (double)vi); };
      if (form == 0) regular_group<T>(tabs, p, x, y, z, use);
      else if (form == 1) irregular_group<T>(tabs, p, x, y, z, use);
      else if (form == 2) regular_group_s<T>(tabs, p, x, y, z, (T)s, use);
      else if (form == 3) irregular_group_s<T>(tabs, p, x, y, z, (T)s, use);
      else if (form == 4) irregular_group_w<T>(tabs, W, p, x, y, z, (T)s, use);
      else {
        T d1r, d1i, d2r, d2i;
        auto useq = [&](int, int n, int m, bool v, bool first, T q) {
          const double dr = (double)(first ? d1r : d2r), di = (double)(first ? d1i : d2i);
          put(n, m, v, dr * (double)q, di * (double)q);
        };
        if (form == 5) regular_group_q<T>(tabs, p, x, y, z, &d1r, &d1i, &d2r, &d2i, useq);
        else irregular_group_q<T>(tabs, p, x, y, z, &d1r, &d1i, &d2r, &d2i, useq);
      }
    });
  }
  for (auto& t : th) t.join();
}

template <typename T>
static void check(const char* name, double& worst_out, int& bad_cover) {
  static HarmTabs<T> tabs;
  static T W[MC_PMAX + 1][16];
  static double P[(MC_PMAX + 1) * (MC_PMAX + 1)];
  t_lane = 0;
  harm_tabs_init<T>(&tabs);
  irregular_w_tabs<T>(W, P);
  std::mt19937_64 rng(5);
  std::uniform_real_distribution<double> U(-1.0, 1.0);
  const int ps[4] = {4, 8, 12, 15};
  double worst = 0;
  for (int form = 0; form < 7; form++) {
    for (int c = 0; c < 12; c++) {
      const int p = ps[c % 4];
      double d[3];
      for (double& v : d) v = U(rng) * (form == 0 || form == 2 || form == 5 ? 0.8 : 3.0);
      if (form != 0 && form != 2 && form != 5) d[c % 3] += (c & 1) ? 2.0 : -2.0;
      const double s = (form == 2 || form == 3 || form == 4) ? ((c & 1) ? -0.5 : 1.5) : 1.0;
      std::vector<CX> out(256, CX(0, 0));
      std::vector<int> hits(256, 0);
      run_case<T>(form, p, d, s, out, hits, &tabs, W);
      const int kind = (form == 0 || form == 2 || form == 5) ? 0 : (form == 4 ? 2 : 1);
      for (int m = 0; m <= p; m++) {
        double colmax = 0;
        for (int n = m; n <= p; n++) colmax = std::max(colmax, std::abs(s * closed(kind, n, m, d[0], d[1], d[2])));
        for (int n = m; n <= p; n++) {
          if (hits[n * 16 + m] != 1) bad_cover++;
          const CX ref = s * closed(kind, n, m, d[0], d[1], d[2]);
          worst = std::max(worst, std::abs(out[n * 16 + m] - ref) / colmax);
        }
      }
      for (int n = 0; n < 16; n++)
        for (int m = 0; m < 16; m++)
          if ((m > n || n > p) && hits[n * 16 + m] != 0) bad_cover++;
    }
  }
  std::printf("%s %.6g\n", name, worst);
  worst_out = worst;
}

int main() {
  double w64 = 0, w32 = 0;
  int bad = 0;
  check<double>("fp64", w64, bad);
  check<float>("fp32", w32, bad);
  std::printf("RESULT %.6g %.6g %d\n", w64, w32, bad);
  return 0;
}
"""


def test_harmonic_groups_match_closed_forms(tmp_path):
    gxx = shutil.which("g++")
    if gxx is None:
        pytest.skip("no host C++ compiler")
    src = tmp_path / "harm.cpp"
    src.write_text(HARNESS.replace("HEADER", os.path.abspath(HEADER)))
    exe = tmp_path / "harm"
    r = subprocess.run([gxx, "-O2", "-std=c++17", "-ffp-contract=off", "-pthread", "-o", str(exe), str(src), "-lm"],
                       capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-4000:]
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True, timeout=300).stdout
    res = [ln for ln in out.splitlines() if ln.startswith("RESULT")][0].split()
    w64, w32, bad = float(res[1]), float(res[2]), int(res[3])
    assert bad == 0
    assert w64 <= 1e-13, w64
    assert w32 <= 1e-4, w32
