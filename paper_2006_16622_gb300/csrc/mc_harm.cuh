// Solid harmonics by recurrence: the scaled regular and irregular sets of
// the expansions, column by column (harm_columns) or one set per group of 8
// lanes (harm_group and its consumers), the column-scaled irregular form and
// the column factorisation, and the tables they read.  Needs MC_PMAX and
// MC_MAXLEV from its includer (mc_dev.cuh), CUDA's thread index, warp
// shuffles and rsqrt; nothing else, so it also compiles for host tests.
#pragma once
#include "mc_df64.cuh"
#include "mc_pair_harm.cuh"

#if !defined(MC_PMAX) || !defined(MC_MAXLEV)
#error "mc_harm.cuh needs MC_PMAX and MC_MAXLEV"
#endif

// ------------------------------------------------------ recurrence tables
template <typename T>
struct HarmTabs {
  T rA[MC_PMAX + 1][16], rB[MC_PMAX + 1][16];  // regular
  T iA[MC_PMAX + 1][16], iB[MC_PMAX + 1][16];  // irregular
};

template <typename T>
__device__ void harm_tabs_init(HarmTabs<T>* t) {
  for (int k = threadIdx.x; k < (MC_PMAX + 1) * 16; k += blockDim.x) {
    int n = k / 16, m = k % 16;
    double ra = 0, rb = 0, ia = 0, ib = 0;
    if (n >= 1) {
      if (n <= m) {
        ra = 1.0 / (2.0 * n);
        ia = 2.0 * n - 1.0;
      } else {
        double den = (double)(n + m) * (double)(n - m);
        ra = (2.0 * n - 1.0) / den;
        rb = 1.0 / den;
        ia = 2.0 * n - 1.0;
        ib = (double)(n + m - 1) * (double)(n - m - 1);
      }
    }
    t->rA[n][m] = (T)ra;
    t->rB[n][m] = (T)rb;
    t->iA[n][m] = (T)ia;
    t->iB[n][m] = (T)ib;
  }
}

// Column m of the scaled harmonics for n = 0..p; use(n, re, im) is called
// for every n (values are meaningful for n >= m).
template <typename T, typename F>
__device__ __forceinline__ void harm_columns(const T (*A)[16], const T (*B)[16], int p, int m,
                                             T X, T Y, T Z, T Q, T start, F&& use) {
  T p1r = start, p1i = T(0), p2r = T(0), p2i = T(0);
  use(0, p1r, p1i);
#pragma unroll
  for (int n = 1; n <= MC_PMAX; n++) {
    if (n <= p) {
      const bool diag = n <= m;
      const T ca = A[n][m], cb = B[n][m];
      const T ar = (diag ? X : Z) * ca;
      const T ai = diag ? Y * ca : T(0);
      const T b = -Q * cb;
      const T cr = ar * p1r - ai * p1i + b * p2r;
      const T ci = ar * p1i + ai * p1r + b * p2i;
      p2r = diag ? T(0) : p1r;
      p2i = diag ? T(0) : p1i;
      p1r = cr;
      p1i = ci;
      use(n, cr, ci);
    }
  }
}

// regular harmonics of displacement (x, y, z)
template <typename T, typename F>
__device__ __forceinline__ void regular_columns(const HarmTabs<T>* t, int p, int m, T x, T y, T z,
                                                F&& use) {
  T r2 = x * x + y * y + z * z;
  harm_columns<T>(t->rA, t->rB, p, m, x, y, z, r2, T(1), use);
}

__device__ __forceinline__ double mc_rsqrt(double v) { return rsqrt(v); }
__device__ __forceinline__ float mc_rsqrt(float v) { return rsqrtf(v); }

// irregular harmonics of displacement (x, y, z) (source minus centre)
template <typename T, typename F>
__device__ __forceinline__ void irregular_columns(const HarmTabs<T>* t, int p, int m, T x, T y,
                                                  T z, F&& use) {
  T r2 = x * x + y * y + z * z;
  T ir = mc_rsqrt(r2);
  T ir2 = ir * ir;
  harm_columns<T>(t->iA, t->iB, p, m, x * ir2, y * ir2, z * ir2, ir2, ir, use);
}

// ----------------------------------------------------- grouped evaluation
// One harmonic set per group of 8 lanes (4 sets per warp).  Lane g of a
// group owns the columns m1 = g and m2 = p - g (when m2 > m1), so every lane
// makes p + 2 values in p + 2 identical steps (the triangle n >= m is split
// evenly).  The diagonal values X_m^m = prod_{k<=m} f_k (f_0 = start, f_k =
// A_k (x + i y)) come from a log-depth product scan over the group; the
// columns then run the two-term recurrence with 6 flops per step.
// use(t, n, m, re, im) is called for t = 0..p+1 (t is a compile-time
// constant after unrolling); the value is valid when `valid` is passed true.
template <typename T>
__device__ __forceinline__ void cmul(T ar, T ai, T br, T bi, T* cr, T* ci) {
  *cr = ar * br - ai * bi;
  *ci = ar * bi + ai * br;
}

template <typename T, typename F, bool kUnroll = true, bool kW = false>
__device__ __forceinline__ void harm_group(const T (*A)[16], const T (*B)[16], int p, T X, T Y,
                                           T Z, T Q, T start, F&& use) {
  const int g = threadIdx.x & 7;
  // factors f_{2g}, f_{2g+1} (the diagonal entries of the tables are A_k)
  const int k0 = 2 * g, k1 = 2 * g + 1;
  const T a0 = A[k0][k0], a1 = A[k1][k1];
  T f0r = (k0 == 0) ? start : X * a0, f0i = (k0 == 0) ? T(0) : Y * a0;
  const T f1r = X * a1, f1i = Y * a1;
  T Pr, Pi;
  cmul(f0r, f0i, f1r, f1i, &Pr, &Pi);
  // inclusive product scan of P over the 8 lanes of the group
  T Ir = Pr, Ii = Pi;
#pragma unroll
  for (int d = 1; d < 8; d <<= 1) {
    const T ur = __shfl_up_sync(0xffffffffu, Ir, d, 8), ui = __shfl_up_sync(0xffffffffu, Ii, d, 8);
    if (g >= d) {
      T nr, ni;
      cmul(ur, ui, Ir, Ii, &nr, &ni);
      Ir = nr;
      Ii = ni;
    }
  }
  T Er = __shfl_up_sync(0xffffffffu, Ir, 1, 8), Ei = __shfl_up_sync(0xffffffffu, Ii, 1, 8);
  if (g == 0) {
    Er = T(1);
    Ei = T(0);
  }
  T D0r, D0i;  // X_{2g}^{2g}
  cmul(Er, Ei, f0r, f0i, &D0r, &D0i);
  const T D1r = Ir, D1i = Ii;  // X_{2g+1}^{2g+1}
  const int m1 = g, m2 = p - g;
  const bool active = m1 <= m2;
  const bool two = m2 > m1;
  // fetch X_m^m for m = m1, m2 from lane m/2 of the group
  const T e1r = __shfl_sync(0xffffffffu, D0r, m1 >> 1, 8), e1i = __shfl_sync(0xffffffffu, D0i, m1 >> 1, 8);
  const T o1r = __shfl_sync(0xffffffffu, D1r, m1 >> 1, 8), o1i = __shfl_sync(0xffffffffu, D1i, m1 >> 1, 8);
  const int m2c = (m2 >= 0 && m2 <= 15) ? m2 : 0;
  const T e2r = __shfl_sync(0xffffffffu, D0r, m2c >> 1, 8), e2i = __shfl_sync(0xffffffffu, D0i, m2c >> 1, 8);
  const T o2r = __shfl_sync(0xffffffffu, D1r, m2c >> 1, 8), o2i = __shfl_sync(0xffffffffu, D1i, m2c >> 1, 8);
  const T d1r = (m1 & 1) ? o1r : e1r, d1i = (m1 & 1) ? o1i : e1i;
  const T d2r = (m2c & 1) ? o2r : e2r, d2i = (m2c & 1) ? o2i : e2i;
  const int len1 = p - m1 + 1;
  T p1r = T(0), p1i = T(0), p2r = T(0), p2i = T(0);
  auto step = [&](int t) {
    const bool c1 = t < len1;
    const int m = c1 ? m1 : m2c;
    const int n = c1 ? (m1 + t) : (m2c + t - len1);
    const bool valid = active && (c1 || two) && n <= p;
    const bool st = (n == m);
    const int nn = n > 15 ? 15 : n;
    const T a = kW ? Z : Z * A[nn][m], b = Q * B[nn][m];
    T vr = a * p1r - b * p2r, vi = a * p1i - b * p2i;
    const T sr = c1 ? d1r : d2r, si = c1 ? d1i : d2i;
    vr = st ? sr : vr;
    vi = st ? si : vi;
    p2r = st ? T(0) : p1r;
    p2i = st ? T(0) : p1i;
    p1r = vr;
    p1i = vi;
    use(t, n, m, valid, vr, vi);
  };
  if constexpr (kUnroll) {
    // consumers that keep per-step values in register arrays need t constant
#pragma unroll
    for (int t = 0; t <= MC_PMAX + 1; t++)
      if (t <= p + 1) step(t);
  } else {
    // a rolled loop: much less code where every step writes memory
#pragma unroll 1
    for (int t = 0; t <= p + 1; t++) step(t);
  }
}

// (n, m) of step t of this lane in harm_group, for preloading coefficients
__device__ __forceinline__ void group_nm(int p, int t, int* n, int* m, bool* valid) {
  const int g = threadIdx.x & 7;
  const int m1 = g, m2 = p - g;
  const int m2c = (m2 >= 0 && m2 <= 15) ? m2 : 0;
  const int len1 = p - m1 + 1;
  const bool c1 = t < len1;
  *m = c1 ? m1 : m2c;
  *n = c1 ? (m1 + t) : (m2c + t - len1);
  *valid = (m1 <= m2) && (c1 || m2 > m1) && *n <= p;
}

template <typename T>
__device__ __forceinline__ T group_sum(T v) {
#pragma unroll
  for (int o = 4; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

template <typename T, typename F>
__device__ __forceinline__ void regular_group(const HarmTabs<T>* t, int p, T x, T y, T z, F&& use) {
  const T r2 = x * x + y * y + z * z;
  harm_group<T>(t->rA, t->rB, p, x, y, z, r2, T(1), use);
}

template <typename T, typename F>
__device__ __forceinline__ void irregular_group(const HarmTabs<T>* t, int p, T x, T y, T z, F&& use) {
  const T r2 = x * x + y * y + z * z;
  const T ir = mc_rsqrt(r2);
  const T ir2 = ir * ir;
  harm_group<T>(t->iA, t->iB, p, x * ir2, y * ir2, z * ir2, ir2, ir, use);
}

// The same sets times a factor s (the recurrence is linear in its start
// value, so the factor costs one multiply instead of one per coefficient),
// with a rolled step loop (use() sees a run-time t).
template <typename T, typename F>
__device__ __forceinline__ void regular_group_s(const HarmTabs<T>* t, int p, T x, T y, T z, T s,
                                                F&& use) {
  const T r2 = x * x + y * y + z * z;
  harm_group<T, F, false>(t->rA, t->rB, p, x, y, z, r2, s, static_cast<F&&>(use));
}

template <typename T, typename F>
__device__ __forceinline__ void irregular_group_s(const HarmTabs<T>* t, int p, T x, T y, T z, T s,
                                                  F&& use) {
  const T r2 = x * x + y * y + z * z;
  const T ir = mc_rsqrt(r2);
  const T ir2 = ir * ir;
  harm_group<T, F, false>(t->iA, t->iB, p, x * ir2, y * ir2, z * ir2, ir2, ir * s, static_cast<F&&>(use));
}

// Column-scaled irregular sets: below the diagonal, value (n, m) divided by
// P_n^m = prod_{k=m+1..n} (2k - 1), so the recurrence loses the factor
// (2n - 1) of its first term (5 instead of 6 flops per step) and its second
// term takes W[n][m] = ((n-1)^2 - m^2) / ((2n-1)(2n-3)) (irregular_w_tabs).
// The consumer multiplies by P_n^m (irregular_p), e.g. in the fused
// multiply-add that adds the value into an expansion.
template <typename T, typename F>
__device__ __forceinline__ void irregular_group_w(const HarmTabs<T>* t, const T (*W)[16], int p, T x,
                                                  T y, T z, T s, F&& use) {
  const T r2 = x * x + y * y + z * z;
  const T ir = mc_rsqrt(r2);
  const T ir2 = ir * ir;
  harm_group<T, F, false, true>(t->iA, W, p, x * ir2, y * ir2, z * ir2, ir2, ir * s,
                                static_cast<F&&>(use));
}

// The same column-scaled sets with the step loop unrolled: for consumers
// that keep the values in register arrays indexed by the step.
template <typename T, typename F>
__device__ __forceinline__ void irregular_group_wu(const HarmTabs<T>* t, const T (*W)[16], int p, T x,
                                                   T y, T z, T s, F&& use) {
  const T r2 = x * x + y * y + z * z;
  const T ir = mc_rsqrt(r2);
  const T ir2 = ir * ir;
  harm_group<T, F, true, true>(t->iA, W, p, x * ir2, y * ir2, z * ir2, ir2, ir * s,
                               static_cast<F&&>(use));
}

__device__ __forceinline__ f2 f2_of(double v) { return f2_from_double(v, 0); }

// Tables of irregular_group_w2 and of the apply that takes its pairs (read
// after irregular_w_tabs has filled W and P): W and P_n^m as pairs, the
// diagonal factors A_k = 2k - 1, n of every real-layout index, and per level
// l the unit exponent k_l with 2^k_l <= lev_w[l] < 2^(k_l + 1).
template <typename T>
__device__ void pair_w_tabs(const T (*W)[16], const double* P, f2 (*W2)[16], f2* A2, f2* P2,
                            unsigned char* nn, int* kl, const double* lev_w, int L) {
  for (int k = threadIdx.x; k < (MC_PMAX + 1) * 16; k += blockDim.x) W2[k / 16][k % 16] = f2_of((double)W[k / 16][k % 16]);
  for (int k = threadIdx.x; k < (MC_PMAX + 1) * (MC_PMAX + 1); k += blockDim.x) {
    P2[k] = f2_of(P[k]);
    int n = 0;
    while ((n + 1) * (n + 1) <= k) n++;
    nn[k] = (unsigned char)n;
  }
  if (threadIdx.x < 16) A2[threadIdx.x] = f2_of(threadIdx.x ? 2.0 * threadIdx.x - 1.0 : 0.0);
  if (threadIdx.x < MC_MAXLEV + 2) {
    const int l = threadIdx.x;
    kl[l] = (l >= 1 && l <= L) ? (int)((__double_as_longlong(lev_w[l]) >> 52) & 0x7ff) - 1023 : 0;
  }
}

template <typename T>
__device__ void irregular_w_tabs(T (*W)[16], double* P) {
  for (int k = threadIdx.x; k < (MC_PMAX + 1) * 16; k += blockDim.x) {
    const int n = k / 16, m = k % 16;
    double w = 0.0;
    if (n >= m + 2) w = ((double)(n - 1) * (n - 1) - (double)m * m) / ((2.0 * n - 1.0) * (2.0 * n - 3.0));
    W[n][m] = (T)w;
  }
  // P_n^m at the real layout index of (n, m) (both parts)
  for (int k = threadIdx.x; k < (MC_PMAX + 1) * (MC_PMAX + 1); k += blockDim.x) {
    int n = 0;
    while ((n + 1) * (n + 1) <= k) n++;
    const int m = (k == n * n) ? 0 : (k - n * n + 1) / 2;
    double pr = 1.0;
    for (int j = m + 1; j <= n; j++) pr *= 2.0 * j - 1.0;
    P[k] = pr;
  }
}

// Column factorisation: every scaled harmonic of column m is the diagonal
// value X_m^m times a real polynomial q_n^m(z, r^2) with q_m^m = 1 and the
// same two-term recurrence, so a consumer that contracts a whole column
// with coefficients (the evaluation of Eq. 2) runs the recurrence on reals
// (4 flops per step instead of 6) and applies X_m^m once per column.
// use(t, n, m, valid, first_column, q); the diagonal values of this lane's
// two columns are returned in (d1r, d1i), (d2r, d2i).
template <typename T, typename F>
__device__ __forceinline__ void harm_group_q(const T (*A)[16], const T (*B)[16], int p, T X, T Y,
                                             T Z, T Q, T start, T* d1r_out, T* d1i_out, T* d2r_out,
                                             T* d2i_out, F&& use) {
  const int g = threadIdx.x & 7;
  const int k0 = 2 * g, k1 = 2 * g + 1;
  const T a0 = A[k0][k0], a1 = A[k1][k1];
  T f0r = (k0 == 0) ? start : X * a0, f0i = (k0 == 0) ? T(0) : Y * a0;
  const T f1r = X * a1, f1i = Y * a1;
  T Pr, Pi;
  cmul(f0r, f0i, f1r, f1i, &Pr, &Pi);
  T Ir = Pr, Ii = Pi;
#pragma unroll
  for (int d = 1; d < 8; d <<= 1) {
    const T ur = __shfl_up_sync(0xffffffffu, Ir, d, 8), ui = __shfl_up_sync(0xffffffffu, Ii, d, 8);
    if (g >= d) {
      T nr, ni;
      cmul(ur, ui, Ir, Ii, &nr, &ni);
      Ir = nr;
      Ii = ni;
    }
  }
  T Er = __shfl_up_sync(0xffffffffu, Ir, 1, 8), Ei = __shfl_up_sync(0xffffffffu, Ii, 1, 8);
  if (g == 0) {
    Er = T(1);
    Ei = T(0);
  }
  T D0r, D0i;
  cmul(Er, Ei, f0r, f0i, &D0r, &D0i);
  const T D1r = Ir, D1i = Ii;
  const int m1 = g, m2 = p - g;
  const bool active = m1 <= m2;
  const bool two = m2 > m1;
  const T e1r = __shfl_sync(0xffffffffu, D0r, m1 >> 1, 8), e1i = __shfl_sync(0xffffffffu, D0i, m1 >> 1, 8);
  const T o1r = __shfl_sync(0xffffffffu, D1r, m1 >> 1, 8), o1i = __shfl_sync(0xffffffffu, D1i, m1 >> 1, 8);
  const int m2c = (m2 >= 0 && m2 <= 15) ? m2 : 0;
  const T e2r = __shfl_sync(0xffffffffu, D0r, m2c >> 1, 8), e2i = __shfl_sync(0xffffffffu, D0i, m2c >> 1, 8);
  const T o2r = __shfl_sync(0xffffffffu, D1r, m2c >> 1, 8), o2i = __shfl_sync(0xffffffffu, D1i, m2c >> 1, 8);
  *d1r_out = (m1 & 1) ? o1r : e1r;
  *d1i_out = (m1 & 1) ? o1i : e1i;
  *d2r_out = (m2c & 1) ? o2r : e2r;
  *d2i_out = (m2c & 1) ? o2i : e2i;
  const int len1 = p - m1 + 1;
  T q1 = T(0), q2 = T(0);
#pragma unroll
  for (int t = 0; t <= MC_PMAX + 1; t++) {
    if (t <= p + 1) {
      const bool c1 = t < len1;
      const int m = c1 ? m1 : m2c;
      const int n = c1 ? (m1 + t) : (m2c + t - len1);
      const bool valid = active && (c1 || two) && n <= p;
      const bool st = (n == m);
      const int nn = n > 15 ? 15 : n;
      const T a = Z * A[nn][m], b = Q * B[nn][m];
      T v = a * q1 - b * q2;
      v = st ? T(1) : v;
      q2 = st ? T(0) : q1;
      q1 = v;
      use(t, n, m, valid, c1, v);
    }
  }
}

template <typename T, typename F>
__device__ __forceinline__ void regular_group_q(const HarmTabs<T>* t, int p, T x, T y, T z, T* d1r,
                                                T* d1i, T* d2r, T* d2i, F&& use) {
  const T r2 = x * x + y * y + z * z;
  harm_group_q<T>(t->rA, t->rB, p, x, y, z, r2, T(1), d1r, d1i, d2r, d2i, use);
}

// irregular sets in the column-factorised form (unrolled: consumers keep
// per-step values in register arrays)
template <typename T, typename F>
__device__ __forceinline__ void irregular_group_q(const HarmTabs<T>* t, int p, T x, T y, T z, T* d1r,
                                                  T* d1i, T* d2r, T* d2i, F&& use) {
  const T r2 = x * x + y * y + z * z;
  const T ir = mc_rsqrt(r2);
  const T ir2 = ir * ir;
  harm_group_q<T>(t->iA, t->iB, p, x * ir2, y * ir2, z * ir2, ir2, ir, d1r, d1i, d2r, d2i, use);
}
