// Device-side data layout and building blocks of the GB300 multilevel
// Monte Carlo electrostatics library (Saunders, Grant & Mueller,
// arXiv 2006.16622).
//
// Representation.  Expansion coefficients are kept in a scaled real layout
// that removes every normalisation constant from the hot loops:
//   Lhat_n^m = L_n^m * s_nm,   s_nm = sqrt((n-m)! (n+m)!),   m >= 0,
// so that (Eq. 2)   Psi(x) = sum_n [Lhat_n^0 Rt_n^0 + 2 Re sum_{m>0} Lhat_n^m Rt_n^m]
// and (Alg. L.2)    Lhat_n^m += q conj(It_n^m(x_src - R_target))
// with the scaled solid harmonics (P_n^m without Condon-Shortley phase)
//   Rt_n^m(x) = r^n P_n^m(cos t) e^{i m phi} / (n+m)!
//   It_n^m(x) = (n-m)! r^-(n+1) P_n^m(cos t) e^{i m phi}.
// Real layout of one expansion: index n*n for m = 0, n*n + 2m - 1 (re) and
// n*n + 2m (im) for m > 0; (p+1)^2 doubles.
//
// Both scaled harmonics obey the same two-term recurrences, run per column m
// by one lane of a half-warp (lane = m, n advancing in lock step):
//   diagonal (n <= m):  X_n = A_n (x + i y) X_{n-1}
//   column   (n >  m):  X_n = A_nm z X_{n-1} - B_nm Q X_{n-2}
// regular:   A = 1/(2n) | (2n-1)/((n+m)(n-m)),  B = 1/((n+m)(n-m)), Q = r^2
// irregular: (x, y, z) -> (x, y, z)/r^2, A = 2n-1, B = (n+m-1)(n-m-1), Q = 1/r^2.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "mc_df64.cuh"
#include "mc_pair_harm.cuh"

#define MC_PMAX 15
#define MC_MAXLEV 8
#define MC_THREADS 256
#define MC_WARPS (MC_THREADS / 32)
#define MC_MAX_ITEMS 256
#define MC_NF_ROWS 6    // far-field row blocks of 32 rows (covers C <= 192)
#define MC_NF_COLS 16   // far-field column chunks (maximum; RunParams.nf_cols <= this)
#define MC_GPRE 16      // far-operator columns a warp keeps in registers
// CTAs per SM of the batched form's kernels, by evaluation type (registers
// per thread capped at 256 / this; measured on GB300 with 64 chains: FP64
// best at 2, FP32-eval at 3; the single-chain kernels keep one CTA per SM)
#define MC_BATCH_CTAS_PER_SM(TE) (sizeof(TE) == 8 ? 2 : 3)
#define MC_VAR_PLAIN 0  // chain kernel variants (see chain_body)
#define MC_VAR_SPEC 1
#define MC_VAR_MM 2
#define MC_VAR_SPECW 3  // MC_VAR_SPEC, column-scaled contributions (batched FP64)
#define MC_DSLOTS 380   // staged accept contributions per level (>= 378 targets)

// ---------------------------------------------------------------- state
struct McSys {
  int n, L, p, C, bc, dip, prec;
  int nL, cap, ncellL, lmin, ncell_total;
  double a, inv_wL, V;
  int lev_off[MC_MAXLEV + 2];  // first cell of level l in Lhat
  int lev_n[MC_MAXLEV + 2];    // cells per axis on level l
  double lev_w[MC_MAXLEV + 2]; // cell width on level l
  double4* ppos;     // [n]        (x, y, z, q) by particle id
  double4* cpos;     // [ncellL*cap] slot positions (x, y, z, q)
  float4* cpos32;    // [ncellL*cap] slot position relative to the cell centre, q
  int* cpid;         // [ncellL*cap] particle id of a slot
  int* ccount;       // [ncellL]
  int* pslot;        // [n] slot of a particle
  double* Lhat;      // [ncell_total * C] per-level local expansions
  double* Khat;      // [C] box multipole (scaled, conj of regular harmonics)
  double* Hhat;      // [C] lattice local expansion H = R(K) (scaled)
  double* G;         // [C*C] real far-field operator: Hhat = G Khat
  double* dipv;      // [3] dipole sum q r
  double* energy;    // [1] running energy
  double* partials;  // [4 * MC_MAX_ITEMS] (two used by the phased kernels, a ring of four by mc_async.cu)
  double* dK;        // [4 * C] change of Khat of the current proposal (by step: 2 or 4 buffers)
  double* gK;        // [4 * MC_NF_COLS * C] partial G dK of the current proposal (2 or 4 buffers)
  unsigned long long* bar;  // grid barrier counter
  int* status;       // device status word (MC_OK or MC_ERR_*)
  long long* stats;  // [4] steps, accepted, borderline, spare
  double* result;    // [4] dE of a single proposal, ...
  // pipelined chain (mc_pipe.cu): second H and dipole buffers, speculative
  // coarse-level deltas (3 rotating buffers of nsmall cells x C), sync words
  double* Hhat2;     // [C]
  double* dipv2;     // [3]
  double* dsmall;    // [4 * nsmall * C] (rotating buffers: three or four)
  int ls_end;        // first level with more than 4 cells per axis (or L + 1)
  int nsmall;        // cells of levels lmin .. ls_end-1 (the first cells of Lhat)
  unsigned long long* sync;  // [128]: [l] read epoch of level l, [12] near items done;
                             // mc_async.cu: counters at [16 i], i = 1..6
  // speculative accept: Alg. L.2 contributions staged during the proposal
  double* dacc;      // [4 (step) * (L - lmin + 1) * 2 * MC_DSLOTS * C] (phased: by step parity;
                     // mc_async.cu: by step mod 4 and side)
  double* dKpre;     // [4 * C] dK of the next proposal, by step (2 or 4 buffers)
  // multipole method (Sec. 3.2, alternative algorithm; method 1): per-level
  // scaled multipoles Mhat_n^m = sum q conj Rt_n^m(r - R_cell), Lhat's layout
  int method;
  double* Mhat;
  // short-range Lennard-Jones term (Sec. 5.4): 4 eps ((sig/r)^12 - (sig/r)^6)
  // for r^2 < rc2, between different particles of the near cells
  int lj_on;
  double lj_eps4, lj_s6, lj_s12, lj_rc2;
};

struct RunParams {
  int mode;  // 0: chain with Philox proposals, 1: propose a given move, 2: accept a given move
  long long step0, nsteps;
  unsigned long long seed;
  double beta, h;
  long long jg;
  double rx, ry, rz;
  int has_dE;
  double dEg;
  long long stop_after_accepts;  // 0 = none
  long long* log_j;
  double* log_dE;
  unsigned char* log_acc;
  long long wait_ns;
  unsigned long long* prof;  // optional phase/item timers (see mc_chain.cu), may be null
  int nf_cols;               // far-field column blocks per row block, 1..MC_NF_COLS
  unsigned chain;            // Philox counter word 2 (chain id)
  unsigned bar_missing;      // arrivals each grid barrier waits for that never
                             // come (failure-path tests; 0 in normal runs)
  int spec;                  // 1: Alg. L.2 contributions computed during the
                             // proposal phase, applied after the decision
};

// ------------------------------------------------------------ error codes
#define MCD_OK 0
#define MCD_ERR_TIMEOUT (-7)
#define MCD_ERR_CAPACITY (-8)

// ------------------------------------------------------------ Philox4x32-10
// Salmon et al. (SC'11): two 32x32 multiplies per round, Weyl key bumps.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Proposal of global step s: j = floor(A0 n / 2^32); delta_k = h (2u_k - 1),
// u_k = (A_k + 1/2) 2^-32; acceptance uniform ((B0>>5) 2^26 + (B1>>6)) 2^-53.
// Written with explicit round-to-nearest intrinsics so that no contraction
// changes the bits of the displacement.
__device__ __forceinline__ void mc_proposal(unsigned long long seed, unsigned long long s,
                                            uint32_t chain, int n, double h, int* j,
                                            double d[3], double* u) {
  uint32_t A[4] = {(uint32_t)s, (uint32_t)(s >> 32), chain, 0u};
  uint32_t B[4] = {(uint32_t)s, (uint32_t)(s >> 32), chain, 1u};
  philox4x32_10(A, (uint32_t)seed, (uint32_t)(seed >> 32));
  philox4x32_10(B, (uint32_t)seed, (uint32_t)(seed >> 32));
  *j = (int)(((unsigned long long)A[0] * (unsigned long long)n) >> 32);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    double uk = __dmul_rn(__dadd_rn((double)A[k + 1], 0.5), 2.3283064365386963e-10);
    d[k] = __dmul_rn(h, __dsub_rn(__dmul_rn(2.0, uk), 1.0));
  }
  *u = __dmul_rn(__dadd_rn(__dmul_rn((double)(B[0] >> 5), 67108864.0), (double)(B[1] >> 6)),
                 1.1102230246251565e-16);
}

// One axis of the proposal: every lane runs both Philox blocks (integer
// work), the FP64 arithmetic of the displacement is per axis, u only where
// requested.
__device__ __forceinline__ void mc_proposal_axis(unsigned long long seed, unsigned long long s,
                                                 uint32_t chain, int n, double h, int axis, int* j,
                                                 double* d, double* u) {
  uint32_t A[4] = {(uint32_t)s, (uint32_t)(s >> 32), chain, 0u};
  uint32_t B[4] = {(uint32_t)s, (uint32_t)(s >> 32), chain, 1u};
  philox4x32_10(A, (uint32_t)seed, (uint32_t)(seed >> 32));
  philox4x32_10(B, (uint32_t)seed, (uint32_t)(seed >> 32));
  *j = (int)(((unsigned long long)A[0] * (unsigned long long)n) >> 32);
  const uint32_t w = axis == 0 ? A[1] : (axis == 1 ? A[2] : A[3]);
  const double uk = __dmul_rn(__dadd_rn((double)w, 0.5), 2.3283064365386963e-10);
  *d = __dmul_rn(h, __dsub_rn(__dmul_rn(2.0, uk), 1.0));
  if (u)
    *u = __dmul_rn(__dadd_rn(__dmul_rn((double)(B[0] >> 5), 67108864.0), (double)(B[1] >> 6)),
                   1.1102230246251565e-16);
}

// IEEE-754 conversions on the integer pipe (the FP64 pipe is 1/64 rate).
// float -> double is exact for normal floats; subnormal floats become 0.
__device__ __forceinline__ double f2d_int(float f) {
  const uint32_t b = __float_as_uint(f);
  const uint32_t e = (b >> 23) & 0xffu;
  const uint32_t sign = b & 0x80000000u;
  const uint32_t hi = e ? (sign | ((e + 896u) << 20) | ((b & 0x7fffffu) >> 3)) : sign;
  const uint32_t lo = e ? (b << 29) : 0u;
  return __hiloint2double((int)hi, (int)lo);
}
// double -> float rounded toward zero; |x| beyond the float range saturates
// to +-inf, below it flushes to 0 (branch-free).
__device__ __forceinline__ float d2f_int(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const int e = (int)((hi >> 20) & 0x7ffu) - 896;
  uint32_t mag = ((uint32_t)e << 23) | ((hi & 0xfffffu) << 3) | (lo >> 29);
  mag = (e <= 0) ? 0u : mag;
  mag = (e >= 255) ? 0x7f800000u : mag;
  return __uint_as_float((hi & 0x80000000u) | mag);
}
template <typename T> __device__ __forceinline__ T from_double(double x);
template <> __device__ __forceinline__ double from_double<double>(double x) { return x; }
template <> __device__ __forceinline__ float from_double<float>(double x) { return d2f_int(x); }
__device__ __forceinline__ double to_double(double x) { return x; }
__device__ __forceinline__ double to_double(float x) { return f2d_int(x); }

// ---------------------------------------------------------- grid barrier
// Monotone 64-bit arrival counter; thread 0 of every CTA arrives with a
// release add and spins with acquire loads until all CTAs of this
// generation arrived.  The spin is bounded by wall time (globaltimer): on
// expiry the status word gets MCD_ERR_TIMEOUT and the caller leaves its loop.
__device__ __forceinline__ unsigned long long mc_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ bool grid_barrier(unsigned long long* ctr, unsigned long long target,
                                             int* status, long long wait_ns) {
  __syncthreads();
  __shared__ int s_ok;
  if (threadIdx.x == 0) {
    asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(ctr) : "memory");
    unsigned long long v;
    unsigned long long t0 = mc_globaltimer();
    int ok = 1;
    unsigned spins = 0;
    // poll with relaxed loads (an acquire per poll would invalidate the SM's
    // L1 for every warp on it); one acquire fence once the count is reached
    while (true) {
      asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
      if (v >= target) break;
      if ((++spins & 255u) == 0u) {
        if ((long long)(mc_globaltimer() - t0) > wait_ns) {
          atomicExch(status, MCD_ERR_TIMEOUT);
          ok = 0;
          break;
        }
        if (*((volatile int*)status) != MCD_OK) {
          ok = 0;
          break;
        }
      }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
    s_ok = ok;
  }
  __syncthreads();
  return s_ok != 0;
}

// Split grid barrier: arrive (release) without waiting ...
__device__ __forceinline__ void grid_arrive(unsigned long long* ctr) {
  __syncthreads();
  if (threadIdx.x == 0) asm volatile("red.release.gpu.global.add.u64 [%0], 1;" ::"l"(ctr) : "memory");
}

// ... and a wait of one warp for a target count (lane 0 polls, bounded by
// wait_ns; acquire once the count is reached); false on timeout or when
// another CTA has set an error status
__device__ __forceinline__ bool warp_wait(unsigned long long* ctr, unsigned long long target,
                                          int* status, long long wait_ns) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
    if (v < target) {
      const unsigned long long t0 = mc_globaltimer();
      unsigned spins = 0;
      while (true) {
        asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
        if (v >= target) break;
        if ((++spins & 63u) == 0u) {
          if ((long long)(mc_globaltimer() - t0) > wait_ns) {
            atomicExch(status, MCD_ERR_TIMEOUT);
            ok = 0;
            break;
          }
          if (*((volatile int*)status) != MCD_OK) {
            ok = 0;
            break;
          }
        }
      }
    }
    asm volatile("fence.acq_rel.gpu;" ::: "memory");
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

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

// Lennard-Jones pair energy from 1/r^2 (0 at or beyond the cutoff)
template <typename T>
__device__ __forceinline__ T lj_energy(T inv2, T d2, T eps4, T s6, T s12, T rc2) {
  const T inv6 = inv2 * inv2 * inv2;
  return d2 < rc2 ? eps4 * (s12 * inv6 * inv6 - s6 * inv6) : T(0);
}

// sign flip on the integer pipe (a negation alone would be an FP64 op)
__device__ __forceinline__ double neg_bits(double x) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)0x8000000000000000ULL);
}
__device__ __forceinline__ float neg_bits(float x) { return -x; }

// index of (n, m) in the real layout (re part; im part is +1 for m > 0)
__device__ __forceinline__ int rl_re(int n, int m) { return n * n + (m ? 2 * m - 1 : 0); }

// ------------------------------------------------------------- geometry
// Interaction-list offsets (Sec. 3.1) for the 8 parity classes of a cell:
// children of the parent's 27 neighbours span [-2-b, 3-b] per axis (b the
// cell's parity on that axis); the 27 near offsets are removed.  Built per
// CTA in shared memory: il[parity][k] = packed (ox+4) | (oy+4)<<4 | (oz+4)<<8.
__device__ __forceinline__ void il_table_init(unsigned short (*il)[189]) {
  for (int t = threadIdx.x; t < 8 * 216; t += blockDim.x) {
    const int par = t / 216, b = t % 216;
    const int bx = (par >> 2) & 1, by = (par >> 1) & 1, bz = par & 1;
    const int i = b / 36, jj = (b / 6) % 6, l = b % 6;
    const int ox = i - 2 - bx, oy = jj - 2 - by, oz = l - 2 - bz;
    const bool inner = (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1);
    if (inner) continue;
    // rank of b among the non-inner entries of this parity class
    int k = 0;
    for (int bb = 0; bb < b; bb++) {
      const int ii = bb / 36, j2 = (bb / 6) % 6, l2 = bb % 6;
      const int px = ii - 2 - bx, py = j2 - 2 - by, pz = l2 - 2 - bz;
      if (!(px >= -1 && px <= 1 && py >= -1 && py <= 1 && pz >= -1 && pz <= 1)) k++;
    }
    il[par][k] = (unsigned short)((ox + 4) | ((oy + 4) << 4) | ((oz + 4) << 8));
  }
}
__device__ __forceinline__ void il_unpack(unsigned short v, int* ox, int* oy, int* oz) {
  *ox = (int)(v & 15) - 4;
  *oy = (int)((v >> 4) & 15) - 4;
  *oz = (int)((v >> 8) & 15) - 4;
}

__device__ __forceinline__ int mc_wrap_coord(int e, int n) { return ((e % n) + n) % n; }

__device__ __forceinline__ bool in_il(int ox, int oy, int oz, int cx, int cy, int cz) {
  const int bx = cx & 1, by = cy & 1, bz = cz & 1;
  if (ox < -2 - bx || ox > 3 - bx || oy < -2 - by || oy > 3 - by || oz < -2 - bz || oz > 3 - bz)
    return false;
  return (ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1);
}

__device__ __forceinline__ int finest_coord(double x, double inv_w, int nL) {
  int v = (int)floor(__dmul_rn(x, inv_w));
  return v < 0 ? 0 : (v > nL - 1 ? nL - 1 : v);
}

// 32-byte record loaded through L2 only (state written by other CTAs)
__device__ __forceinline__ double4 ldcg4(const double4* p) {
  const double2* q = reinterpret_cast<const double2*>(p);
  const double2 a = __ldcg(q), b = __ldcg(q + 1);
  return make_double4(a.x, a.y, b.x, b.y);
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
template <typename T>
__device__ __forceinline__ T half_sum(T v) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}
