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

#define MC_PMAX 15
#define MC_MAXLEV 8
#define MC_THREADS 256
#define MC_WARPS (MC_THREADS / 32)
#define MC_MAX_ITEMS 384  // partial slots per step (the last one holds log u)
#define MC_NEAR_PARTS_MAX 4  // items per near cell and side (McSys.near_parts)
#define MC_NF_ROWS 6    // far-field row blocks of 32 rows (covers C <= 192)
#define MC_NF_COLS 16   // far-field column chunks (maximum; RunParams.nf_cols <= this)
#define MC_GPRE 16      // far-operator columns a warp keeps in registers
// CTAs per SM of the batched form's kernels (registers per thread capped at
// 256 / this; measured on GB300 with 64 chains: 3 for both evaluation types,
// FP64 with the pair-of-floats contributions 557k -> 572k MH steps/s from 2
// to 3, 527k at 4; the single-chain kernels keep one CTA per SM)
#define MC_BATCH_CTAS_PER_SM(TE) 3
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
  // speculative small-level deltas (rotating buffers of nsmall cells x C)
  double* dsmall;    // [4 * nsmall * C] (rotating buffers: three or four)
  int ls_end;        // first level with more than 4 cells per axis (or L + 1)
  int nsmall;        // cells of levels lmin .. ls_end-1 (the first cells of Lhat)
  unsigned long long* sync;  // [128]: [l] read epoch of level l, [12] near items done;
                             // mc_async.cu: counters at [16 i], i = 1..6
  // speculative accept: Alg. L.2 contributions staged during the proposal
  double* dacc;      // [4 (step) * (L - lmin + 1) * 2 * MC_DSLOTS * C] (phased: by step parity;
                     // mc_async.cu: by step mod 4 and side)
  double* dKpre;     // [4 * C] dK of the next proposal, by step (2 or 4 buffers)
  // multipole method (Sec. 3.3, alternative algorithm; method 1): per-level
  // scaled multipoles Mhat_n^m = sum q conj Rt_n^m(r - R_cell), Lhat's layout
  int method;
  double* Mhat;
  // short-range Lennard-Jones term (Sec. 5.3): 4 eps ((sig/r)^12 - (sig/r)^6)
  // for r^2 < rc2, between different particles of the near cells
  int lj_on;
  double lj_eps4, lj_s6, lj_s12, lj_rc2;
  // Alg. 1 split: each near cell's slots are shared by near_parts items per
  // side (2 near_parts items when r and r' share their finest cell), slot
  // blocks of 32 taken round robin; 1..MC_NEAR_PARTS_MAX
  int near_parts;
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

#include "mc_philox.cuh"

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
    // (acquire only: this thread's own writes were released by its arrival)
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
    asm volatile("fence.acquire.gpu;" ::: "memory");
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
    asm volatile("fence.acquire.gpu;" ::: "memory");
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

// relaxed FP64 reduction without a returned value.  Measured on GB300: the
// small-level contributions of the barrier-free chain and the accept of the
// plain schedule are faster with it than with atomicAdd (+3 % FP64 chain at
// N = 1e5 and NaCl, +8 % batched FP32-eval), the speculative items of the
// phased chain and the pair-of-floats batch slightly slower (-1 %), so
// those keep atomicAdd.  Ordered before the item's release like any store.
__device__ __forceinline__ void red_add_f64(double* p, double v) {
  asm volatile("red.relaxed.gpu.global.add.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}

#include "mc_harm.cuh"

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
#include "mc_geom.cuh"

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
