// C-ABI entry points of the GB300 multilevel Monte Carlo electrostatics
// library (declared in include/mcfmm.h).  Host code only: argument checks,
// device memory ownership, kernel launches and copies.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <map>
#include <mutex>
#include <utility>
#include <vector>

#include "../../include/mcfmm.h"
#include "mc_dev.cuh"

// kernels defined in the other translation units
cudaError_t mc_launch_chain(const McSys* d_sys, const RunParams& rp, int prec, int var, int nCTA,
                            cudaStream_t stream);
cudaError_t mc_launch_async(const McSys* d_sys, const RunParams& rp, int prec, int nCTA,
                            cudaStream_t stream);
cudaError_t mc_launch_batch(const McSys* const* d_systems, RunParams* d_rps, const int* d_cta_chain,
                            const int* d_cta_rank, const int* d_chain_ctas, int prec, int var,
                            int nCTA, cudaStream_t stream);
int mc_chain_max_ctas(int prec);
int mc_batch_max_ctas(int prec);
__global__ void k_cell_count(int, const double4*, double, int, int*, int*);
__global__ void k_cell_fill(int, const int*, int, int*, int*);
__global__ void k_cell_sort(int, int, int, double, const int*, const double4*, int*, double4*,
                            float4*, int*);
__global__ void k_max_int(int, const int*, int*);
__global__ void k_p2l_level(const McSys*, int, int, double*);
__global__ void k_reduce_chunks(int, int, int, const double*, double*);
__global__ void k_box_multipole(const McSys*, int, double*);
__global__ void k_far_finish(const McSys*, int, const double*);
__global__ void k_energy_particles(const McSys*, double*);
__global__ void k_energy_finish(const McSys*, int, const double*, double*);
__global__ void k_lattice_sums(int, double*);
__global__ void k_far_operator(int, double, const double*, double*);
__global__ void k_p2m_level(const McSys*, int, int, double*);
__global__ void k_offset_table(int, double*);
cudaError_t m2l_launch(const McSys*, int, int, int, int, const double*, const double*, double*, double*,
                       size_t, cudaStream_t);
int m2l_offset_chunks(int nl, int sms);

struct mc_ctx {
  McSys h;        // host copy holding device pointers
  McSys* d_sys;   // device copy
  cudaStream_t stream;
  int dev;
  int nCTA;  // chain grid set by mc_set_ctas; 0: the default by form and schedule
  int sms;
  int setup_done;
  long long steps_total;
  long long wait_ns;
  unsigned bar_missing;  // mc_inject_wait_fault
  double* d_scratch;
  size_t scratch_doubles;
  double* d_energy_tmp;  // fresh-energy target
  unsigned long long* d_prof;  // MC_PROF_COUNTERS timers when profiling is on, else null
  int schedule;                // MC_SCHEDULE_*
  double* d_mpole;             // per-level multipoles (fast setup), allocated on first use
  double* d_otab;              // offset harmonics table (fast setup)
  std::vector<void*> allocs;
};

namespace {

#define CK(x)                              \
  do {                                     \
    cudaError_t e_ = (x);                  \
    if (e_ != cudaSuccess) return MC_ERR_CUDA; \
  } while (0)

int dalloc(mc_ctx* c, void** p, size_t bytes) {
  if (bytes == 0) bytes = 16;
  if (cudaMalloc(p, bytes) != cudaSuccess) {
    cudaGetLastError();
    return MC_ERR_NOMEM;
  }
  c->allocs.push_back(*p);
  return MC_OK;
}

double fact(int k) {
  double f = 1.0;
  for (int i = 2; i <= k; i++) f *= i;
  return f;
}

// s_nm = sqrt((n-m)! (n+m)!) of real-layout index k
double scale_of(int k) {
  int n = (int)floor(sqrt((double)k) + 1e-9);
  while (n * n > k) n--;
  while ((n + 1) * (n + 1) <= k) n++;
  const int rem = k - n * n, m = (rem + 1) / 2;
  return sqrt(fact(n - m) * fact(n + m));
}

// chunks of the interaction list per target on level l (1 = write in place)
// chunks per target cell of the Alg. L.3 gather on level l: about eight
// equal tasks per resident warp (one CTA per SM), at most one chunk per
// source unit (189 finest cells of the list per target and level cell)
int chunks_for_level(const McSys& h, int sms, int l, size_t max_doubles) {
  const long long ncl = (long long)h.lev_n[l] * h.lev_n[l] * h.lev_n[l];
  const long long f = 1LL << (h.L - l);
  const long long units = 189LL * f * f * f;
  long long nchunk = std::min<long long>(units, std::max<long long>(1, (8LL * sms * MC_WARPS + ncl - 1) / ncl));
  if (nchunk > 1 && (size_t)(ncl * nchunk * h.C) > max_doubles)
    nchunk = std::max<long long>(1, (long long)(max_doubles / ((size_t)ncl * h.C)));
  return (int)nchunk;
}

const size_t kScratchCap = (size_t)1 << 24;  // doubles (128 MiB)

int grid_for(int sms, size_t work, int per_block) {
  size_t b = (work + per_block - 1) / per_block;
  size_t lim = (size_t)sms * 8;
  if (b > lim) b = lim;
  if (b < 1) b = 1;
  return (int)b;
}

int sync_status(mc_ctx* c) {
  if (cudaStreamSynchronize(c->stream) != cudaSuccess) return MC_ERR_CUDA;
  int st = 0;
  if (cudaMemcpy(&st, c->h.status, sizeof(int), cudaMemcpyDeviceToHost) != cudaSuccess)
    return MC_ERR_CUDA;
  return st;
}

int launch_chain(mc_ctx* c, RunParams& rp) {
  rp.wait_ns = c->wait_ns;
  rp.bar_missing = c->bar_missing;
  rp.prof = c->d_prof;
  const bool mm = c->h.method == 1;
  // single proposals and the multipole method run on the phased kernel
  const bool async = !mm && rp.mode == 0 && c->schedule == MC_SCHEDULE_ASYNC;
  rp.nf_cols = MC_NF_COLS;
  rp.spec = (!mm && (c->schedule == MC_SCHEDULE_PHASED || c->schedule == MC_SCHEDULE_ASYNC)) ? 1 : 0;
  rp.chain = 0u;
  // grid: the caller's (mc_set_ctas), else every SM, except for the phased
  // FP32-eval chain of the local method, which is faster on 5/7 of the SMs
  // (GB300, 108 of 152 CTAs: +0.5..4 % at N = 1e4..1e6, its short items pay
  // more for the barrier arrivals than they gain from the extra warps); the
  // barrier-free chain needs every SM (its step's items fill the grid's
  // warps: -4 % on 128 CTAs, -15 % on 114 at N = 1e5)
  int grid = c->nCTA;
  if (grid == 0)
    grid = (!mm && !async && rp.spec && c->h.prec == MC_FP32_EVAL) ? std::max(1, (5 * c->sms) / 7) : c->sms;
  CK(cudaMemsetAsync(c->h.bar, 0, sizeof(unsigned long long), c->stream));
  CK(cudaMemsetAsync(c->h.status, 0, sizeof(int), c->stream));
  if (async) {
    // counters, partial-slot ring at its "not written" pattern (all bits
    // set), the four small-level contribution buffers clear
    CK(cudaMemsetAsync(c->h.sync, 0, sizeof(unsigned long long) * 128, c->stream));
    CK(cudaMemsetAsync(c->h.partials, 0xFF, sizeof(double) * 4 * MC_MAX_ITEMS, c->stream));
    if (c->h.nsmall > 0)
      CK(cudaMemsetAsync(c->h.dsmall, 0, sizeof(double) * 4 * (size_t)c->h.nsmall * c->h.C, c->stream));
    CK(mc_launch_async(c->d_sys, rp, c->h.prec, grid, c->stream));
  } else {
    // the two small-level delta buffers of the speculative accept start clear
    if (rp.spec && c->h.nsmall > 0)
      CK(cudaMemsetAsync(c->h.dsmall, 0, sizeof(double) * 3 * (size_t)c->h.nsmall * c->h.C, c->stream));
    CK(mc_launch_chain(c->d_sys, rp, c->h.prec,
                       mm ? MC_VAR_MM : (rp.spec ? MC_VAR_SPEC : MC_VAR_PLAIN), grid, c->stream));
  }
  return MC_OK;
}

int run_setup(mc_ctx* c) {
  McSys& h = c->h;
  const int C = h.C;
  // Alg. L.3 per level (gather, chunked over the interaction list)
  for (int l = h.lmin; l <= h.L; l++) {
    const int nl = h.lev_n[l], ncl = nl * nl * nl;
    const int nchunk = chunks_for_level(h, c->sms, l, c->scratch_doubles);
    const int ntask = ncl * nchunk;
    double* dst = h.Lhat + (size_t)h.lev_off[l] * C;
    k_p2l_level<<<grid_for(c->sms, ntask, MC_WARPS), MC_THREADS, 0, c->stream>>>(
        c->d_sys, l, nchunk, nchunk > 1 ? c->d_scratch : dst);
    CK(cudaGetLastError());
    if (nchunk > 1) {
      k_reduce_chunks<<<grid_for(c->sms, (size_t)ncl * C, 256), 256, 0, c->stream>>>(
          ncl, nchunk, C, c->d_scratch, dst);
      CK(cudaGetLastError());
    }
  }
  // K, dipole, H = G K
  const int nch = std::min<int>(1024, std::max<int>(1, h.n / 64));
  k_box_multipole<<<grid_for(c->sms, nch, MC_WARPS), MC_THREADS, 0, c->stream>>>(c->d_sys, nch,
                                                                                c->d_scratch);
  CK(cudaGetLastError());
  k_far_finish<<<1, 256, 0, c->stream>>>(c->d_sys, nch, c->d_scratch);
  CK(cudaGetLastError());
  return MC_OK;
}

// FMM-variant initialisation (fast mode): multipoles of every level, then
// multipole-to-local over the interaction lists
// per-level multipoles (Eq. 4) of every cell into d_mpole (allocated on
// first use): the fast setup's first pass and Alg. M.3
int p2m_levels(mc_ctx* c) {
  McSys& h = c->h;
  const int C = h.C;
  if (!c->d_mpole &&
      dalloc(c, (void**)&c->d_mpole, sizeof(double) * (size_t)std::max(1, h.ncell_total) * C) != MC_OK)
    return MC_ERR_NOMEM;
  for (int l = h.lmin; l <= h.L; l++) {
    const int nl = h.lev_n[l], ncl = nl * nl * nl;
    const int f = 1 << (h.L - l);
    double* M = c->d_mpole + (size_t)h.lev_off[l] * C;
    long long nchunk = std::min<long long>((long long)f * f * f,
                                           std::max<long long>(1, (4LL * c->sms * MC_WARPS + ncl - 1) / ncl));
    if (nchunk > 1 && (size_t)(ncl * nchunk * C) > c->scratch_doubles)
      nchunk = std::max<long long>(1, (long long)(c->scratch_doubles / ((size_t)ncl * C)));
    const long long ntask = (long long)ncl * nchunk;
    k_p2m_level<<<grid_for(c->sms, (size_t)ntask, MC_WARPS), MC_THREADS, 0, c->stream>>>(
        c->d_sys, l, (int)nchunk, nchunk > 1 ? c->d_scratch : M);
    CK(cudaGetLastError());
    if (nchunk > 1) {
      k_reduce_chunks<<<grid_for(c->sms, (size_t)ncl * C, 256), 256, 0, c->stream>>>(
          ncl, (int)nchunk, C, c->d_scratch, M);
      CK(cudaGetLastError());
    }
  }
  return MC_OK;
}

// the box multipole K, dipole and H = G K
int setup_far(mc_ctx* c) {
  const int nch = std::min<int>(1024, std::max<int>(1, c->h.n / 64));
  k_box_multipole<<<grid_for(c->sms, nch, MC_WARPS), MC_THREADS, 0, c->stream>>>(c->d_sys, nch,
                                                                                c->d_scratch);
  CK(cudaGetLastError());
  k_far_finish<<<1, 256, 0, c->stream>>>(c->d_sys, nch, c->d_scratch);
  CK(cudaGetLastError());
  return MC_OK;
}

// the state of one method on the device: method 0 (local) or 1 (multipole)
int set_method(mc_ctx* c, int method) {
  c->h.method = method;
  c->h.Mhat = method ? c->d_mpole : nullptr;
  CK(cudaMemcpyAsync(c->d_sys, &c->h, sizeof(McSys), cudaMemcpyHostToDevice, c->stream));
  return MC_OK;
}

// Alg. M.3 with K/E/H: the multipole method's initialisation
int run_setup_mm(mc_ctx* c) {
  int rc = p2m_levels(c);
  if (rc != MC_OK) return rc;
  if ((rc = set_method(c, 1)) != MC_OK) return rc;
  return setup_far(c);
}

int run_setup_fmm(mc_ctx* c) {
  McSys& h = c->h;
  const int C = h.C, p = h.p;
  const int per = (2 * p + 1) * (2 * p + 2) / 2;
  if (!c->d_otab) {
    if (dalloc(c, (void**)&c->d_otab, sizeof(double) * 2 * 343 * (size_t)per) != MC_OK)
      return MC_ERR_NOMEM;
    k_offset_table<<<grid_for(c->sms, 343 * (size_t)per, 256), 256, 0, c->stream>>>(p, c->d_otab);
    CK(cudaGetLastError());
  }
  int rc = p2m_levels(c);
  if (rc != MC_OK) return rc;
  for (int l = h.lmin; l <= h.L; l++) {
    CK(m2l_launch(c->d_sys, p, l, h.lev_n[l], c->sms, c->d_mpole + (size_t)h.lev_off[l] * C,
                  c->d_otab, h.Lhat + (size_t)h.lev_off[l] * C, c->d_scratch, c->scratch_doubles,
                  c->stream));
  }
  const int nch = std::min<int>(1024, std::max<int>(1, h.n / 64));
  k_box_multipole<<<grid_for(c->sms, nch, MC_WARPS), MC_THREADS, 0, c->stream>>>(c->d_sys, nch,
                                                                                c->d_scratch);
  CK(cudaGetLastError());
  k_far_finish<<<1, 256, 0, c->stream>>>(c->d_sys, nch, c->d_scratch);
  CK(cudaGetLastError());
  return MC_OK;
}

int energy_into(mc_ctx* c, double* d_dst) {
  const int blocks = c->sms * 2;
  const int nw = blocks * MC_WARPS;
  k_energy_particles<<<blocks, MC_THREADS, 0, c->stream>>>(c->d_sys, c->d_scratch);
  CK(cudaGetLastError());
  k_energy_finish<<<1, 256, 0, c->stream>>>(c->d_sys, nw, c->d_scratch, d_dst);
  CK(cudaGetLastError());
  return MC_OK;
}

// The unit-lattice sums depend only on lmax: one device table per (device,
// lmax), computed on first use and kept for the life of the process
// (2 (lmax+1)^2 doubles each).
std::map<std::pair<int, int>, double*> g_lattice_cache;
std::mutex g_lattice_mutex;

int lattice_table(int dev, int lmax, cudaStream_t stream, const double** out) {
  std::lock_guard<std::mutex> lock(g_lattice_mutex);
  auto it = g_lattice_cache.find({dev, lmax});
  if (it != g_lattice_cache.end()) {
    *out = it->second;
    return MC_OK;
  }
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 2 * (lmax + 1) * (lmax + 1)) != cudaSuccess) {
    cudaGetLastError();
    return MC_ERR_NOMEM;
  }
  k_lattice_sums<<<(lmax + 1) * (lmax + 2) / 2, 256, 0, stream>>>(lmax, d);
  if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(stream) != cudaSuccess) {
    cudaFree(d);
    return MC_ERR_CUDA;
  }
  g_lattice_cache[{dev, lmax}] = d;
  *out = d;
  return MC_OK;
}

// partial slots per step of the chain kernels with near_parts = P: the
// barrier-free chain's far items (row blocks x MC_NF_COLS column chunks),
// 54 P near items, image and log u, four expansion items per level (the
// phased chain takes fewer); the last slot holds log u itself
bool near_parts_fit(const McSys& h, int P) {
  const int nF = h.bc == MC_BC_PBC ? ((h.C + 31) / 32) * MC_NF_COLS : 0;
  return nF + 54 * P + 2 + 4 * (h.L - h.lmin + 1) <= MC_MAX_ITEMS - 1;
}

// Near items per cell and side by mean finest-cell occupancy: one item per
// 48 charges, at most MC_NEAR_PARTS_MAX, within the slot budget.  Alg. 1 is
// the longest FP64 item of dense cells (about 190 charges at the NaCl
// full-MC setting, L = 4), so its loop is split there (measured on GB300,
// FP64 barrier-free chain: 66k / 81k / 84k / 86k MH steps/s for 1..4 items;
// uniform N = 1e5 at 24 per cell is fastest with one).
int near_parts_auto(const McSys& h) {
  const double mean = (double)h.n / (double)std::max(1, h.ncellL);
  int P = std::min(MC_NEAR_PARTS_MAX, std::max(1, (int)ceil(mean / 48.0)));
  while (P > 1 && !near_parts_fit(h, P)) P--;
  return P;
}

int in_box(const double* x, double a) {
  for (int k = 0; k < 3; k++)
    if (!(x[k] >= 0.0 && x[k] < a)) return 0;
  return 1;
}

}  // namespace

extern "C" {

const char* mc_strerror(int s) {
  switch (s) {
    case MC_OK: return "ok";
    case MC_ERR_ARG: return "invalid argument";
    case MC_ERR_NONNEUTRAL: return "periodic boundaries need a neutral system";
    case MC_ERR_LEVELS: return "levels must be in 2..8";
    case MC_ERR_OUTSIDE: return "position outside [0, a)^3";
    case MC_ERR_CUDA: return "CUDA runtime error";
    case MC_ERR_TIMEOUT: return "device-side wait timed out";
    case MC_ERR_CAPACITY: return "finest cell capacity exceeded";
    case MC_ERR_ORDER: return "expansion order must be in 0..15";
    case MC_ERR_STATE: return "call out of order";
    case MC_ERR_NOMEM: return "device allocation failed";
    case MC_ERR_SCRATCH: return "request exceeds the fixed no-allocation scratch";
    case MC_ERR_PENDING: return "a CUDA error of earlier work was pending";
    default: return "unknown status";
  }
}

void mc_destroy(mc_ctx* c) {
  if (!c) return;
  cudaSetDevice(c->dev);
  cudaStreamSynchronize(c->stream);
  for (void* p : c->allocs) cudaFree(p);
  delete c;
}

int mc_init(mc_ctx** out, int64_t n, const double* pos, const double* q, double box, int levels,
            int p, int bc, int dipole_bc, int precision, void* cuda_stream) {
  if (!out || !pos || !q || n < 1 || n > (1LL << 30) || !(box > 0.0) || !isfinite(box))
    return MC_ERR_ARG;
  *out = nullptr;
  if (levels < 2 || levels > 8) return MC_ERR_LEVELS;
  if (p < 0 || p > MC_PMAX) return MC_ERR_ORDER;
  if ((bc != MC_BC_PBC && bc != MC_BC_FREE) || (dipole_bc != MC_TINFOIL && dipole_bc != MC_VACUUM) ||
      (precision != MC_FP64 && precision != MC_FP32_EVAL))
    return MC_ERR_ARG;
  double qs = 0.0;
  for (int64_t i = 0; i < n; i++) {
    if (!in_box(pos + 3 * i, box)) return MC_ERR_OUTSIDE;
    if (!isfinite(q[i])) return MC_ERR_ARG;
    qs += q[i];
  }
  if (bc == MC_BC_PBC && fabs(qs) > 1e-9) return MC_ERR_NONNEUTRAL;

  mc_ctx* c = new mc_ctx();
  c->stream = (cudaStream_t)cuda_stream;
  c->wait_ns = 2000000000LL;
  if (cudaGetDevice(&c->dev) != cudaSuccess) {
    delete c;
    return MC_ERR_CUDA;
  }
  cudaDeviceGetAttribute(&c->sms, cudaDevAttrMultiProcessorCount, c->dev);
  McSys& h = c->h;
  memset(&h, 0, sizeof(h));
  h.n = (int)n;
  h.L = levels;
  h.p = p;
  h.C = (p + 1) * (p + 1);
  h.bc = bc;
  h.dip = dipole_bc;
  h.prec = precision;
  h.a = box;
  h.V = box * box * box;
  h.nL = 1 << (levels - 1);
  h.inv_wL = (double)h.nL / box;
  h.ncellL = h.nL * h.nL * h.nL;
  h.lmin = (bc == MC_BC_PBC) ? 2 : 3;
  int off = 0;
  for (int l = 1; l <= levels; l++) {
    h.lev_n[l] = 1 << (l - 1);
    h.lev_w[l] = box / (double)h.lev_n[l];
    h.lev_off[l] = off;
    if (l >= h.lmin) off += h.lev_n[l] * h.lev_n[l] * h.lev_n[l];
  }
  h.ncell_total = off;

  int rc = MC_OK;
#define DA(ptr, bytes)                                  \
  do {                                                  \
    rc = dalloc(c, (void**)&(ptr), (bytes));            \
    if (rc != MC_OK) {                                  \
      mc_destroy(c);                                    \
      return rc;                                        \
    }                                                   \
  } while (0)
#define DCK(x)              \
  do {                      \
    if ((x) != cudaSuccess) { \
      mc_destroy(c);        \
      return MC_ERR_CUDA;   \
    }                       \
  } while (0)

  // particles
  std::vector<double4> hp(n);
  for (int64_t i = 0; i < n; i++) hp[i] = make_double4(pos[3 * i], pos[3 * i + 1], pos[3 * i + 2], q[i]);
  DA(h.ppos, sizeof(double4) * n);
  DCK(cudaMemcpyAsync(h.ppos, hp.data(), sizeof(double4) * n, cudaMemcpyHostToDevice, c->stream));
  int *d_cell_of = nullptr, *d_cnt = nullptr, *d_max = nullptr;
  DA(d_cell_of, sizeof(int) * n);
  DA(d_cnt, sizeof(int) * h.ncellL);
  DA(d_max, sizeof(int));
  DCK(cudaMemsetAsync(d_cnt, 0, sizeof(int) * h.ncellL, c->stream));
  DCK(cudaMemsetAsync(d_max, 0, sizeof(int), c->stream));
  k_cell_count<<<grid_for(c->sms, n, 256), 256, 0, c->stream>>>(h.n, h.ppos, h.inv_wL, h.nL, d_cell_of, d_cnt);
  k_max_int<<<grid_for(c->sms, h.ncellL, 256), 256, 0, c->stream>>>(h.ncellL, d_cnt, d_max);
  int maxc = 0;
  DCK(cudaMemcpyAsync(&maxc, d_max, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  DCK(cudaStreamSynchronize(c->stream));
  // slot capacity: twice the initial occupancy plus room, multiple of 32
  int cap = std::max(32, std::max(2 * maxc, maxc + 32));
  cap = (cap + 31) / 32 * 32;
  h.cap = cap;
  const size_t nslot = (size_t)h.ncellL * cap;
  DA(h.cpos, sizeof(double4) * nslot);
  DA(h.cpos32, sizeof(float4) * nslot);
  DA(h.cpid, sizeof(int) * nslot);
  DA(h.ccount, sizeof(int) * h.ncellL);
  DA(h.pslot, sizeof(int) * n);
  DCK(cudaMemcpyAsync(h.ccount, d_cnt, sizeof(int) * h.ncellL, cudaMemcpyDeviceToDevice, c->stream));
  DCK(cudaMemsetAsync(d_cnt, 0, sizeof(int) * h.ncellL, c->stream));
  k_cell_fill<<<grid_for(c->sms, n, 256), 256, 0, c->stream>>>(h.n, d_cell_of, cap, d_cnt, h.cpid);
  k_cell_sort<<<grid_for(c->sms, h.ncellL, 128), 128, 0, c->stream>>>(
      h.ncellL, h.nL, cap, h.lev_w[levels], h.ccount, h.ppos, h.cpid, h.cpos, h.cpos32, h.pslot);
  DCK(cudaGetLastError());

  // expansions and far field
  const int C = h.C;
  DA(h.Lhat, sizeof(double) * (size_t)std::max(1, h.ncell_total) * C);
  DCK(cudaMemsetAsync(h.Lhat, 0, sizeof(double) * (size_t)std::max(1, h.ncell_total) * C, c->stream));
  DA(h.Khat, sizeof(double) * C);
  DA(h.Hhat, sizeof(double) * C);
  DA(h.G, sizeof(double) * (size_t)C * C);
  DA(h.dipv, sizeof(double) * 3);
  DA(h.energy, sizeof(double));
  DA(h.partials, sizeof(double) * 4 * MC_MAX_ITEMS);
  DA(h.dK, sizeof(double) * 4 * C);
  DA(h.gK, sizeof(double) * 4 * MC_NF_COLS * C);
  DA(h.bar, sizeof(unsigned long long));
  DA(h.status, sizeof(int));
  DA(h.stats, sizeof(long long) * 4);
  DA(h.result, sizeof(double) * 4);
  DA(c->d_energy_tmp, sizeof(double));
  h.ls_end = h.L + 1;
  for (int l = h.lmin; l <= h.L; l++)
    if (h.lev_n[l] > 4) {
      h.ls_end = l;
      break;
    }
  h.nsmall = h.lev_off[h.ls_end > h.L ? h.L : h.ls_end] + (h.ls_end > h.L ? h.lev_n[h.L] * h.lev_n[h.L] * h.lev_n[h.L] : 0);
  if (h.ls_end <= h.lmin) h.nsmall = 0;
  DA(h.dsmall, sizeof(double) * 4 * (size_t)std::max(1, h.nsmall) * C);
  DA(h.sync, sizeof(unsigned long long) * 128);
  DA(h.dacc, sizeof(double) * 8 * (size_t)(levels - h.lmin + 1) * MC_DSLOTS * C);
  DA(h.dKpre, sizeof(double) * 4 * C);
  DCK(cudaMemsetAsync(h.dsmall, 0, sizeof(double) * 4 * (size_t)std::max(1, h.nsmall) * C, c->stream));
  DCK(cudaMemsetAsync(h.Khat, 0, sizeof(double) * C, c->stream));
  DCK(cudaMemsetAsync(h.Hhat, 0, sizeof(double) * C, c->stream));
  DCK(cudaMemsetAsync(h.G, 0, sizeof(double) * (size_t)C * C, c->stream));
  DCK(cudaMemsetAsync(h.dipv, 0, sizeof(double) * 3, c->stream));
  DCK(cudaMemsetAsync(h.energy, 0, sizeof(double), c->stream));
  DCK(cudaMemsetAsync(h.status, 0, sizeof(int), c->stream));
  DCK(cudaMemsetAsync(h.stats, 0, sizeof(long long) * 4, c->stream));
  DCK(cudaMemsetAsync(h.partials, 0, sizeof(double) * 4 * MC_MAX_ITEMS, c->stream));

  // setup scratch: chunk partials of the gather (bounded), K chunks, energy
  size_t need = 0;
  for (int l = h.lmin; l <= levels; l++) {
    const size_t ncl = (size_t)h.lev_n[l] * h.lev_n[l] * h.lev_n[l];
    const int nchunk = chunks_for_level(h, c->sms, l, kScratchCap);
    if (nchunk > 1) need = std::max(need, ncl * nchunk * C);
    // offset chunks of the fast setup's multipole-to-local pass
    const size_t nco = (size_t)m2l_offset_chunks(h.lev_n[l], c->sms);
    if (nco > 1) need = std::max(need, std::min(ncl * nco * C, kScratchCap));
  }
  need = std::max(need, (size_t)1024 * (C + 3));
  need = std::max(need, (size_t)c->sms * 2 * MC_WARPS);
  c->scratch_doubles = need;
  DA(c->d_scratch, sizeof(double) * need);

  if (bc == MC_BC_PBC) {
    const double* d_st = nullptr;
    rc = lattice_table(c->dev, 2 * p, c->stream, &d_st);
    if (rc != MC_OK) {
      mc_destroy(c);
      return rc;
    }
    k_far_operator<<<grid_for(c->sms, (size_t)C * C, 256), 256, 0, c->stream>>>(p, box, d_st, h.G);
    DCK(cudaGetLastError());
  }
  if (mc_chain_max_ctas(precision) < 1) {
    mc_destroy(c);
    return MC_ERR_CUDA;
  }
  // default schedule by precision (measured on GB300: the barrier-free chain
  // is 8-30 % faster in FP64 over N = 1e3..1e6; in FP32-eval the phased one
  // is as fast or faster)
  c->schedule = precision == MC_FP64 ? MC_SCHEDULE_ASYNC : MC_SCHEDULE_PHASED;
  h.near_parts = near_parts_auto(h);
  DA(c->d_sys, sizeof(McSys));
  DCK(cudaMemcpyAsync(c->d_sys, &h, sizeof(McSys), cudaMemcpyHostToDevice, c->stream));
  DCK(cudaStreamSynchronize(c->stream));
  *out = c;
  return MC_OK;
#undef DA
#undef DCK
}

int mc_setup(mc_ctx* c, int mode) {
  if (!c || (mode != MC_SETUP_P2L && mode != MC_SETUP_FMM && mode != MC_SETUP_MULTIPOLE))
    return MC_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  int rc;
  if (mode == MC_SETUP_MULTIPOLE) {
    rc = run_setup_mm(c);
  } else {
    rc = set_method(c, 0);
    if (rc == MC_OK) rc = mode == MC_SETUP_FMM ? run_setup_fmm(c) : run_setup(c);
  }
  if (rc != MC_OK) return rc;
  rc = energy_into(c, c->h.energy);
  if (rc != MC_OK) return rc;
  CK(cudaStreamSynchronize(c->stream));
  c->setup_done = 1;
  return MC_OK;
}

int mc_propose(mc_ctx* c, int64_t j, const double r_new[3], double* dE_out) {
  if (!c || !r_new || !dE_out || j < 0 || j >= c->h.n) return MC_ERR_ARG;
  if (!c->setup_done) return MC_ERR_STATE;
  if (!in_box(r_new, c->h.a)) return MC_ERR_OUTSIDE;
  CK(cudaSetDevice(c->dev));
  RunParams rp{};
  memset(&rp, 0, sizeof(rp));
  rp.mode = 1;
  rp.nsteps = 1;
  rp.jg = j;
  rp.rx = r_new[0];
  rp.ry = r_new[1];
  rp.rz = r_new[2];
  int rc = launch_chain(c, rp);
  if (rc != MC_OK) return rc;
  rc = sync_status(c);
  if (rc != MC_OK) return rc;
  CK(cudaMemcpy(dE_out, c->h.result, sizeof(double), cudaMemcpyDeviceToHost));
  return MC_OK;
}

int mc_accept(mc_ctx* c, int64_t j, const double r_new[3], const double* dE_or_null) {
  if (!c || !r_new || j < 0 || j >= c->h.n) return MC_ERR_ARG;
  if (!c->setup_done) return MC_ERR_STATE;
  if (!in_box(r_new, c->h.a)) return MC_ERR_OUTSIDE;
  CK(cudaSetDevice(c->dev));
  RunParams rp{};
  memset(&rp, 0, sizeof(rp));
  rp.mode = 2;
  rp.nsteps = 1;
  rp.jg = j;
  rp.rx = r_new[0];
  rp.ry = r_new[1];
  rp.rz = r_new[2];
  rp.has_dE = dE_or_null ? 1 : 0;
  rp.dEg = dE_or_null ? *dE_or_null : 0.0;
  int rc = launch_chain(c, rp);
  if (rc != MC_OK) return rc;
  return sync_status(c);
}

int mc_run(mc_ctx* c, int64_t n_steps, uint64_t seed, double beta, double half_width,
           int64_t resetup_every, mc_stats* stats, int64_t* log_j, double* log_dE, uint8_t* log_acc) {
  if (!c || n_steps < 0 || !(half_width >= 0.0) || !isfinite(beta) || resetup_every < 0)
    return MC_ERR_ARG;
  if ((log_j || log_dE || log_acc) && !(log_j && log_dE && log_acc)) return MC_ERR_ARG;
  if (!c->setup_done) return MC_ERR_STATE;
  CK(cudaSetDevice(c->dev));
  const bool logging = log_j != nullptr;
  long long *d_lj = nullptr;
  double* d_ld = nullptr;
  unsigned char* d_la = nullptr;
  if (logging && n_steps > 0) {
    if (cudaMalloc(&d_lj, sizeof(long long) * n_steps) != cudaSuccess ||
        cudaMalloc(&d_ld, sizeof(double) * n_steps) != cudaSuccess ||
        cudaMalloc(&d_la, n_steps) != cudaSuccess) {
      cudaFree(d_lj);
      cudaFree(d_ld);
      cudaFree(d_la);
      return MC_ERR_NOMEM;
    }
  }
  mc_stats st;
  memset(&st, 0, sizeof(st));
  const bool sync = stats || logging || resetup_every > 0;
  long long done = 0;
  int rc = MC_OK;
  while (done < n_steps || n_steps == 0) {
    RunParams rp{};
    memset(&rp, 0, sizeof(rp));
    rp.mode = 0;
    rp.step0 = c->steps_total;
    rp.nsteps = n_steps - done;
    rp.seed = seed;
    rp.beta = beta;
    rp.h = half_width;
    rp.stop_after_accepts = resetup_every;
    if (logging) {
      rp.log_j = d_lj + done;
      rp.log_dE = d_ld + done;
      rp.log_acc = d_la + done;
    }
    if (n_steps == 0) break;
    rc = launch_chain(c, rp);
    if (rc != MC_OK) break;
    if (!sync) {
      c->steps_total += n_steps;
      return MC_OK;
    }
    rc = sync_status(c);
    if (rc != MC_OK) break;
    long long hs[4];
    if (cudaMemcpy(hs, c->h.stats, sizeof(hs), cudaMemcpyDeviceToHost) != cudaSuccess) {
      rc = MC_ERR_CUDA;
      break;
    }
    done += hs[0];
    c->steps_total += hs[0];
    st.steps += hs[0];
    st.accepted += hs[1];
    st.borderline += hs[2];
    if (resetup_every > 0 && done < n_steps) {
      // full FP64 re-setup from the current positions; drift = running - fresh
      double run_e = 0.0, fresh = 0.0;
      if ((rc = c->h.method ? run_setup_mm(c) : run_setup(c)) != MC_OK) break;
      if ((rc = energy_into(c, c->d_energy_tmp)) != MC_OK) break;
      if (cudaMemcpyAsync(&run_e, c->h.energy, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaMemcpyAsync(&fresh, c->d_energy_tmp, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        rc = MC_ERR_CUDA;
        break;
      }
      st.max_drift = std::max(st.max_drift, fabs(run_e - fresh));
      st.sum_drift += run_e - fresh;
      st.sum_abs_drift += fabs(run_e - fresh);
      st.resetups++;
      if (cudaMemcpy(c->h.energy, &fresh, sizeof(double), cudaMemcpyHostToDevice) != cudaSuccess) {
        rc = MC_ERR_CUDA;
        break;
      }
    }
  }
  if (rc == MC_OK && logging && n_steps > 0) {
    std::vector<long long> tmp(n_steps);
    if (cudaMemcpy(tmp.data(), d_lj, sizeof(long long) * n_steps, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(log_dE, d_ld, sizeof(double) * n_steps, cudaMemcpyDeviceToHost) != cudaSuccess ||
        cudaMemcpy(log_acc, d_la, n_steps, cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = MC_ERR_CUDA;
    for (int64_t i = 0; i < n_steps; i++) log_j[i] = tmp[i];
  }
  if (logging) {
    cudaFree(d_lj);
    cudaFree(d_ld);
    cudaFree(d_la);
  }
  if (rc == MC_OK && stats) {
    if (cudaMemcpy(&st.energy, c->h.energy, sizeof(double), cudaMemcpyDeviceToHost) != cudaSuccess)
      return MC_ERR_CUDA;
    *stats = st;
  }
  return rc;
}

int mc_step_counter(mc_ctx* c, int64_t* out) {
  if (!c || !out) return MC_ERR_ARG;
  *out = (int64_t)c->steps_total;
  return MC_OK;
}

int mc_energy(mc_ctx* c, double* e) {
  if (!c || !e) return MC_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(e, c->h.energy, sizeof(double), cudaMemcpyDeviceToHost));
  return MC_OK;
}

int mc_energy_fresh(mc_ctx* c, double* e) {
  if (!c || !e) return MC_ERR_ARG;
  if (!c->setup_done) return MC_ERR_STATE;
  CK(cudaSetDevice(c->dev));
  int rc = energy_into(c, c->d_energy_tmp);
  if (rc != MC_OK) return rc;
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(e, c->d_energy_tmp, sizeof(double), cudaMemcpyDeviceToHost));
  return MC_OK;
}

int mc_get_positions(mc_ctx* c, double* pos_out) {
  if (!c || !pos_out) return MC_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  std::vector<double4> hp(c->h.n);
  CK(cudaMemcpy(hp.data(), c->h.ppos, sizeof(double4) * c->h.n, cudaMemcpyDeviceToHost));
  for (int i = 0; i < c->h.n; i++) {
    pos_out[3 * i] = hp[i].x;
    pos_out[3 * i + 1] = hp[i].y;
    pos_out[3 * i + 2] = hp[i].z;
  }
  return MC_OK;
}

int mc_get_local(mc_ctx* c, int level, double* out) {
  if (!c || !out) return MC_ERR_ARG;
  if (level < 2 || level > c->h.L) return MC_ERR_LEVELS;
  if (c->h.method != 0) return MC_ERR_STATE;  // the multipole method keeps no locals
  const int nl = c->h.lev_n[level], C = c->h.C;
  const size_t cnt = (size_t)nl * nl * nl * C;
  if (level < c->h.lmin) {  // free space: the interaction lists of level 2 are empty
    memset(out, 0, sizeof(double) * cnt);
    return MC_OK;
  }
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(out, c->h.Lhat + (size_t)c->h.lev_off[level] * C, sizeof(double) * cnt,
                cudaMemcpyDeviceToHost));
  std::vector<double> inv(C);
  for (int k = 0; k < C; k++) inv[k] = 1.0 / scale_of(k);
  for (size_t i = 0; i < cnt; i++) out[i] *= inv[i % C];
  return MC_OK;
}

int mc_set_lj(mc_ctx* c, double eps, double sigma, double cutoff) {
  if (!c || !(eps >= 0.0) || !(sigma > 0.0) || !(cutoff > 0.0)) return MC_ERR_ARG;
  if (cutoff > c->h.lev_w[c->h.L]) return MC_ERR_ARG;  // pairs in range must be near-cell pairs
  CK(cudaSetDevice(c->dev));
  const double s6 = pow(sigma, 6.0);
  c->h.lj_on = eps > 0.0 ? 1 : 0;
  c->h.lj_eps4 = 4.0 * eps;
  c->h.lj_s6 = s6;
  c->h.lj_s12 = s6 * s6;
  c->h.lj_rc2 = cutoff * cutoff;
  CK(cudaMemcpyAsync(c->d_sys, &c->h, sizeof(McSys), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  c->setup_done = 0;  // the energy changes: set up again
  return MC_OK;
}

int mc_set_near_parts(mc_ctx* c, int parts, int* used_out) {
  if (!c || parts < 0 || parts > MC_NEAR_PARTS_MAX) return MC_ERR_ARG;
  const int P = parts == 0 ? near_parts_auto(c->h) : parts;
  if (!near_parts_fit(c->h, P)) return MC_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  c->h.near_parts = P;
  CK(cudaMemcpyAsync(c->d_sys, &c->h, sizeof(McSys), cudaMemcpyHostToDevice, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (used_out) *used_out = P;
  return MC_OK;
}

int mc_get_multipole(mc_ctx* c, int level, double* out) {
  if (!c || !out) return MC_ERR_ARG;
  if (level < 2 || level > c->h.L) return MC_ERR_LEVELS;
  if (c->h.method != 1 || !c->d_mpole) return MC_ERR_STATE;
  const int nl = c->h.lev_n[level], C = c->h.C;
  const size_t cnt = (size_t)nl * nl * nl * C;
  if (level < c->h.lmin) {
    memset(out, 0, sizeof(double) * cnt);
    return MC_OK;
  }
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(out, c->d_mpole + (size_t)c->h.lev_off[level] * C, sizeof(double) * cnt,
                cudaMemcpyDeviceToHost));
  std::vector<double> sc(C);
  for (int k = 0; k < C; k++) sc[k] = scale_of(k);
  for (size_t i = 0; i < cnt; i++) out[i] *= sc[i % C];
  return MC_OK;
}

int mc_get_far(mc_ctx* c, double* K, double* H) {
  if (!c || !K || !H) return MC_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  const int C = c->h.C;
  CK(cudaMemcpy(K, c->h.Khat, sizeof(double) * C, cudaMemcpyDeviceToHost));
  CK(cudaMemcpy(H, c->h.Hhat, sizeof(double) * C, cudaMemcpyDeviceToHost));
  for (int k = 0; k < C; k++) {
    const double s = scale_of(k);
    K[k] *= s;
    H[k] /= s;
  }
  if (c->h.bc != MC_BC_PBC)
    for (int k = 0; k < C; k++) K[k] = H[k] = 0.0;
  return MC_OK;
}

int mc_lattice_sums(int lmax, double* out) {
  if (!out || lmax < 0 || lmax > 2 * MC_PMAX) return MC_ERR_ARG;
  const int n = (lmax + 1) * (lmax + 1);
  double* d = nullptr;
  if (cudaMalloc(&d, sizeof(double) * 2 * n) != cudaSuccess) return MC_ERR_NOMEM;
  k_lattice_sums<<<(lmax + 1) * (lmax + 2) / 2, 256>>>(lmax, d);
  cudaError_t e = cudaMemcpy(out, d, sizeof(double) * 2 * n, cudaMemcpyDeviceToHost);
  cudaFree(d);
  if (e != cudaSuccess) return MC_ERR_CUDA;
  // device sums are of the scaled harmonics; divide by s_l,mu for S_l^mu
  for (int l = 0; l <= lmax; l++)
    for (int m = -l; m <= l; m++) {
      const double s = sqrt(fact(l - abs(m)) * fact(l + abs(m)));
      out[2 * (l * l + l + m)] /= s;
      out[2 * (l * l + l + m) + 1] /= s;
    }
  return MC_OK;
}

int mc_profile(mc_ctx* c, int on) {
  if (!c) return MC_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  if (on && !c->d_prof) {
    if (dalloc(c, (void**)&c->d_prof, MC_PROF_COUNTERS * sizeof(unsigned long long)) != MC_OK) return MC_ERR_NOMEM;
    CK(cudaMemset(c->d_prof, 0, MC_PROF_COUNTERS * sizeof(unsigned long long)));
  } else if (!on) {
    c->d_prof = nullptr;  // the buffer stays owned by the context
  }
  return MC_OK;
}

int mc_profile_read(mc_ctx* c, uint64_t* out) {
  if (!c || !out) return MC_ERR_ARG;
  if (!c->d_prof) return MC_ERR_STATE;
  CK(cudaSetDevice(c->dev));
  CK(cudaStreamSynchronize(c->stream));
  CK(cudaMemcpy(out, c->d_prof, MC_PROF_COUNTERS * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  CK(cudaMemset(c->d_prof, 0, MC_PROF_COUNTERS * sizeof(unsigned long long)));
  return MC_OK;
}

int mc_set_schedule(mc_ctx* c, int schedule) {
  if (!c || (schedule != MC_SCHEDULE_PHASED && schedule != MC_SCHEDULE_PLAIN &&
             schedule != MC_SCHEDULE_ASYNC))
    return MC_ERR_ARG;
  c->schedule = schedule;
  return MC_OK;
}

int mc_set_ctas(mc_ctx* c, int n_cta) {
  if (!c || n_cta < 0 || n_cta > c->sms) return MC_ERR_ARG;
  c->nCTA = n_cta;
  return MC_OK;
}

int mc_status(mc_ctx* c) {
  if (!c) return MC_ERR_ARG;
  return sync_status(c);
}

int mc_set_wait_limit(mc_ctx* c, int64_t ns) {
  if (!c || ns < 0) return MC_ERR_ARG;
  c->wait_ns = ns;
  return MC_OK;
}

int mc_inject_wait_fault(mc_ctx* c, int missing_arrivals) {
  if (!c || missing_arrivals < 0 || missing_arrivals > 1024) return MC_ERR_ARG;
  c->bar_missing = (unsigned)missing_arrivals;
  return MC_OK;
}

}  // extern "C"

// ------------------------------------------------------------------ batches
struct mc_batch {
  int n;
  std::vector<mc_ctx*> ctxs;
  int prec, dev, sms;
  cudaStream_t stream;
  std::vector<int> ctas;  // CTAs per chain
  int nf_cols;
  int schedule;
  // device copies
  const McSys** d_systems;
  RunParams* d_rps;
  int *d_cta_chain, *d_cta_rank, *d_chain_ctas;
  int nCTA;
  // graph cache
  cudaGraphExec_t gexec;
  long long g_steps;
  double g_beta, g_h;
  int g_valid;
  std::vector<uint64_t> seeds;
  int seeds_valid;
};

namespace {

int batch_upload_map(mc_batch* b) {
  std::vector<int> cchain, crank;
  for (int i = 0; i < b->n; i++)
    for (int r = 0; r < b->ctas[i]; r++) {
      cchain.push_back(i);
      crank.push_back(r);
    }
  b->nCTA = (int)cchain.size();
  if (b->nCTA > b->sms) return MC_ERR_ARG;
  CK(cudaMemcpy(b->d_cta_chain, cchain.data(), sizeof(int) * b->nCTA, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->d_cta_rank, crank.data(), sizeof(int) * b->nCTA, cudaMemcpyHostToDevice));
  CK(cudaMemcpy(b->d_chain_ctas, b->ctas.data(), sizeof(int) * b->n, cudaMemcpyHostToDevice));
  if (b->g_valid) {
    cudaGraphExecDestroy(b->gexec);
    b->g_valid = 0;
  }
  return MC_OK;
}

// split `total` CTAs: one each, the rest by largest remainder of the weights
std::vector<int> split_by_weight(const std::vector<double>& w, int total) {
  const int n = (int)w.size();
  std::vector<int> out(n, 1);
  int left = total - n;
  double sw = 0.0;
  for (double x : w) sw += x;
  if (left <= 0 || sw <= 0.0) return out;
  std::vector<std::pair<double, int>> rem;
  int used = 0;
  for (int i = 0; i < n; i++) {
    const double share = w[i] / sw * left;
    const int fl = (int)floor(share);
    out[i] += fl;
    used += fl;
    rem.push_back({share - fl, i});
  }
  std::sort(rem.begin(), rem.end(), [](const std::pair<double, int>& x, const std::pair<double, int>& y) {
    return x.first > y.first || (x.first == y.first && x.second < y.second);
  });
  for (int k = 0; k < left - used && k < n; k++) out[rem[k].second]++;
  return out;
}

int batch_set_params(mc_batch* b, long long n_steps, const uint64_t* seeds, double beta, double h,
                     long long* const* logj, double* const* logd, unsigned char* const* loga) {
  std::vector<RunParams> rps(b->n);
  // current step counters live on the device (advanced by the kernel)
  std::vector<RunParams> cur(b->n);
  CK(cudaMemcpy(cur.data(), b->d_rps, sizeof(RunParams) * b->n, cudaMemcpyDeviceToHost));
  for (int i = 0; i < b->n; i++) {
    RunParams& rp = rps[i];
    memset(&rp, 0, sizeof(rp));
    rp.mode = 0;
    rp.step0 = cur[i].step0;
    rp.nsteps = n_steps;
    rp.seed = seeds[i];
    rp.beta = beta;
    rp.h = h;
    rp.wait_ns = b->ctxs[i]->wait_ns;
    rp.bar_missing = 0u;
    rp.spec = (b->ctxs[i]->h.method == 0 && b->schedule == MC_SCHEDULE_PHASED) ? 1 : 0;
    rp.nf_cols = b->nf_cols;
    rp.chain = (unsigned)i;
    if (logj) {
      rp.log_j = logj[i];
      rp.log_dE = logd[i];
      rp.log_acc = loga[i];
    }
  }
  CK(cudaMemcpy(b->d_rps, rps.data(), sizeof(RunParams) * b->n, cudaMemcpyHostToDevice));
  return MC_OK;
}

int batch_enqueue(mc_batch* b) {
  for (int i = 0; i < b->n; i++) {
    CK(cudaMemsetAsync(b->ctxs[i]->h.bar, 0, sizeof(unsigned long long), b->stream));
    CK(cudaMemsetAsync(b->ctxs[i]->h.status, 0, sizeof(int), b->stream));
    CK(cudaMemsetAsync(b->ctxs[i]->h.sync, 0, sizeof(unsigned long long) * 16, b->stream));
    CK(cudaMemsetAsync(b->ctxs[i]->h.dsmall, 0,
                       sizeof(double) * 3 * (size_t)b->ctxs[i]->h.nsmall * b->ctxs[i]->h.C, b->stream));
  }
  {
    // phased FP64: the column-scaled contributions (fewer FP64 instructions
    // for this throughput-bound form)
    const int var = b->ctxs[0]->h.method == 1 ? MC_VAR_MM
                    : b->schedule == MC_SCHEDULE_PHASED ? (b->prec == MC_FP64 ? MC_VAR_SPECW : MC_VAR_SPEC)
                                                       : MC_VAR_PLAIN;
    CK(mc_launch_batch(b->d_systems, b->d_rps, b->d_cta_chain, b->d_cta_rank, b->d_chain_ctas,
                       b->prec, var, b->nCTA, b->stream));
  }
  return MC_OK;
}

int batch_collect(mc_batch* b, mc_stats* stats, std::vector<long long>* ns) {
  CK(cudaStreamSynchronize(b->stream));
  int worst = MC_OK;
  for (int i = 0; i < b->n; i++) {
    int st = 0;
    long long hs[4];
    CK(cudaMemcpy(&st, b->ctxs[i]->h.status, sizeof(int), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(hs, b->ctxs[i]->h.stats, sizeof(hs), cudaMemcpyDeviceToHost));
    if (st != MC_OK) worst = st;
    b->ctxs[i]->steps_total += hs[0];
    if (stats) {
      memset(&stats[i], 0, sizeof(mc_stats));
      stats[i].steps = hs[0];
      stats[i].accepted = hs[1];
      stats[i].borderline = hs[2];
      CK(cudaMemcpy(&stats[i].energy, b->ctxs[i]->h.energy, sizeof(double), cudaMemcpyDeviceToHost));
    }
    if (ns) (*ns)[i] = hs[3];
  }
  return worst;
}

}  // namespace

extern "C" {

int mc_batch_create(mc_batch** out, int n_chains, mc_ctx* const* ctxs) {
  if (!out || n_chains < 1 || !ctxs) return MC_ERR_ARG;
  *out = nullptr;
  for (int i = 0; i < n_chains; i++) {
    if (!ctxs[i]) return MC_ERR_ARG;
    if (!ctxs[i]->setup_done) return MC_ERR_STATE;
    if (ctxs[i]->h.prec != ctxs[0]->h.prec || ctxs[i]->dev != ctxs[0]->dev ||
        ctxs[i]->h.method != ctxs[0]->h.method)
      return MC_ERR_ARG;
    for (int k = 0; k < i; k++)
      if (ctxs[k] == ctxs[i]) return MC_ERR_ARG;
  }
  mc_batch* b = new mc_batch();
  b->n = n_chains;
  b->ctxs.assign(ctxs, ctxs + n_chains);
  b->prec = ctxs[0]->h.prec;
  b->dev = ctxs[0]->dev;
  b->stream = ctxs[0]->stream;
  if (cudaSetDevice(b->dev) != cudaSuccess) {
    delete b;
    return MC_ERR_CUDA;
  }
  {
    // the batch's CTAs: its kernels' occupancy
    b->sms = mc_batch_max_ctas(b->prec);
  }
  if (b->sms < 1) {
    delete b;
    return MC_ERR_CUDA;
  }
  if (n_chains > b->sms) {
    delete b;
    return MC_ERR_ARG;  // every chain needs at least one CTA
  }
  b->nf_cols = 4;
  // measured on GB300 (64 chains, p = 10): speculation pays in FP64, where
  // each item is long, and costs in the FP32-eval form
  b->schedule = b->prec == MC_FP64 ? MC_SCHEDULE_PHASED : MC_SCHEDULE_PLAIN;
  std::vector<double> w(n_chains);
  for (int i = 0; i < n_chains; i++) w[i] = (double)(ctxs[i]->h.L - ctxs[i]->h.lmin + 1);
  b->ctas = split_by_weight(w, b->sms);
  bool ok = cudaMalloc((void**)&b->d_systems, sizeof(McSys*) * n_chains) == cudaSuccess &&
            cudaMalloc((void**)&b->d_rps, sizeof(RunParams) * n_chains) == cudaSuccess &&
            cudaMalloc((void**)&b->d_cta_chain, sizeof(int) * b->sms) == cudaSuccess &&
            cudaMalloc((void**)&b->d_cta_rank, sizeof(int) * b->sms) == cudaSuccess &&
            cudaMalloc((void**)&b->d_chain_ctas, sizeof(int) * n_chains) == cudaSuccess;
  if (!ok) {
    mc_batch_destroy(b);
    return MC_ERR_NOMEM;
  }
  std::vector<const McSys*> sp(n_chains);
  std::vector<RunParams> rp(n_chains);
  for (int i = 0; i < n_chains; i++) {
    sp[i] = ctxs[i]->d_sys;
    memset(&rp[i], 0, sizeof(RunParams));
    rp[i].step0 = ctxs[i]->steps_total;
  }
  if (cudaMemcpy(b->d_systems, sp.data(), sizeof(McSys*) * n_chains, cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(b->d_rps, rp.data(), sizeof(RunParams) * n_chains, cudaMemcpyHostToDevice) != cudaSuccess) {
    mc_batch_destroy(b);
    return MC_ERR_CUDA;
  }
  int rc = batch_upload_map(b);
  if (rc != MC_OK) {
    mc_batch_destroy(b);
    return rc;
  }
  *out = b;
  return MC_OK;
}

void mc_batch_destroy(mc_batch* b) {
  if (!b) return;
  cudaSetDevice(b->dev);
  cudaStreamSynchronize(b->stream);
  if (b->g_valid) cudaGraphExecDestroy(b->gexec);
  cudaFree(b->d_systems);
  cudaFree(b->d_rps);
  cudaFree(b->d_cta_chain);
  cudaFree(b->d_cta_rank);
  cudaFree(b->d_chain_ctas);
  delete b;
}

int mc_batch_set_schedule(mc_batch* b, int schedule) {
  if (!b || (schedule != MC_SCHEDULE_PHASED && schedule != MC_SCHEDULE_PLAIN))
    return MC_ERR_ARG;
  b->schedule = schedule;
  if (b->g_valid) {
    cudaGraphExecDestroy(b->gexec);
    b->g_valid = 0;
  }
  return MC_OK;
}

int mc_batch_info(mc_batch* b, int* ctas_out, int* nf_cols_out) {
  if (!b) return MC_ERR_ARG;
  if (ctas_out)
    for (int i = 0; i < b->n; i++) ctas_out[i] = b->ctas[i];
  if (nf_cols_out) *nf_cols_out = b->nf_cols;
  return MC_OK;
}

int mc_batch_run(mc_batch* b, int64_t n_steps, const uint64_t* seeds, double beta, double half_width,
                 mc_stats* stats, int64_t* log_j, double* log_dE, uint8_t* log_acc) {
  if (!b || !seeds || n_steps < 0 || !(half_width >= 0.0) || !isfinite(beta)) return MC_ERR_ARG;
  if ((log_j || log_dE || log_acc) && !(log_j && log_dE && log_acc)) return MC_ERR_ARG;
  if (n_steps == 0) return MC_OK;
  CK(cudaSetDevice(b->dev));
  const bool logging = log_j != nullptr;
  int rc = MC_OK;
  if (logging) {
    const size_t tot = (size_t)b->n * n_steps;
    long long* dj = nullptr;
    double* dd = nullptr;
    unsigned char* da = nullptr;
    if (cudaMalloc(&dj, sizeof(long long) * tot) != cudaSuccess ||
        cudaMalloc(&dd, sizeof(double) * tot) != cudaSuccess || cudaMalloc(&da, tot) != cudaSuccess) {
      cudaFree(dj);
      cudaFree(dd);
      cudaFree(da);
      return MC_ERR_NOMEM;
    }
    std::vector<long long*> pj(b->n);
    std::vector<double*> pd(b->n);
    std::vector<unsigned char*> pa(b->n);
    for (int i = 0; i < b->n; i++) {
      pj[i] = dj + (size_t)i * n_steps;
      pd[i] = dd + (size_t)i * n_steps;
      pa[i] = da + (size_t)i * n_steps;
    }
    rc = batch_set_params(b, n_steps, seeds, beta, half_width, pj.data(), pd.data(), pa.data());
    if (rc == MC_OK) rc = batch_enqueue(b);
    if (rc == MC_OK) rc = batch_collect(b, stats, nullptr);
    if (rc == MC_OK) {
      std::vector<long long> tj(tot);
      if (cudaMemcpy(tj.data(), dj, sizeof(long long) * tot, cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(log_dE, dd, sizeof(double) * tot, cudaMemcpyDeviceToHost) != cudaSuccess ||
          cudaMemcpy(log_acc, da, tot, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = MC_ERR_CUDA;
      for (size_t k = 0; k < tot; k++) log_j[k] = tj[k];
    }
    cudaFree(dj);
    cudaFree(dd);
    cudaFree(da);
    b->seeds_valid = 0;
    return rc;
  }
  // graph path: parameters live in device memory, the step counters advance there
  const bool same_seeds =
      b->seeds_valid && std::equal(b->seeds.begin(), b->seeds.end(), seeds);
  if (!(b->g_valid && b->g_steps == n_steps && b->g_beta == beta && b->g_h == half_width &&
        same_seeds)) {
    rc = batch_set_params(b, n_steps, seeds, beta, half_width, nullptr, nullptr, nullptr);
    if (rc != MC_OK) return rc;
    b->seeds.assign(seeds, seeds + b->n);
    b->seeds_valid = 1;
    if (b->g_valid) {
      cudaGraphExecDestroy(b->gexec);
      b->g_valid = 0;
    }
    cudaStream_t cs = b->stream;
    bool own = false;
    if (!cs) {
      // legacy stream cannot be captured: capture on a private stream
      CK(cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking));
      own = true;
    }
    cudaStream_t saved = b->stream;
    b->stream = cs;
    cudaGraph_t graph;
    if (cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      b->stream = saved;
      if (own) cudaStreamDestroy(cs);
      return MC_ERR_CUDA;
    }
    rc = batch_enqueue(b);
    cudaError_t e = cudaStreamEndCapture(cs, &graph);
    b->stream = saved;
    if (own) cudaStreamDestroy(cs);
    if (rc != MC_OK || e != cudaSuccess) return MC_ERR_CUDA;
    e = cudaGraphInstantiate(&b->gexec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return MC_ERR_CUDA;
    b->g_valid = 1;
    b->g_steps = n_steps;
    b->g_beta = beta;
    b->g_h = half_width;
  }
  CK(cudaGraphLaunch(b->gexec, b->stream));
  if (!stats) {
    for (int i = 0; i < b->n; i++) b->ctxs[i]->steps_total += n_steps;
    return MC_OK;
  }
  return batch_collect(b, stats, nullptr);
}

int mc_batch_tune(mc_batch* b, int64_t trial_steps, double beta, double half_width) {
  if (!b || trial_steps < 1) return MC_ERR_ARG;
  CK(cudaSetDevice(b->dev));
  std::vector<uint64_t> seeds(b->n);
  for (int i = 0; i < b->n; i++) seeds[i] = 0x5EEDULL + i;
  std::vector<long long> ns(b->n);
  // time per proposal of every chain at 1 and 2 CTAs per chain
  std::vector<double> t1(b->n), t2(b->n);
  const int saved_nf = b->nf_cols;
  for (int g = 1; g <= 2; g++) {
    if (b->n * g > b->sms) {
      // not enough SMs for a uniform g: reuse g = 1
      for (int i = 0; i < b->n; i++) t2[i] = t1[i];
      break;
    }
    b->ctas.assign(b->n, g);
    int rc = batch_upload_map(b);
    if (rc != MC_OK) return rc;
    rc = batch_set_params(b, trial_steps, seeds.data(), beta, half_width, nullptr, nullptr, nullptr);
    if (rc == MC_OK) rc = batch_enqueue(b);
    if (rc == MC_OK) rc = batch_collect(b, nullptr, &ns);
    if (rc != MC_OK) return rc;
    for (int i = 0; i < b->n; i++) (g == 1 ? t1 : t2)[i] = (double)ns[i] / (double)trial_steps;
  }
  // model t(g) = a + b/g from the two points; greedy: give the next CTA to
  // the chain with the largest predicted time
  std::vector<double> A(b->n), B(b->n);
  for (int i = 0; i < b->n; i++) {
    B[i] = std::max(0.0, 2.0 * (t1[i] - t2[i]));
    A[i] = std::max(0.0, t1[i] - B[i]);
  }
  std::vector<int> g(b->n, 1);
  for (int left = b->sms - b->n; left > 0; left--) {
    int worst = 0;
    double wt = -1.0;
    for (int i = 0; i < b->n; i++) {
      const double ti = A[i] + B[i] / g[i];
      if (ti > wt) {
        wt = ti;
        worst = i;
      }
    }
    g[worst]++;
  }
  b->ctas = g;
  int rc = batch_upload_map(b);
  if (rc != MC_OK) return rc;
  // far-field tiles: pick the count with the shortest slowest chain
  int best_nf = saved_nf;
  double best = 1e300;
  for (int nf : {1, 2, 4, 8, 16}) {
    b->nf_cols = nf;
    rc = batch_set_params(b, trial_steps, seeds.data(), beta, half_width, nullptr, nullptr, nullptr);
    if (rc == MC_OK) rc = batch_enqueue(b);
    if (rc == MC_OK) rc = batch_collect(b, nullptr, &ns);
    if (rc != MC_OK) return rc;
    const double mk = (double)*std::max_element(ns.begin(), ns.end());
    if (mk < best) {
      best = mk;
      best_nf = nf;
    }
  }
  b->nf_cols = best_nf;
  b->seeds_valid = 0;
  if (b->g_valid) {
    cudaGraphExecDestroy(b->gexec);
    b->g_valid = 0;
  }
  return MC_OK;
}

}  // extern "C"
