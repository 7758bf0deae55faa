// C-ABI entry points of the GB300 multilevel Monte Carlo electrostatics
// library (declared in include/mcfmm.h).  Host code only: argument checks,
// device memory ownership, kernel launches and copies.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <vector>

#include "../../include/mcfmm.h"
#include "mc_dev.cuh"

// kernels defined in the other translation units
cudaError_t mc_launch_chain(const McSys* d_sys, const RunParams& rp, int prec, int nCTA,
                            cudaStream_t stream);
int mc_chain_max_ctas(int prec);
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

struct mc_ctx {
  McSys h;        // host copy holding device pointers
  McSys* d_sys;   // device copy
  cudaStream_t stream;
  int dev;
  int nCTA;
  int sms;
  int setup_done;
  long long steps_total;
  long long wait_ns;
  double* d_scratch;
  size_t scratch_doubles;
  double* d_energy_tmp;  // fresh-energy target
  unsigned long long* d_prof;  // 32 timers when profiling is on, else null
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
int chunks_for_level(const McSys& h, int sms, int l, size_t max_doubles) {
  const long long ncl = (long long)h.lev_n[l] * h.lev_n[l] * h.lev_n[l];
  long long nchunk = std::min<long long>(189, std::max<long long>(1, (4LL * sms * MC_WARPS + ncl - 1) / ncl));
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
  rp.prof = c->d_prof;
  CK(cudaMemsetAsync(c->h.bar, 0, sizeof(unsigned long long), c->stream));
  CK(cudaMemsetAsync(c->h.status, 0, sizeof(int), c->stream));
  CK(mc_launch_chain(c->d_sys, rp, c->h.prec, c->nCTA, c->stream));
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

int energy_into(mc_ctx* c, double* d_dst) {
  const int blocks = c->sms * 2;
  const int nw = blocks * MC_WARPS;
  k_energy_particles<<<blocks, MC_THREADS, 0, c->stream>>>(c->d_sys, c->d_scratch);
  CK(cudaGetLastError());
  k_energy_finish<<<1, 256, 0, c->stream>>>(c->d_sys, nw, c->d_scratch, d_dst);
  CK(cudaGetLastError());
  return MC_OK;
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
  DA(h.partials, sizeof(double) * 2 * MC_MAX_ITEMS);
  DA(h.dK, sizeof(double) * 2 * C);
  DA(h.gK, sizeof(double) * 2 * MC_NF_COLS * C);
  DA(h.bar, sizeof(unsigned long long));
  DA(h.status, sizeof(int));
  DA(h.stats, sizeof(long long) * 4);
  DA(h.result, sizeof(double) * 4);
  DA(c->d_energy_tmp, sizeof(double));
  DCK(cudaMemsetAsync(h.Khat, 0, sizeof(double) * C, c->stream));
  DCK(cudaMemsetAsync(h.Hhat, 0, sizeof(double) * C, c->stream));
  DCK(cudaMemsetAsync(h.G, 0, sizeof(double) * (size_t)C * C, c->stream));
  DCK(cudaMemsetAsync(h.dipv, 0, sizeof(double) * 3, c->stream));
  DCK(cudaMemsetAsync(h.energy, 0, sizeof(double), c->stream));
  DCK(cudaMemsetAsync(h.status, 0, sizeof(int), c->stream));
  DCK(cudaMemsetAsync(h.stats, 0, sizeof(long long) * 4, c->stream));
  DCK(cudaMemsetAsync(h.partials, 0, sizeof(double) * 2 * MC_MAX_ITEMS, c->stream));

  // setup scratch: chunk partials of the gather (bounded), K chunks, energy
  size_t need = 0;
  for (int l = h.lmin; l <= levels; l++) {
    const size_t ncl = (size_t)h.lev_n[l] * h.lev_n[l] * h.lev_n[l];
    const int nchunk = chunks_for_level(h, c->sms, l, kScratchCap);
    if (nchunk > 1) need = std::max(need, ncl * nchunk * C);
  }
  need = std::max(need, (size_t)1024 * (C + 3));
  need = std::max(need, (size_t)c->sms * 2 * MC_WARPS);
  c->scratch_doubles = need;
  DA(c->d_scratch, sizeof(double) * need);

  if (bc == MC_BC_PBC) {
    const int lmax = 2 * p;
    double* d_st = nullptr;
    DA(d_st, sizeof(double) * 2 * (lmax + 1) * (lmax + 1));
    k_lattice_sums<<<(lmax + 1) * (lmax + 2) / 2, 256, 0, c->stream>>>(lmax, d_st);
    k_far_operator<<<grid_for(c->sms, (size_t)C * C, 256), 256, 0, c->stream>>>(p, box, d_st, h.G);
    DCK(cudaGetLastError());
  }
  c->nCTA = mc_chain_max_ctas(precision);
  if (c->nCTA < 1) {
    mc_destroy(c);
    return MC_ERR_CUDA;
  }
  DA(c->d_sys, sizeof(McSys));
  DCK(cudaMemcpyAsync(c->d_sys, &h, sizeof(McSys), cudaMemcpyHostToDevice, c->stream));
  DCK(cudaStreamSynchronize(c->stream));
  *out = c;
  return MC_OK;
#undef DA
#undef DCK
}

int mc_setup(mc_ctx* c, int mode) {
  if (!c || mode != MC_SETUP_P2L) return MC_ERR_ARG;
  CK(cudaSetDevice(c->dev));
  int rc = run_setup(c);
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
  RunParams rp;
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
  RunParams rp;
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
    RunParams rp;
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
      if ((rc = run_setup(c)) != MC_OK) break;
      if ((rc = energy_into(c, c->d_energy_tmp)) != MC_OK) break;
      if (cudaMemcpyAsync(&run_e, c->h.energy, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaMemcpyAsync(&fresh, c->d_energy_tmp, sizeof(double), cudaMemcpyDeviceToHost, c->stream) != cudaSuccess ||
          cudaStreamSynchronize(c->stream) != cudaSuccess) {
        rc = MC_ERR_CUDA;
        break;
      }
      st.max_drift = std::max(st.max_drift, fabs(run_e - fresh));
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
    if (dalloc(c, (void**)&c->d_prof, 32 * sizeof(unsigned long long)) != MC_OK) return MC_ERR_NOMEM;
    CK(cudaMemset(c->d_prof, 0, 32 * sizeof(unsigned long long)));
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
  CK(cudaMemcpy(out, c->d_prof, 32 * sizeof(uint64_t), cudaMemcpyDeviceToHost));
  CK(cudaMemset(c->d_prof, 0, 32 * sizeof(unsigned long long)));
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

}  // extern "C"
