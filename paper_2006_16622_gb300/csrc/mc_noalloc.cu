// Allocation-free entry point: the local expansions of one level (computed
// as the gather form of Alg. L.3 that mc_setup uses) from caller-owned device buffers, with
// the per-chunk partial expansions kept in a fixed device array that this
// file owns.  It exists for callers that must not have the library call
// cudaMalloc or cudaFree: code that manages every byte of device memory
// through its own pool or allocator, code that runs where allocation would
// synchronise the device at a bad moment, and embedders that forbid hidden
// allocations.  Nothing here allocates device or pinned host memory.
#include <cuda_runtime.h>
#include <math.h>
#include <stdint.h>

#include <mutex>

#include "../../include/mcfmm.h"
#include "mc_dev.cuh"

// The fixed scratch: MC_NOALLOC_SCRATCH_DOUBLES doubles (8 MiB) of device
// memory per GPU that loads the library, held until the process exits.  In
// host code `g_noalloc_scratch` is only a host-side stand-in for the symbol;
// its device address comes from cudaGetSymbolAddress below.
static __device__ __align__(256) double g_noalloc_scratch[MC_NOALLOC_SCRATCH_DOUBLES];

namespace {

struct NoAllocP2L {
  int L, l, p, C, bc, nL, nchunk;
  double a, w;
};

// One warp task per (target cell t of level l, chunk of t's interaction
// list); two charges per warp step (one per half-warp, lane = column m).
// Charges of finest cell c are rows [cstart[c], cstart[c+1]) of `part`
// (x, y, z, q per row).  Every task writes all C values of its partial.
__global__ void __launch_bounds__(MC_THREADS)
    k_p2l_level_noalloc(NoAllocP2L P, const double* __restrict__ part,
                        const int* __restrict__ cstart, double* __restrict__ scratch) {
  __shared__ HarmTabs<double> tabs;
  __shared__ unsigned short il[8][189];
  __shared__ double stage[MC_WARPS][256];
  harm_tabs_init<double>(&tabs);
  il_table_init(il);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, half = lane >> 4, m = lane & 15;
  const int p = P.p, C = P.C, nl = 1 << (P.l - 1), f = 1 << (P.L - P.l), nL = P.nL;
  const bool pbc = P.bc == MC_BC_PBC;
  const int ntask = nl * nl * nl * P.nchunk;
  const int per = (189 + P.nchunk - 1) / P.nchunk;
  for (int task = blockIdx.x * MC_WARPS + warp; task < ntask; task += gridDim.x * MC_WARPS) {
    const int t = task / P.nchunk, ch = task % P.nchunk;
    const int tc[3] = {t / (nl * nl), (t / nl) % nl, t % nl};
    const int par = ((tc[0] & 1) << 2) | ((tc[1] & 1) << 1) | (tc[2] & 1);
    const double Rt[3] = {(tc[0] + 0.5) * P.w, (tc[1] + 0.5) * P.w, (tc[2] + 0.5) * P.w};
    double ar[MC_PMAX + 1], ai[MC_PMAX + 1];
#pragma unroll
    for (int n = 0; n <= MC_PMAX; n++) ar[n] = ai[n] = 0.0;
    const int kb = ch * per, ke = min(189, kb + per);
    for (int k = kb; k < ke; k++) {
      int ox, oy, oz;
      il_unpack(il[par][k], &ox, &oy, &oz);
      const int e[3] = {tc[0] + ox, tc[1] + oy, tc[2] + oz};
      int src[3];
      double shift[3];
      bool ok = true;
      for (int d = 0; d < 3; d++) {
        if (pbc) {
          src[d] = mc_wrap_coord(e[d], nl);
        } else {
          src[d] = e[d];
          if (e[d] < 0 || e[d] >= nl) ok = false;
        }
        shift[d] = (double)((e[d] - src[d]) / nl) * P.a;
      }
      if (!ok) continue;
      for (int fc = 0; fc < f * f * f; fc++) {
        const int gx = src[0] * f + fc / (f * f), gy = src[1] * f + (fc / f) % f,
                  gz = src[2] * f + fc % f;
        const int cell = (gx * nL + gy) * nL + gz;
        const int b = cstart[cell], cnt = cstart[cell + 1] - b;
        for (int s0 = 0; s0 < cnt; s0 += 2) {
          const int s = s0 + half;
          const bool act = s < cnt;
          const double* v = part + 4 * (size_t)(b + (act ? s : 0));
          const double dx = act ? v[0] + shift[0] - Rt[0] : 3.0;
          const double dy = act ? v[1] + shift[1] - Rt[1] : 3.0;
          const double dz = act ? v[2] + shift[2] - Rt[2] : 3.0;
          const double qi = act ? v[3] : 0.0;
          irregular_columns<double>(&tabs, p, m, dx, dy, dz, [&](int n, double cr, double ci) {
            ar[n] += qi * cr;
            ai[n] -= qi * ci;
          });
        }
      }
    }
    double* st = stage[warp];
#pragma unroll
    for (int n = 0; n <= MC_PMAX; n++) {
      const double orr = __shfl_xor_sync(0xffffffffu, ar[n], 16);
      const double oii = __shfl_xor_sync(0xffffffffu, ai[n], 16);
      if (half == 0 && n <= p && m <= n) {
        const int kk = rl_re(n, m);
        st[kk] = ar[n] + orr;
        if (m) st[kk + 1] = ai[n] + oii;
      }
    }
    __syncwarp();
    double* o = scratch + ((size_t)t * P.nchunk + ch) * C;
    for (int kk = lane; kk < C; kk += 32) o[kk] = st[kk];
    __syncwarp();
  }
}

// out[t][k] = (sum over chunks in order) / sqrt((n-m)!(n+m)!): the paper's
// normalisation of the coefficients (the same layout as mc_get_local)
__global__ void k_reduce_noalloc(int ntarget, int nchunk, int C, const double* __restrict__ in,
                                 double* __restrict__ out) {
  const size_t total = (size_t)ntarget * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t t = i / C;
    const int k = (int)(i % C);
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ch++) s += in[(t * nchunk + ch) * C + k];
    int n = (int)sqrtf((float)k + 0.5f);
    while (n * n > k) n--;
    while ((n + 1) * (n + 1) <= k) n++;
    const int rem = k - n * n, mm = (rem + 1) / 2;
    double f = 1.0;
    for (int q = 2; q <= n - mm; q++) f *= q;
    for (int q = 2; q <= n + mm; q++) f *= q;
    out[i] = s / sqrt(f);
  }
}

// device address of the scratch, looked up once per device and kept for the
// life of the process (a cudaDeviceReset would make it stale; the header
// forbids calls after one)
constexpr int kMaxDevices = 64;
double* g_scratch_ptr[kMaxDevices];
std::mutex g_scratch_mutex;

int scratch_for_current_device(double** out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MC_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) {
      cudaGetLastError();  // the failed lookup's own error (none was pending)
      return MC_ERR_CUDA;
    }
    g_scratch_ptr[dev] = (double*)ptr;
  }
  *out = g_scratch_ptr[dev];
  return MC_OK;
}

}  // namespace

extern "C" int mc_p2l_level_noalloc(const double* d_part, const int* d_cell_start, int64_t n,
                                    double box, int levels, int level, int p, int bc,
                                    double* d_out, void* cuda_stream) {
  if (!d_part || !d_cell_start || !d_out || n < 0 || !(box > 0.0) || !isfinite(box))
    return MC_ERR_ARG;
  if (levels < 2 || levels > 8 || level < 2 || level > levels) return MC_ERR_LEVELS;
  if (p < 0 || p > MC_PMAX) return MC_ERR_ORDER;
  if (bc != MC_BC_PBC && bc != MC_BC_FREE) return MC_ERR_ARG;
  const int C = (p + 1) * (p + 1);
  const long long nl = 1LL << (level - 1), ncl = nl * nl * nl;
  // chunks of the interaction list per target: as many as fit the scratch,
  // up to enough tasks to fill the GPU; a level whose single-chunk partials
  // do not fit is refused
  if (ncl * C > (long long)MC_NOALLOC_SCRATCH_DOUBLES) return MC_ERR_SCRATCH;
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess ||
      cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MC_ERR_CUDA;
  long long nchunk = (4LL * sms * MC_WARPS + ncl - 1) / ncl;
  nchunk = nchunk < 1 ? 1 : (nchunk > 189 ? 189 : nchunk);
  while (nchunk > 1 && ncl * nchunk * C > (long long)MC_NOALLOC_SCRATCH_DOUBLES) nchunk--;
  // an error left by the caller's earlier work is not ours to clear or
  // report as this call's own: launch nothing
  if (cudaPeekAtLastError() != cudaSuccess) return MC_ERR_PENDING;
  double* scratch = nullptr;
  int rc = scratch_for_current_device(&scratch);
  if (rc != MC_OK) return rc;
  NoAllocP2L P;
  P.L = levels;
  P.l = level;
  P.p = p;
  P.C = C;
  P.bc = bc;
  P.nL = 1 << (levels - 1);
  P.nchunk = (int)nchunk;
  P.a = box;
  P.w = box / (double)nl;
  cudaStream_t stream = (cudaStream_t)cuda_stream;
  const long long ntask = ncl * nchunk;
  long long blocks = (ntask + MC_WARPS - 1) / MC_WARPS;
  if (blocks > 8LL * sms) blocks = 8LL * sms;
  k_p2l_level_noalloc<<<(int)blocks, MC_THREADS, 0, stream>>>(P, d_part, d_cell_start, scratch);
  // no error was pending before the launch, so one now is the launch's own
  if (cudaGetLastError() != cudaSuccess) return MC_ERR_CUDA;
  long long rb = (ncl * C + 255) / 256;
  if (rb > 8LL * sms) rb = 8LL * sms;
  k_reduce_noalloc<<<(int)rb, 256, 0, stream>>>((int)ncl, (int)nchunk, C, scratch, d_out);
  if (cudaGetLastError() != cudaSuccess) return MC_ERR_CUDA;
  return MC_OK;
}
