// Setup-side kernels: cell lists, Alg. L.3 (initialise the level local
// expansions) as a per-target gather, the box multipole K and lattice local
// expansion H = R(K) of Sec. 3.4 (ii)/(iv), the total energy, and the lattice
// sums / far-field operator behind R.  All FP64.
#include <math.h>

#include "mc_dev.cuh"

// ---------------------------------------------------------------- cell lists
__global__ void k_cell_count(int n, const double4* __restrict__ ppos, double inv_w, int nL,
                             int* __restrict__ cell_of, int* __restrict__ counts) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double4 v = ppos[i];
    const int cx = finest_coord(v.x, inv_w, nL), cy = finest_coord(v.y, inv_w, nL),
              cz = finest_coord(v.z, inv_w, nL);
    const int c = (cx * nL + cy) * nL + cz;
    cell_of[i] = c;
    atomicAdd(&counts[c], 1);
  }
}

__global__ void k_cell_fill(int n, const int* __restrict__ cell_of, int cap, int* __restrict__ fill,
                            int* __restrict__ cpid) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const int c = cell_of[i];
    const int s = atomicAdd(&fill[c], 1);
    cpid[(size_t)c * cap + s] = i;
  }
}

// per cell: order the slots by particle id (deterministic layout), then
// write slot positions (absolute FP64 and FP32 relative to the cell centre)
__global__ void k_cell_sort(int ncell, int nL, int cap, double w, const int* __restrict__ counts,
                            const double4* __restrict__ ppos, int* __restrict__ cpid,
                            double4* __restrict__ cpos, float4* __restrict__ cpos32,
                            int* __restrict__ pslot) {
  for (int c = blockIdx.x * blockDim.x + threadIdx.x; c < ncell; c += gridDim.x * blockDim.x) {
    int* ids = cpid + (size_t)c * cap;
    const int cnt = counts[c];
    for (int a = 1; a < cnt; a++) {
      const int v = ids[a];
      int b = a - 1;
      while (b >= 0 && ids[b] > v) {
        ids[b + 1] = ids[b];
        b--;
      }
      ids[b + 1] = v;
    }
    const int cx = c / (nL * nL), cy = (c / nL) % nL, cz = c % nL;
    const double Rx = (cx + 0.5) * w, Ry = (cy + 0.5) * w, Rz = (cz + 0.5) * w;
    for (int a = 0; a < cnt; a++) {
      const int i = ids[a];
      const double4 v = ppos[i];
      cpos[(size_t)c * cap + a] = v;
      cpos32[(size_t)c * cap + a] =
          make_float4((float)(v.x - Rx), (float)(v.y - Ry), (float)(v.z - Rz), (float)v.w);
      pslot[i] = c * cap + a;
    }
  }
}

__global__ void k_max_int(int n, const int* __restrict__ v, int* __restrict__ out) {
  int m = 0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    m = max(m, v[i]);
  atomicMax(out, m);
}

// -------------------------------------------- Alg. L.3 as a per-target gather
// Each warp task is (target cell t of level l, chunk of t's source units).
// By the symmetry of the interaction list, the cells whose lists contain t
// are exactly t's own list (with the opposite image shift), so
//   Lhat_t = sum_{e in IL(t)} sum_{i in cell(e)} q_i conj It(r_i + shift a - R_t).
// A source unit is one finest cell of one list entry (189 f^3 units per
// target, f = 2^(L-l) finest cells per axis of a level-l cell), so chunks
// have equal work on every level.  Four charges per warp step (one per
// group of 8 lanes).  Partial expansions of the chunks go to `out`
// ([t][chunk][C]), reduced in a fixed order by k_reduce_chunks.
__global__ void __launch_bounds__(MC_THREADS)
    k_p2l_level(const McSys* __restrict__ sysp, int l, int nchunk, double* __restrict__ out) {
  __shared__ McSys S;
  __shared__ HarmTabs<double> tabs;
  __shared__ unsigned short il[8][189];
  __shared__ double stage[MC_WARPS][256];
  __shared__ double s_iW[MC_PMAX + 1][16];
  __shared__ double s_P[(MC_PMAX + 1) * (MC_PMAX + 1)];
  if (threadIdx.x == 0) S = *sysp;
  harm_tabs_init<double>(&tabs);
  irregular_w_tabs<double>(s_iW, s_P);
  il_table_init(il);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane >> 3;
  const int p = S.p, C = S.C, L = S.L;
  const bool pbc = S.bc == 0;
  const int nl = S.lev_n[l], f = 1 << (L - l), nL = S.nL;
  const double w = S.lev_w[l];
  const int ntask = nl * nl * nl * nchunk;
  const int f3 = f * f * f;
  const long long units = 189LL * f3;
  const long long per = (units + nchunk - 1) / nchunk;
  for (int task = blockIdx.x * MC_WARPS + warp; task < ntask; task += gridDim.x * MC_WARPS) {
    const int t = task / nchunk, ch = task % nchunk;
    const int tc[3] = {t / (nl * nl), (t / nl) % nl, t % nl};
    const int par = ((tc[0] & 1) << 2) | ((tc[1] & 1) << 1) | (tc[2] & 1);
    const double Rt[3] = {(tc[0] + 0.5) * w, (tc[1] + 0.5) * w, (tc[2] + 0.5) * w};
    double ar[MC_PMAX + 2], ai[MC_PMAX + 2];
#pragma unroll
    for (int q = 0; q <= MC_PMAX + 1; q++) ar[q] = ai[q] = 0.0;
    const long long ub = (long long)ch * per, ue = min(units, ub + per);
    // units [ub, ue): list entries kb..ke-1; of each entry the finest cells
    // fcb..fce-1 (all but possibly the first and last entry: every one)
    const int kb = (int)(ub / f3), ke = ue > ub ? (int)((ue - 1) / f3) + 1 : kb;
    for (int k = kb; k < ke; k++) {
      const int fcb = (int)max(0LL, ub - (long long)k * f3);
      const int fce = (int)min((long long)f3, ue - (long long)k * f3);
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
        shift[d] = (double)((e[d] - src[d]) / nl) * S.a;
      }
      if (!ok) continue;
      const double bx = shift[0] - Rt[0], by = shift[1] - Rt[1], bz = shift[2] - Rt[2];
      // this chunk's finest cells of the source cell; four charges per step
      for (int fc = fcb; fc < fce; fc++) {
        const int gx = src[0] * f + fc / (f * f), gy = src[1] * f + (fc / f) % f,
                  gz = src[2] * f + fc % f;
        const int cell = (gx * nL + gy) * nL + gz;
        const int cnt = S.ccount[cell];
        for (int s0 = 0; s0 < cnt; s0 += 4) {
          const int s = s0 + grp;
          const bool act = s < cnt;
          double4 v = make_double4(0, 0, 0, 0);
          if (act) v = S.cpos[(size_t)cell * S.cap + s];
          const double dx = act ? v.x + bx : 3.0;
          const double dy = act ? v.y + by : 3.0;
          const double dz = act ? v.z + bz : 3.0;
          const double qi = act ? v.w : 0.0;
          // column-scaled irregular set with the charge folded into its start
          // value (value (n, m) / P_n^m); P_n^m is applied once per chunk
          irregular_group_wu<double>(&tabs, s_iW, p, dx, dy, dz, qi,
                                     [&](int t2, int n, int m, bool vld, double cr, double ci) {
                                       ar[t2] += cr;
                                       ai[t2] -= ci;
                                     });
        }
      }
    }
    double* st = stage[warp];
#pragma unroll
    for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
      double vr = ar[t2], vi = ai[t2];
      vr += __shfl_xor_sync(0xffffffffu, vr, 8);
      vi += __shfl_xor_sync(0xffffffffu, vi, 8);
      vr += __shfl_xor_sync(0xffffffffu, vr, 16);
      vi += __shfl_xor_sync(0xffffffffu, vi, 16);
      int n, m;
      bool vld;
      group_nm(p, t2, &n, &m, &vld);
      if (grp == 0 && vld) {
        const int kk = rl_re(n, m);
        st[kk] = vr * s_P[kk];
        if (m) st[kk + 1] = vi * s_P[kk + 1];
      }
    }
    __syncwarp();
    double* o = out + ((size_t)t * nchunk + ch) * C;
    for (int kk = lane; kk < C; kk += 32) o[kk] = st[kk];
    __syncwarp();
  }
}

// out[t][k] = sum over chunks in order
__global__ void k_reduce_chunks(int ntarget, int nchunk, int C, const double* __restrict__ in,
                                double* __restrict__ out) {
  const size_t total = (size_t)ntarget * C;
  for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < total;
       i += (size_t)gridDim.x * blockDim.x) {
    const size_t t = i / C, k = i % C;
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ch++) s += in[(t * nchunk + ch) * C + k];
    out[i] = s;
  }
}

// ------------------------------------------- K (Sec. 3.4 ii) and the dipole
// chunk ch of the particles: partial Khat = sum q conj Rt(r - R1); dipole
// sum q r appended at [C .. C+2].
__global__ void __launch_bounds__(MC_THREADS)
    k_box_multipole(const McSys* __restrict__ sysp, int nchunk, double* __restrict__ out) {
  __shared__ McSys S;
  __shared__ HarmTabs<double> tabs;
  __shared__ double stage[MC_WARPS][256];
  if (threadIdx.x == 0) S = *sysp;
  harm_tabs_init<double>(&tabs);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane >> 3, g8 = lane & 7;
  const int p = S.p, C = S.C;
  const int per = (S.n + nchunk - 1) / nchunk;
  const double c1 = 0.5 * S.a;
  for (int ch = blockIdx.x * MC_WARPS + warp; ch < nchunk; ch += gridDim.x * MC_WARPS) {
    double ar[MC_PMAX + 2], ai[MC_PMAX + 2];
#pragma unroll
    for (int q = 0; q <= MC_PMAX + 1; q++) ar[q] = ai[q] = 0.0;
    double D[3] = {0, 0, 0};
    const int ib = ch * per, ie = min(S.n, ib + per);
    for (int i0 = ib; i0 < ie; i0 += 4) {
      const int i = i0 + grp;
      const bool act = i < ie;
      double4 v = make_double4(c1, c1, c1, 0.0);
      if (act) v = S.ppos[i];
      regular_group<double>(&tabs, p, v.x - c1, v.y - c1, v.z - c1,
                            [&](int t2, int n, int m, bool vld, double cr, double ci) {
                              ar[t2] += v.w * cr;
                              ai[t2] -= v.w * ci;
                            });
      if (g8 == 0) {
        D[0] += v.w * v.x;
        D[1] += v.w * v.y;
        D[2] += v.w * v.z;
      }
    }
    double* st = stage[warp];
#pragma unroll
    for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
      double vr = ar[t2], vi = ai[t2];
      vr += __shfl_xor_sync(0xffffffffu, vr, 8);
      vi += __shfl_xor_sync(0xffffffffu, vi, 8);
      vr += __shfl_xor_sync(0xffffffffu, vr, 16);
      vi += __shfl_xor_sync(0xffffffffu, vi, 16);
      int n, m;
      bool vld;
      group_nm(p, t2, &n, &m, &vld);
      if (grp == 0 && vld) {
        const int kk = rl_re(n, m);
        st[kk] = vr;
        if (m) st[kk + 1] = vi;
      }
    }
    for (int d = 0; d < 3; d++) {
      D[d] += __shfl_xor_sync(0xffffffffu, D[d], 8);
      D[d] += __shfl_xor_sync(0xffffffffu, D[d], 16);
    }
    __syncwarp();
    double* o = out + (size_t)ch * (C + 3);
    for (int kk = lane; kk < C; kk += 32) o[kk] = st[kk];
    if (lane == 0) {
      o[C] = D[0];
      o[C + 1] = D[1];
      o[C + 2] = D[2];
    }
    __syncwarp();
  }
}

// Khat, dipole from the chunk partials (fixed order), then Hhat = G Khat
__global__ void k_far_finish(const McSys* __restrict__ sysp, int nchunk,
                             const double* __restrict__ in) {
  const McSys& S = *sysp;
  const int C = S.C;
  __shared__ double kh[256 + 3];
  for (int k = threadIdx.x; k < C + 3; k += blockDim.x) {
    double s = 0.0;
    for (int ch = 0; ch < nchunk; ch++) s += in[(size_t)ch * (C + 3) + k];
    kh[k] = s;
  }
  __syncthreads();
  for (int k = threadIdx.x; k < C; k += blockDim.x) {
    S.Khat[k] = kh[k];
    double h = 0.0;
    if (S.bc == 0)
      for (int c = 0; c < C; c++) h += S.G[(size_t)c * C + k] * kh[c];
    S.Hhat[k] = h;
  }
  if (threadIdx.x < 3) S.dipv[threadIdx.x] = kh[C + threadIdx.x];
}

// ------------------------------------------------------------ total energy
// U = 1/2 sum_i q_i phi_i + 1/2 sum_k W_k Khat_k Hhat_k + dipole term, where
// phi_i sums the level expansions at r_i and the direct near-cell charges
// other than i itself.  One warp per particle; per-warp running sums in
// `out` (fixed assignment), reduced by k_energy_finish.
__global__ void __launch_bounds__(MC_THREADS)
    k_energy_particles(const McSys* __restrict__ sysp, double* __restrict__ out) {
  __shared__ McSys S;
  __shared__ HarmTabs<double> tabs;
  __shared__ unsigned short il[8][189];
  if (threadIdx.x == 0) S = *sysp;
  harm_tabs_init<double>(&tabs);
  il_table_init(il);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = S.p, C = S.C, L = S.L, nL = S.nL;
  const bool pbc = S.bc == 0;
  const int gw = blockIdx.x * MC_WARPS + warp, nw = gridDim.x * MC_WARPS;
  double usum = 0.0;
  for (int i = gw; i < S.n; i += nw) {
    const double4 v = S.ppos[i];
    const int cf[3] = {finest_coord(v.x, S.inv_wL, nL), finest_coord(v.y, S.inv_wL, nL),
                       finest_coord(v.z, S.inv_wL, nL)};
    double phi = 0.0, ulj = 0.0;
    // level expansions: four levels per warp step (one per 8-lane group)
    const int nlev = L - S.lmin + 1;
    const int grp = lane >> 3;
    if (S.method == 1) {
      // multipole method: the multipole expansions of the cells of the
      // interaction list on every level, four entries per warp step
      for (int l = L; l >= S.lmin; l--) {
        const int sh = L - l, nl = S.lev_n[l];
        const double w = S.lev_w[l];
        const int cs[3] = {cf[0] >> sh, cf[1] >> sh, cf[2] >> sh};
        const int par = ((cs[0] & 1) << 2) | ((cs[1] & 1) << 1) | (cs[2] & 1);
        for (int e0 = 0; e0 < 189; e0 += 4) {
          const int e = e0 + grp;
          int ox = 0, oy = 0, oz = 0;
          if (e < 189) il_unpack(il[par][e], &ox, &oy, &oz);
          const int ex[3] = {cs[0] + ox, cs[1] + oy, cs[2] + oz};
          const bool act = e < 189 && (pbc || (ex[0] >= 0 && ex[0] < nl && ex[1] >= 0 &&
                                               ex[1] < nl && ex[2] >= 0 && ex[2] < nl));
          const int t3[3] = {mc_wrap_coord(ex[0], nl), mc_wrap_coord(ex[1], nl),
                             mc_wrap_coord(ex[2], nl)};
          const double* Mb = S.Mhat + (size_t)(S.lev_off[l] + (t3[0] * nl + t3[1]) * nl + t3[2]) * C;
          double Mr[MC_PMAX + 2], Mi[MC_PMAX + 2];
#pragma unroll
          for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
            int n, m;
            bool vld;
            group_nm(p, t2, &n, &m, &vld);
            const int k = rl_re(n, m);
            Mr[t2] = (act && vld) ? Mb[k] : 0.0;
            Mi[t2] = (act && vld && m) ? Mb[k + 1] : 0.0;
          }
          double acc = 0.0;
          const double dx = act ? v.x - (ex[0] + 0.5) * w : 3.0 * w,
                       dy = act ? v.y - (ex[1] + 0.5) * w : 3.0 * w,
                       dz = act ? v.z - (ex[2] + 0.5) * w : 3.0 * w;
          irregular_group<double>(&tabs, p, dx, dy, dz,
                                  [&](int t2, int n, int m, bool vld, double cr, double ci) {
                                    if (vld) acc += (m ? 2.0 : 1.0) * (Mr[t2] * cr - Mi[t2] * ci);
                                  });
          if (act) phi += acc;
        }
      }
    }
    for (int l0 = 0; S.method == 0 && l0 < nlev; l0 += 4) {
      const int li = l0 + grp;
      const bool act = li < nlev;
      const int l = act ? L - li : L;
      const int sh = L - l, nl = S.lev_n[l];
      const double w = S.lev_w[l];
      const int cx = cf[0] >> sh, cy = cf[1] >> sh, cz = cf[2] >> sh;
      const double* Lb = S.Lhat + (size_t)(S.lev_off[l] + (cx * nl + cy) * nl + cz) * C;
      double Lr[MC_PMAX + 2], Li[MC_PMAX + 2];
#pragma unroll
      for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
        int n, m;
        bool vld;
        group_nm(p, t2, &n, &m, &vld);
        const int k = rl_re(n, m);
        Lr[t2] = (act && vld) ? Lb[k] : 0.0;
        Li[t2] = (act && vld && m) ? Lb[k + 1] : 0.0;
      }
      double acc = 0.0;
      regular_group<double>(&tabs, p, v.x - (cx + 0.5) * w, v.y - (cy + 0.5) * w,
                            v.z - (cz + 0.5) * w,
                            [&](int t2, int n, int m, bool vld, double cr, double ci) {
                              if (vld) acc += (m ? 2.0 : 1.0) * (Lr[t2] * cr - Li[t2] * ci);
                            });
      if (!act) acc = 0.0;
      phi += acc;
    }
    // direct near cells
    for (int k = 0; k < 27; k++) {
      const int e0 = cf[0] + k / 9 - 1, e1 = cf[1] + (k / 3) % 3 - 1, e2 = cf[2] + k % 3 - 1;
      int c0 = e0, c1 = e1, c2 = e2;
      if (pbc) {
        c0 = mc_wrap_coord(e0, nL);
        c1 = mc_wrap_coord(e1, nL);
        c2 = mc_wrap_coord(e2, nL);
      } else if (e0 < 0 || e0 >= nL || e1 < 0 || e1 >= nL || e2 < 0 || e2 >= nL) {
        continue;
      }
      const double sx = ((e0 - c0) / nL) * S.a, sy = ((e1 - c1) / nL) * S.a,
                   sz = ((e2 - c2) / nL) * S.a;
      const bool zs = (e0 == c0 && e1 == c1 && e2 == c2);
      const int cell = (c0 * nL + c1) * nL + c2;
      const int cnt = S.ccount[cell];
      for (int s = lane; s < cnt; s += 32) {
        const int pid = S.cpid[(size_t)cell * S.cap + s];
        if (pid == i && zs) continue;
        const double4 xi = S.cpos[(size_t)cell * S.cap + s];
        const double ax = v.x - (xi.x + sx), ay = v.y - (xi.y + sy), az = v.z - (xi.z + sz);
        const double d2 = ax * ax + ay * ay + az * az;
        const double ir = rsqrt(d2);
        phi += xi.w * ir;
        if (S.lj_on && pid != i)  // (i's images lie beyond the cutoff)
          ulj += lj_energy(ir * ir, d2, S.lj_eps4, S.lj_s6, S.lj_s12, S.lj_rc2);
      }
    }
    phi = warp_sum(phi);
    ulj = warp_sum(ulj);
    usum += 0.5 * (v.w * phi + ulj);
  }
  if (lane == 0) out[gw] = usum;
}

__global__ void k_energy_finish(const McSys* __restrict__ sysp, int nw, const double* __restrict__ in,
                                double* __restrict__ dst) {
  const McSys& S = *sysp;
  __shared__ double red[256];
  double s = 0.0;
  for (int i = threadIdx.x; i < nw; i += blockDim.x) s += in[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    double U = red[0];
    if (S.bc == 0) {
      double far = 0.0;
      for (int k = 0; k < S.C; k++) {
        const int r = (int)sqrtf((float)k + 0.5f);
        far += ((r * r == k) ? 1.0 : 2.0) * S.Khat[k] * S.Hhat[k];
      }
      U += 0.5 * far;
      if (S.dip == 0) {
        const double D2 = S.dipv[0] * S.dipv[0] + S.dipv[1] * S.dipv[1] + S.dipv[2] * S.dipv[2];
        U += -2.0 * 3.141592653589793 / (3.0 * S.V) * D2;
      }
    }
    dst[0] = U;
  }
}

// ------------------------------------------------------------ lattice sums
// Scaled lattice sums St_l^mu = sum_{max|v_i| >= 2} It_l^mu(v) over the unit
// lattice (It the scaled irregular harmonic; St = s_l,mu S_l^mu).  Images are
// summed in cubic shells: l = 1, 2 vanish by cubic symmetry and l = 0 only
// meets the total charge (zero), so l < 3 is 0.  For 3 <= l < 20 the sum
// over all v != 0 is split (Poisson summation of the harmonic polynomial
// h(x) = |x|^l Y(x), split at t = 2):
//   sum_v h(v)/|v|^(2l+1) Q(l+1/2, 2 pi |v|^2)
//   + pi^(l-1/2)/Gamma(l+1/2) (-i)^l sum_{k != 0} h(k) e^{-pi |k|^2 / 2} / |k|^2
// and the 26 shell-1 terms are removed.  For l >= 20 shells 2..20 are summed
// directly (tail below 1e-17 relative).  One block per (l, mu >= 0).
__device__ __forceinline__ void rt_single(int l, int mu, double x, double y, double z,
                                          double* re, double* im) {
  // scaled regular harmonic Rt_l^mu(x) via the diagonal then the column
  double dr = 1.0, di = 0.0;
  for (int k = 1; k <= mu; k++) {
    const double nr = (dr * x - di * y) / (2.0 * k), ni = (dr * y + di * x) / (2.0 * k);
    dr = nr;
    di = ni;
  }
  const double r2 = x * x + y * y + z * z;
  double p1r = dr, p1i = di, p2r = 0.0, p2i = 0.0;
  for (int n = mu + 1; n <= l; n++) {
    const double den = (double)(n + mu) * (double)(n - mu);
    const double a = (2.0 * n - 1.0) * z / den, b = r2 / den;
    const double cr = a * p1r - b * p2r, ci = a * p1i - b * p2i;
    p2r = p1r;
    p2i = p1i;
    p1r = cr;
    p1i = ci;
  }
  *re = p1r;
  *im = p1i;
}

__global__ void k_lattice_sums(int lmax, double* __restrict__ out /* complex (lmax+1)^2 */) {
  // block -> (l, mu)
  int b = blockIdx.x, l = 0;
  while (b >= l + 1) {
    b -= l + 1;
    l++;
  }
  const int mu = b;
  __shared__ double rr[256], ri[256];
  double sr = 0.0, si = 0.0;
  double fl = 1.0, fh = 1.0;  // (l-mu)!, (l+mu)!
  for (int k = 2; k <= l - mu; k++) fl *= k;
  for (int k = 2; k <= l + mu; k++) fh *= k;
  const double s2 = fl * fh;  // h = s2 * Rt
  const double pi = 3.141592653589793;
  if (l >= 3 && l < 20) {
    const int R = 7, K = 9;
    const int side = 2 * R + 1;
    for (int idx = threadIdx.x; idx < side * side * side; idx += blockDim.x) {
      const int x = idx / (side * side) - R, y = (idx / side) % side - R, z = idx % side - R;
      if (!x && !y && !z) continue;
      const double r2 = (double)(x * x + y * y + z * z), r = sqrt(r2);
      double hr, hi;
      rt_single(l, mu, x, y, z, &hr, &hi);
      hr *= s2;
      hi *= s2;
      // Q(l + 1/2, 2 pi r^2)
      const double X = 2.0 * pi * r2;
      double Q = erfc(sqrt(X));
      double term = sqrt(X) * exp(-X) / (0.5 * sqrt(pi));  // x^{1/2} e^-x / Gamma(3/2)
      for (int i = 0; i < l; i++) {
        Q += term;
        term *= X / (i + 1.5);
      }
      double wgt = Q;
      if (abs(x) <= 1 && abs(y) <= 1 && abs(z) <= 1) wgt -= 1.0;
      const double inv = pow(r, -(2.0 * l + 1.0));
      sr += hr * wgt * inv;
      si += hi * wgt * inv;
    }
    // reciprocal part
    double gam = sqrt(pi);
    for (int i = 0; i < l; i++) gam *= (0.5 + i);
    const double pref = pow(pi, l - 0.5) / gam;
    // (-i)^l
    const int lm = l & 3;
    const double ur = (lm == 0) ? 1.0 : (lm == 2 ? -1.0 : 0.0);
    const double ui = (lm == 1) ? -1.0 : (lm == 3 ? 1.0 : 0.0);
    const int sk = 2 * K + 1;
    for (int idx = threadIdx.x; idx < sk * sk * sk; idx += blockDim.x) {
      const int x = idx / (sk * sk) - K, y = (idx / sk) % sk - K, z = idx % sk - K;
      if (!x && !y && !z) continue;
      const double k2 = (double)(x * x + y * y + z * z);
      double hr, hi;
      rt_single(l, mu, x, y, z, &hr, &hi);
      const double wgt = pref * s2 * exp(-pi * k2 / 2.0) / k2;
      sr += wgt * (ur * hr - ui * hi);
      si += wgt * (ur * hi + ui * hr);
    }
  } else if (l >= 20) {
    const int R = 20, side = 2 * R + 1;
    for (int idx = threadIdx.x; idx < side * side * side; idx += blockDim.x) {
      const int x = idx / (side * side) - R, y = (idx / side) % side - R, z = idx % side - R;
      if (max(abs(x), max(abs(y), abs(z))) < 2) continue;
      const double r2 = (double)(x * x + y * y + z * z);
      double hr, hi;
      rt_single(l, mu, x, y, z, &hr, &hi);
      const double inv = pow(r2, -(l + 0.5));
      sr += s2 * hr * inv;
      si += s2 * hi * inv;
    }
  }
  rr[threadIdx.x] = sr;
  ri[threadIdx.x] = si;
  __syncthreads();
  for (int o = blockDim.x / 2; o > 0; o >>= 1) {
    if (threadIdx.x < o) {
      rr[threadIdx.x] += rr[threadIdx.x + o];
      ri[threadIdx.x] += ri[threadIdx.x + o];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const int id = l * l + l + mu;
    out[2 * id] = rr[0];
    out[2 * id + 1] = ri[0];
    if (mu > 0) {
      const int idn = l * l + l - mu;
      out[2 * idn] = rr[0];
      out[2 * idn + 1] = -ri[0];
    }
  }
}

// --------------------------------------------------- far-field operator G
// Hhat = G Khat in the scaled real layout.  The multipole-to-local theorem
// of Greengard and Rokhlin, written for the scaled expansions, becomes
//   Hhat_j^k = sum_{n, m=-n..n} (-1)^n sigma(k, m) a^-(j+n+1) St_{j+n}^{m-k} Khat_n^m
// with sigma(k, m) = i^{|k-m|-|k|-|m|} (a real sign), Khat_n^-m = conj Khat_n^m
// and St the scaled lattice sums.  One thread per matrix entry; stored
// column-major: G[c * C + row].
__device__ __forceinline__ void rl_decode(int k, int* n, int* m, int* im) {
  int r = (int)sqrtf((float)k + 0.5f);
  while (r * r > k) r--;
  while ((r + 1) * (r + 1) <= k) r++;
  *n = r;
  const int rem = k - r * r;
  *m = (rem + 1) / 2;
  *im = (rem > 0 && (rem % 2) == 0) ? 1 : 0;
}

__device__ __forceinline__ double sigma_km(int k, int m) {
  const int e = (abs(k) + abs(m) - abs(k - m)) / 2;
  return (e & 1) ? -1.0 : 1.0;
}

__global__ void k_far_operator(int p, double a, const double* __restrict__ St, double* __restrict__ G) {
  const int C = (p + 1) * (p + 1);
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < C * C; idx += gridDim.x * blockDim.x) {
    const int c = idx / C, row = idx % C;
    int j, k, rim, n, m, cim;
    rl_decode(row, &j, &k, &rim);
    rl_decode(c, &n, &m, &cim);
    const int l = j + n;
    const double sc = ((n & 1) ? -1.0 : 1.0) * pow(a, -(double)(l + 1));
    // T1 multiplies Khat_n^m, T2 multiplies conj(Khat_n^m) (the -m term)
    const int mu1 = m - k, mu2 = -m - k;
    const double s1 = sigma_km(k, m) * sc, s2 = sigma_km(k, -m) * sc;
    const double t1r = s1 * St[2 * (l * l + l + mu1)], t1i = s1 * St[2 * (l * l + l + mu1) + 1];
    double t2r = 0.0, t2i = 0.0;
    if (m > 0) {
      t2r = s2 * St[2 * (l * l + l + mu2)];
      t2i = s2 * St[2 * (l * l + l + mu2) + 1];
    }
    double v;
    if (!rim && !cim) v = t1r + t2r;
    else if (!rim && cim) v = -(t1i - t2i);
    else if (rim && !cim) v = t1i + t2i;
    else v = t1r - t2r;
    G[idx] = v;
  }
}

// ------------------------------------------ FMM-variant setup (fast mode)
// Sec. 3.2, last paragraph: multipoles of every cell, then each cell's
// Psi^Delta as the sum of multipole-to-local translations from the cells of
// its interaction list (no local-to-local pass).  Scaled multipoles
// Khat_n^m = sum q conj Rt_n^m(r - R_cell) are formed directly on every level.

// one warp per (cell of level l, chunk of its finest cells); four charges per
// step; chunk partials go to out[(cell * nchunk + chunk) * C] for
// k_reduce_chunks (nchunk = 1 writes the level directly)
__global__ void __launch_bounds__(MC_THREADS)
    k_p2m_level(const McSys* __restrict__ sysp, int l, int nchunk, double* __restrict__ out) {
  __shared__ McSys S;
  __shared__ HarmTabs<double> tabs;
  __shared__ double stage[MC_WARPS][256];
  if (threadIdx.x == 0) S = *sysp;
  harm_tabs_init<double>(&tabs);
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane >> 3;
  const int p = S.p, C = S.C, L = S.L, nL = S.nL;
  const int nl = S.lev_n[l], f = 1 << (L - l);
  const double w = S.lev_w[l];
  const int nf = f * f * f, per = (nf + nchunk - 1) / nchunk;
  const int ntask = nl * nl * nl * nchunk;
  for (int task = blockIdx.x * MC_WARPS + warp; task < ntask; task += gridDim.x * MC_WARPS) {
    const int t = task / nchunk, ch = task % nchunk;
    const int tc[3] = {t / (nl * nl), (t / nl) % nl, t % nl};
    const double Rx = (tc[0] + 0.5) * w, Ry = (tc[1] + 0.5) * w, Rz = (tc[2] + 0.5) * w;
    double ar[MC_PMAX + 2], ai[MC_PMAX + 2];
#pragma unroll
    for (int q = 0; q <= MC_PMAX + 1; q++) ar[q] = ai[q] = 0.0;
    const int fb = ch * per, fe = min(nf, fb + per);
    for (int fc = fb; fc < fe; fc++) {
      const int gx = tc[0] * f + fc / (f * f), gy = tc[1] * f + (fc / f) % f, gz = tc[2] * f + fc % f;
      const int cell = (gx * nL + gy) * nL + gz;
      const int cnt = S.ccount[cell];
      for (int s0 = 0; s0 < cnt; s0 += 4) {
        const int s = s0 + grp;
        double4 v = make_double4(Rx, Ry, Rz, 0.0);  // inactive: zero charge at the centre
        if (s < cnt) v = S.cpos[(size_t)cell * S.cap + s];
        regular_group<double>(&tabs, p, v.x - Rx, v.y - Ry, v.z - Rz,
                              [&](int t2, int n, int m, bool vld, double cr, double ci) {
                                ar[t2] += v.w * cr;
                                ai[t2] -= v.w * ci;
                              });
      }
    }
    double* st = stage[warp];
#pragma unroll
    for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
      double vr = ar[t2], vi = ai[t2];
      vr += __shfl_xor_sync(0xffffffffu, vr, 8);
      vi += __shfl_xor_sync(0xffffffffu, vi, 8);
      vr += __shfl_xor_sync(0xffffffffu, vr, 16);
      vi += __shfl_xor_sync(0xffffffffu, vi, 16);
      int n, m;
      bool vld;
      group_nm(p, t2, &n, &m, &vld);
      if (grp == 0 && vld) {
        const int kk = rl_re(n, m);
        st[kk] = vr;
        if (m) st[kk + 1] = vi;
      }
    }
    __syncwarp();
    double* o = out + ((size_t)t * nchunk + ch) * C;
    for (int kk = lane; kk < C; kk += 32) o[kk] = st[kk];
    __syncwarp();
  }
}

// It_l^mu(o), the scaled irregular harmonic at unit cell width, for every
// integer offset o in [-3, 3]^3 (the interaction-list offsets are among
// them), l <= 2p, 0 <= mu <= l: It = (l-mu)! (l+mu)! Rt / |o|^(2l+1).
// Layout: [((ox+3)*7 + oy+3)*7 + oz+3][l(l+1)/2 + mu] complex (re, im).
__global__ void k_offset_table(int p, double* __restrict__ out) {
  const int lmax = 2 * p, per = (lmax + 1) * (lmax + 2) / 2;
  for (int idx = blockIdx.x * blockDim.x + threadIdx.x; idx < 343 * per;
       idx += gridDim.x * blockDim.x) {
    const int o = idx / per, r = idx % per;
    int l = 0;
    while ((l + 1) * (l + 2) / 2 <= r) l++;
    const int mu = r - l * (l + 1) / 2;
    const int ox = o / 49 - 3, oy = (o / 7) % 7 - 3, oz = o % 7 - 3;
    double re = 0.0, im = 0.0;
    if (ox || oy || oz) {
      double hr, hi;
      rt_single(l, mu, ox, oy, oz, &hr, &hi);
      double f = 1.0;
      for (int q = 2; q <= l - mu; q++) f *= q;
      for (int q = 2; q <= l + mu; q++) f *= q;
      const double r2 = (double)(ox * ox + oy * oy + oz * oz);
      const double sc = f * pow(r2, -(l + 0.5));
      re = hr * sc;
      im = hi * sc;
    }
    out[2 * (size_t)idx] = re;
    out[2 * (size_t)idx + 1] = im;
  }
}

// Multipole-to-local over the interaction lists of level l.  With scaled
// coefficients (Khat = M / s_n^m, Lhat = L s_j^k, s_n^m = sqrt((n-m)!(n+m)!))
// the translation theorem of Greengard and Rokhlin for a source cell at
// offset o (in cell widths w) from the target reads
//   Lhat_j^k = w^-(j+1) sum_{n<=p} sum_{|m|<=n} (-1)^n sigma(k,m)
//              It_{j+n}^{m-k}(o) w^-n Khat_n^m,   sigma(k,m) = (-1)^min(k,m)
// for k, m >= 0 and 1 for m < 0 <= k; Khat^{n,-m} = conj Khat^{n,m} and
// It^{l,-mu} = conj It^{l,mu}.  The m and -m terms are taken together, so
// each (j, k; n, m > 0) needs four real coefficients, shared by the
// MC_M2L_G targets a lane carries.
// A CTA takes MC_M2L_T targets of one parity class, which share the 189
// offsets, and one chunk of those offsets: each offset's It table is staged
// once per CTA, each warp stages its targets' source multipoles (scaled by
// (-1/w)^n), and lane q computes the outputs q, q + 32, ... (j, k >= 0) of
// its warp's targets.  With nco > 1 offset chunks (the small levels, whose
// few targets would otherwise leave most SMs idle) each chunk's sums go to
// part[(cell * nco + chunk) * C], reduced in chunk order by k_reduce_chunks.
#define MC_M2L_G 4
#define MC_M2L_T (MC_WARPS * MC_M2L_G)
__device__ __forceinline__ double flip_sign(double x, unsigned long long mask) {
  return __longlong_as_double(__double_as_longlong(x) ^ (long long)mask);
}

template <int NS>
__global__ void __launch_bounds__(MC_THREADS)
    k_m2l_level(const McSys* __restrict__ sysp, int l, const double* __restrict__ Mlev,
                const double* __restrict__ otab, double* __restrict__ Llev, int nco,
                double* __restrict__ part) {
  __shared__ McSys S;
  __shared__ unsigned short il[8][189];
  __shared__ double s_wn[MC_PMAX + 1];  // (-1)^n w^-n, the source scaling
  extern __shared__ double dyn[];
  if (threadIdx.x == 0) S = *sysp;
  il_table_init(il);
  __syncthreads();
  if (threadIdx.x <= MC_PMAX) {
    const int n = threadIdx.x;
    s_wn[n] = ((n & 1) ? -1.0 : 1.0) * pow(S.lev_w[l], -(double)n);
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = S.p, C = S.C;
  const bool pbc = S.bc == 0;
  const int nl = S.lev_n[l], h = nl >> 1;
  const double w = S.lev_w[l];
  const int per = (2 * p + 1) * (2 * p + 2) / 2;
  const int nout = (p + 1) * (p + 2) / 2;
  double* tab = dyn;
  double* src = dyn + 2 * per + (size_t)warp * MC_M2L_G * C;
  int qj[NS], qk[NS];
#pragma unroll
  for (int u = 0; u < NS; u++) {
    const int q = lane + 32 * u;
    int j = 0;
    while ((j + 1) * (j + 2) / 2 <= q) j++;
    qj[u] = j;
    qk[u] = q - j * (j + 1) / 2;
  }
  const int per_class = h * h * h;
  const int chunks = (per_class + MC_M2L_T - 1) / MC_M2L_T;
  const int per_o = (189 + nco - 1) / nco;
  for (int task = blockIdx.x; task < 8 * chunks * nco; task += gridDim.x) {
    const int oc = task % nco, tk = task / nco;
    const int cls = tk / chunks;
    const int i0 = (tk % chunks) * MC_M2L_T + warp * MC_M2L_G;
    const bool warp_has = i0 < per_class;  // warp-uniform
    const int eb = oc * per_o, ee = min(189, eb + per_o);
    const int bx = (cls >> 2) & 1, by = (cls >> 1) & 1, bz = cls & 1;
    int tgt[MC_M2L_G][3];
#pragma unroll
    for (int g = 0; g < MC_M2L_G; g++) {
      const int ii = min(i0 + g, per_class - 1);
      tgt[g][0] = 2 * (ii / (h * h)) + bx;
      tgt[g][1] = 2 * ((ii / h) % h) + by;
      tgt[g][2] = 2 * (ii % h) + bz;
    }
    double accr[NS][MC_M2L_G], acci[NS][MC_M2L_G];
#pragma unroll
    for (int u = 0; u < NS; u++)
#pragma unroll
      for (int g = 0; g < MC_M2L_G; g++) accr[u][g] = acci[u][g] = 0.0;
    for (int e = eb; e < ee; e++) {
      int ox, oy, oz;
      il_unpack(il[cls][e], &ox, &oy, &oz);
      __syncthreads();  // previous offset's tables are consumed
      const double* tb = otab + 2 * (size_t)(((ox + 3) * 7 + oy + 3) * 7 + oz + 3) * per;
      for (int i = threadIdx.x; i < 2 * per; i += MC_THREADS) tab[i] = tb[i];
#pragma unroll
      for (int g = 0; g < MC_M2L_G; g++) {
        const int e3[3] = {tgt[g][0] + ox, tgt[g][1] + oy, tgt[g][2] + oz};
        bool ok = i0 + g < per_class;
        int sc[3];
        for (int d = 0; d < 3; d++) {
          if (pbc) {
            sc[d] = mc_wrap_coord(e3[d], nl);
          } else {
            sc[d] = e3[d];
            if (e3[d] < 0 || e3[d] >= nl) ok = false;
          }
        }
        const double* ms = Mlev + (size_t)((ok ? (sc[0] * nl + sc[1]) * nl + sc[2] : 0)) * C;
        double* sg = src + g * C;
        for (int i = lane; i < C; i += 32) {
          int n = (int)sqrtf((float)i + 0.5f);
          while (n * n > i) n--;
          while ((n + 1) * (n + 1) <= i) n++;
          sg[i] = ok ? ms[i] * s_wn[n] : 0.0;
        }
      }
      __syncthreads();
#pragma unroll
      for (int u = 0; u < NS; u++) {
        if (!warp_has || lane + 32 * u >= nout) continue;
        const int j = qj[u], k = qk[u];
        for (int n = 0; n <= p; n++) {
          const int L2 = j + n;
          const double* t0 = tab + L2 * (L2 + 1);  // complex entry L2(L2+1)/2
          const double* s0 = src + n * n;
          {  // m = 0: It^{L2,-k} = conj It^{L2,k}
            const double ar = t0[2 * k], ain = t0[2 * k + 1];
#pragma unroll
            for (int g = 0; g < MC_M2L_G; g++) {
              const double kr = s0[g * C];
              accr[u][g] = fma(ar, kr, accr[u][g]);
              acci[u][g] = fma(-ain, kr, acci[u][g]);
            }
          }
          for (int m = 1; m <= n; m++) {
            const int d = m - k, ad = d < 0 ? -d : d;
            const unsigned long long sgn = (unsigned long long)(min(k, m) & 1) << 63;
            const double ar = flip_sign(t0[2 * ad], sgn);
            const double ai = flip_sign(t0[2 * ad + 1], sgn ^ ((unsigned long long)(d < 0) << 63));
            const double br = t0[2 * (m + k)], bir = t0[2 * (m + k) + 1];  // b = conj(br + i bir)
            const double c1 = ar + br, c2n = ai + bir, c3 = ai - bir, c4 = ar - br;
#pragma unroll
            for (int g = 0; g < MC_M2L_G; g++) {
              const double kr = s0[g * C + 2 * m - 1], ki = s0[g * C + 2 * m];
              accr[u][g] = fma(kr, c1, fma(-ki, c2n, accr[u][g]));
              acci[u][g] = fma(kr, c3, fma(ki, c4, acci[u][g]));
            }
          }
        }
      }
    }
#pragma unroll
    for (int g = 0; g < MC_M2L_G; g++) {
      if (i0 + g >= per_class) continue;
      const size_t cell = (size_t)((tgt[g][0] * nl + tgt[g][1]) * nl + tgt[g][2]);
      double* o = nco > 1 ? part + (cell * nco + oc) * C : Llev + cell * C;
#pragma unroll
      for (int u = 0; u < NS; u++) {
        if (lane + 32 * u >= nout) continue;
        const int j = qj[u], k = qk[u];
        const double sc = pow(w, -(double)(j + 1));
        const int kk = rl_re(j, k);
        o[kk] = accr[u][g] * sc;
        if (k) o[kk + 1] = acci[u][g] * sc;
      }
    }
  }
}

size_t m2l_smem_bytes(int p) {
  const int C = (p + 1) * (p + 1), per = (2 * p + 1) * (2 * p + 2) / 2;
  return sizeof(double) * (2 * (size_t)per + (size_t)MC_WARPS * MC_M2L_G * C);
}

// offset chunks of the multipole-to-local pass on a level with nl cells per
// axis: about two tasks per SM (1 on the large levels)
int m2l_offset_chunks(int nl, int sms) {
  const int h = nl / 2, chunks = (h * h * h + MC_M2L_T - 1) / MC_M2L_T;
  const int want = (2 * sms + 8 * chunks - 1) / (8 * chunks);
  return std::max(1, std::min(189, want));
}

// launches the multipole-to-local pass of one level (scratch: room for the
// offset chunks' partial sums, ncl x nco x C doubles)
cudaError_t m2l_launch(const McSys* d_sys, int p, int l, int nl, int sms, const double* M,
               const double* otab, double* Lout, double* scratch, size_t scratch_doubles,
               cudaStream_t st) {
  const int nout = (p + 1) * (p + 2) / 2, ns = (nout + 31) / 32;
  const int C = (p + 1) * (p + 1);
  const int h = nl / 2, chunks = (h * h * h + MC_M2L_T - 1) / MC_M2L_T;
  const size_t ncl = (size_t)nl * nl * nl;
  int nco = m2l_offset_chunks(nl, sms);
  while (nco > 1 && ncl * nco * C > scratch_doubles) nco--;
  const int grid = std::max(1, std::min(8 * chunks * nco, sms * 4));
  const size_t smem = m2l_smem_bytes(p);
  cudaError_t e = cudaSuccess;
#define MC_M2L_CASE(NS_)                                                                   \
  case NS_:                                                                                \
    e = cudaFuncSetAttribute(k_m2l_level<NS_>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                             (int)smem);                                                   \
    if (e == cudaSuccess) {                                                                \
      k_m2l_level<NS_><<<grid, MC_THREADS, smem, st>>>(d_sys, l, M, otab, Lout, nco, scratch); \
      e = cudaGetLastError();                                                              \
    }                                                                                      \
    break;
  switch (ns) {
    MC_M2L_CASE(1)
    MC_M2L_CASE(2)
    MC_M2L_CASE(3)
    MC_M2L_CASE(4)
    MC_M2L_CASE(5)
    default:
      e = cudaErrorInvalidValue;
  }
#undef MC_M2L_CASE
  if (e == cudaSuccess && nco > 1) {
    const int rb = (int)std::min<size_t>((ncl * C + 255) / 256, (size_t)sms * 8);
    k_reduce_chunks<<<std::max(1, rb), 256, 0, st>>>((int)ncl, nco, C, scratch, Lout);
    e = cudaGetLastError();
  }
  return e;
}
