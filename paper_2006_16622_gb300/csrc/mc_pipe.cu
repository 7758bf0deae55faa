// Pipelined Metropolis-Hastings chain (the mc_run path): the accept of step
// k-1 (Alg. L.2 and its bookkeeping) runs in the same phase as the proposal
// of step k (Alg. L.1, Alg. 1, Sec. 3.3), so a step costs one grid barrier.
//
// Phase t holds (a) the propose items of step t and (b) the accept items of
// the pending move M = step t-1 if it was accepted.  The propose items must
// see the state after M although M is written during the phase:
//   - expansions on coarse levels (<= 4 cells per axis): M's contributions
//     were computed speculatively in phase t-1 into a delta buffer; readers
//     add the delta, the accept items add it into storage only after the
//     readers signalled (per-level read epochs);
//   - expansions on finer levels: the expansion item reads storage before M's
//     update of its cell (the accept item of that cell waits for the read
//     epoch) and adds M's contribution to the value at its point through the
//     Legendre addition theorem, sum_n |d|^n / |s|^(n+1) P_n(cos g), which is
//     the same truncated series as the P2L coefficients (Eq. 2, Alg. L.2);
//   - cell lists: near-cell items skip the moved charge and add it at its new
//     position; the list update waits until every near item has read;
//   - H = R(K) and the dipole are double-buffered: readers use the current
//     buffer plus M's change, writers fill the other buffer.
// Every wait is bounded in time and only waits on items of lower index that
// never wait themselves, so no ordering of warps can deadlock.
#include "mc_dev.cuh"

namespace {

constexpr double kImageConstP = 6.0 + 8.0 / 1.7320508075688772 + 12.0 / 1.4142135623730951;
constexpr double kPiP = 3.141592653589793;
constexpr double kInfP = __builtin_huge_val();

struct Geo {
  int j;
  double q;
  double r[3], rn[3];
  int cf[3], cfn[3];
  bool outside;
};

__device__ __forceinline__ bool sq(int k) {
  int s = (int)sqrtf((float)k + 0.5f);
  return s * s == k;
}

__device__ __forceinline__ void p_prof(unsigned long long* prof, int type, unsigned long long t0) {
  const unsigned long long d = mc_globaltimer() - t0;
  atomicAdd(&prof[8 + type], d);
  atomicAdd(&prof[24 + type], 1ULL);
  atomicMax(&prof[40 + type], d);
}

// bounded wait until *w >= target; false (and status set) on timeout
__device__ __forceinline__ bool wait_geq(unsigned long long* w, unsigned long long target,
                                         int* status, long long wait_ns) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(w) : "memory");
  if (v < target) {
    const unsigned long long t0 = mc_globaltimer();
    unsigned spins = 0;
    while (true) {
      asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(w) : "memory");
      if (v >= target) break;
      if ((++spins & 63u) == 0u) {
        if ((long long)(mc_globaltimer() - t0) > wait_ns || *((volatile int*)status) != MCD_OK) {
          atomicExch(status, MCD_ERR_TIMEOUT);
          return false;
        }
      }
    }
  }
  asm volatile("fence.acq_rel.gpu;" ::: "memory");
  return true;
}

// truncated Legendre series sum_{n<=p} |d|^n / |s|^(n+1) P_n(d.s/(|d||s|))
template <typename T>
__device__ __forceinline__ T legendre_pair(int p, T dx, T dy, T dz, T sx, T sy, T sz) {
  const T d2 = dx * dx + dy * dy + dz * dz, s2 = sx * sx + sy * sy + sz * sz;
  const T is = mc_rsqrt(s2);
  // rho^n P_n(c) via u_n = ((2n-1) (d.s/s^2) u_{n-1} - (n-1) (d^2/s^2) u_{n-2}) / n
  const T a = (dx * sx + dy * sy + dz * sz) * (is * is), b = d2 * (is * is);
  T u0 = T(1), u1 = a, sum = T(1) + (p >= 1 ? a : T(0));
#pragma unroll
  for (int n = 2; n <= MC_PMAX; n++) {
    if (n <= p) {
      const T u2 = ((T)(2 * n - 1) * a * u1 - (T)(n - 1) * b * u0) * (T(1) / (T)n);
      sum += u2;
      u0 = u1;
      u1 = u2;
    }
  }
  return sum * is;
}

}  // namespace

template <typename TE>
__device__ __forceinline__ void chain_body_pipe(const McSys* __restrict__ sysp, RunParams& rp,
                                                const int nCTA, const int cta) {
  __shared__ McSys S;
  __shared__ HarmTabs<TE> tabs;
  __shared__ unsigned short il[8][189];
  __shared__ double stage[MC_WARPS][256];
  __shared__ double s_dE, s_logu, s_u;
  __shared__ Geo sg, smv;                                 // proposal, pending move
  __shared__ double s_off[2][MC_MAXLEV + 2][3];           // offsets of the proposal
  __shared__ double s_offm[2][MC_MAXLEV + 2][3];          // offsets of the pending move
  __shared__ double s_kw[MC_MAXLEV + 2][7];
  __shared__ TE s_kwe[MC_MAXLEV + 2][7];

  if (threadIdx.x == 0) S = *sysp;
  harm_tabs_init<TE>(&tabs);
  il_table_init(il);
  __syncthreads();
  for (int i = threadIdx.x; i < (MC_MAXLEV + 2) * 7; i += blockDim.x) {
    const int l = i / 7, k = i % 7 - 3;
    const double v = (l >= 1 && l <= S.L) ? k * S.lev_w[l] : 0.0;
    s_kw[l][k + 3] = v;
    s_kwe[l][k + 3] = (TE)v;
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, grp = lane >> 3;
  const int p = S.p, C = S.C, L = S.L;
  const bool pbc = (S.bc == 0);
  const int nWarpsTot = nCTA * MC_WARPS;
  const int nfc = rp.nf_cols;
  const int ls_end = S.ls_end;
  const size_t nsC = (size_t)S.nsmall * C;
  unsigned long long gen = 0;
  long long n_acc = 0, n_border = 0, steps_done = 0;
  const bool prof_on = rp.prof != nullptr;
  const bool prof_lead = prof_on && cta == 0 && threadIdx.x == 0;
  unsigned long long tp0 = 0, tp1 = 0;
  const unsigned long long t_begin = mc_globaltimer();
  unsigned long long* eflag = S.sync;      // [l]: last step whose level-l expansions were read
  unsigned long long* ncount = S.sync + 12;  // near-cell items that have read their lists
  unsigned long long cumN = 0;
  bool have_mv = false, stop = false;
  double mv_dE = 0.0;
  int hv = 0;  // current H / dipole buffer
  double* Hb[2] = {S.Hhat, S.Hhat2};
  double* Db[2] = {S.dipv, S.dipv2};

  for (long long t = 0;; t++) {
    const bool do_prop = (t < rp.nsteps) && !stop;
    if (!do_prop && !have_mv) break;
    const int buf = (int)(t & 1), mbuf = buf ^ 1;
    const unsigned long long epoch = (unsigned long long)t + 1ULL;
    if (prof_lead) tp0 = mc_globaltimer();
    // ------------------------------------------------ proposal of step t
    if (do_prop && warp == 0) {
      int j;
      double q = 0.0, uu = 0.5, r = 0.0, rn = 0.0, d = 0.0;
      bool out = false;
      mc_proposal_axis(rp.seed, (unsigned long long)(rp.step0 + t), rp.chain, S.n, rp.h,
                       lane < 3 ? lane : 0, &j, &d, lane == 3 ? &uu : nullptr);
      if (lane < 3) {
        if (have_mv && j == smv.j) {
          // the pending move's charge: its position is the move's target
          q = smv.q;
          r = smv.rn[lane];
        } else {
          const double4 pj = ldcg4(&S.ppos[j]);
          q = pj.w;
          r = lane == 0 ? pj.x : (lane == 1 ? pj.y : pj.z);
        }
        double x = __dadd_rn(r, d);
        if (pbc) {
          if (x < 0.0) x = __dadd_rn(x, S.a);
          if (x >= S.a) x = __dsub_rn(x, S.a);
        } else if (!(x >= 0.0 && x < S.a)) {
          out = true;
        }
        rn = x;
      }
      const bool any_out = __any_sync(0xffffffffu, lane < 3 && out);
      int cf = 0, cfn = 0;
      if (lane < 3) {
        cf = finest_coord(r, S.inv_wL, S.nL);
        cfn = any_out ? cf : finest_coord(rn, S.inv_wL, S.nL);
        sg.r[lane] = r;
        sg.rn[lane] = rn;
        sg.cf[lane] = cf;
        sg.cfn[lane] = cfn;
      }
      {
        const int side = lane >> 4, li = lane & 15;
        const int l = L - li;
#pragma unroll
        for (int ax = 0; ax < 3; ax++) {
          const double xo = __shfl_sync(0xffffffffu, r, ax), xn = __shfl_sync(0xffffffffu, rn, ax);
          const int co = __shfl_sync(0xffffffffu, cf, ax), cnn = __shfl_sync(0xffffffffu, cfn, ax);
          if (l >= 1 && l <= L && li <= L - 1) {
            const int c = (side ? cnn : co) >> (L - l);
            s_off[side][l][ax] = (side ? xn : xo) - ((double)c + 0.5) * S.lev_w[l];
          }
        }
      }
      if (lane == 0) {
        sg.j = j;
        sg.q = q;
        sg.outside = any_out;
      }
      if (lane == 3) s_u = uu;
    }
    __syncthreads();
    Geo g;
    if (do_prop) g = sg;
    else {
      g.j = -1;
      g.q = 0.0;
      g.outside = true;
      for (int k = 0; k < 3; k++) {
        g.r[k] = g.rn[k] = 0.0;
        g.cf[k] = g.cfn[k] = 0;
      }
    }
    Geo mv;
    if (have_mv) mv = smv;
    const double u = s_u;
    const bool nomove = do_prop && (g.r[0] == g.rn[0] && g.r[1] == g.rn[1] && g.r[2] == g.rn[2]);
    const bool same = (g.cf[0] == g.cfn[0] && g.cf[1] == g.cfn[1] && g.cf[2] == g.cfn[2]);
    const bool work = do_prop && !nomove && !g.outside;

    // ------------------------------------------------------- item layout
    const int nE = do_prop ? L - S.lmin + 1 : 0;
    const int nN = do_prop ? (same ? 27 : 54) : 0;
    const int nRB = (C + 31) / 32;
    const int nF = (do_prop && pbc) ? nRB * nfc : 0;
    const int nXU = do_prop ? 2 : 0;
    int nD = 0;  // speculative coarse-level deltas of step t
    if (do_prop && work)
      for (int l = S.lmin; l < ls_end; l++) nD += 95;
    const int ZCH = 1024;  // doubles per zero / apply item
    const int nZ = (do_prop && nsC) ? (int)((nsC + ZCH - 1) / ZCH) : 0;
    const int P0 = 0, PN = nE, PF = nE + nN, PX = PF + nF, PD = PX + nXU, PZ = PD + nD;
    const int nProp = PZ + nZ;
    // accept items of the pending move
    const int nAp = (have_mv && nsC) ? (int)((nsC + ZCH - 1) / ZCH) : 0;
    int lev_items[MC_MAXLEV + 2], lev_start[MC_MAXLEV + 2];
    const int nKH = (have_mv && pbc) ? (C + 31) / 32 : 0;
    int nA = nAp + nKH + (have_mv ? 1 : 0);
    const int A0 = nProp, AK = A0 + nAp, AB = AK + nKH, AT = AB + (have_mv ? 1 : 0);
    int nT = 0;
    if (have_mv) {
      for (int l = L; l >= ls_end; l--) {
        const int sh = L - l;
        const bool samel = ((mv.cf[0] >> sh) == (mv.cfn[0] >> sh)) &&
                           ((mv.cf[1] >> sh) == (mv.cfn[1] >> sh)) &&
                           ((mv.cf[2] >> sh) == (mv.cfn[2] >> sh));
        lev_items[l] = samel ? 189 : 378;
        lev_start[l] = AT + nT;
        nT += lev_items[l];
      }
    }
    nA += nT;
    const int nItems = nProp + nA;
    const unsigned long long cumN_now = cumN + (unsigned long long)nN;
    double* part = S.partials + buf * MC_MAX_ITEMS;
    double* dcur = S.dsmall + (size_t)(t % 3) * nsC;            // delta of step t
    double* dmv = S.dsmall + (size_t)((t + 2) % 3) * nsC;       // delta of step t-1
    double* dzero = S.dsmall + (size_t)((t + 1) % 3) * nsC;     // cleared for step t+1

    // item schedule: with many CTAs the items the decision waits for (E, N,
    // F, X, U: indices below PD) run alone on warp 0 of each CTA (warp 4,
    // which shares its SM sub-partition, stays idle); the rest run on warps
    // 1-3 and 5-7.  Each warp takes its items in increasing index order.
    const bool split = nCTA >= 64;
    int it0, istep;
    if (!split) {
      it0 = warp * nCTA + cta;
      istep = nWarpsTot;
    } else if (warp == 0) {
      it0 = cta;
      istep = nCTA;
    } else if (warp == 4) {
      it0 = nItems;
      istep = 1;
    } else {
      const int ws = warp < 4 ? warp - 1 : warp - 2;
      it0 = PD + ws * nCTA + cta;
      istep = 6 * nCTA;
    }
    for (int it = it0; it < nItems; it += istep) {
      if (split && warp == 0 && it >= PD) break;
      const unsigned long long t_item = prof_on ? mc_globaltimer() : 0ULL;
      int ptype = -1;
      if (it < PN) {
        // ---- E: level expansion at r (group 0) and r' (group 1) of level l
        ptype = 0;
        const int l = L - (it - P0), sh = L - l;
        const int side = grp & 1;
        const int* cc = side ? g.cfn : g.cf;
        const int c3[3] = {cc[0] >> sh, cc[1] >> sh, cc[2] >> sh};
        const int nl = S.lev_n[l];
        const int cell = (c3[0] * nl + c3[1]) * nl + c3[2];
        const double* Lb = S.Lhat + (size_t)(S.lev_off[l] + cell) * C;
        const bool small = l < ls_end;
        const double* Db2 = dmv + (size_t)(S.lev_off[l] + cell) * C;
        double ld[MC_PMAX + 2], lid[MC_PMAX + 2];
#pragma unroll
        for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
          int n, m;
          bool v;
          group_nm(p, t2, &n, &m, &v);
          const int k = rl_re(n, m);
          double a = v ? __ldcg(&Lb[k]) : 0.0, b = (v && m) ? __ldcg(&Lb[k + 1]) : 0.0;
          if (small && have_mv && v) {
            a += __ldcg(&Db2[k]);
            if (m) b += __ldcg(&Db2[k + 1]);
          }
          ld[t2] = a;
          lid[t2] = b;
        }
        TE Lr[MC_PMAX + 2], Li[MC_PMAX + 2];
#pragma unroll
        for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
          Lr[t2] = from_double<TE>(ld[t2]);
          Li[t2] = from_double<TE>(lid[t2]);
        }
        // the storage of this level has been read: the pending move may now update it
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(&eflag[l]), "l"(epoch) : "memory");
        }
        TE acc = TE(0);
        if (work) {
          const TE dx = from_double<TE>(s_off[side][l][0]), dy = from_double<TE>(s_off[side][l][1]),
                   dz = from_double<TE>(s_off[side][l][2]);
          regular_group<TE>(&tabs, p, dx, dy, dz, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
            if (v) acc += (m ? TE(2) : TE(1)) * (Lr[t2] * vr - Li[t2] * vi);
          });
          acc = group_sum(acc);
          // pending move on a finer level: its contribution to this cell
          // (at most one image per side), by the Legendre addition theorem
          if (have_mv && !small) {
            const int g8 = lane & 7;
            TE corr = TE(0);
            if (g8 < 2) {
              const int ms = g8;  // 0: old position (-q), 1: new position (+q)
              const int* mcs = ms ? mv.cfn : mv.cf;
              const int b3[3] = {mcs[0] >> sh, mcs[1] >> sh, mcs[2] >> sh};
              for (int s = 0; s < 27; s++) {
                const int sx = s / 9 - 1, sy = (s / 3) % 3 - 1, sz = s % 3 - 1;
                if (!pbc && (sx || sy || sz)) continue;
                const int o0 = c3[0] + sx * nl - b3[0], o1 = c3[1] + sy * nl - b3[1],
                          o2 = c3[2] + sz * nl - b3[2];
                if (in_il(o0, o1, o2, b3[0], b3[1], b3[2])) {
                  TE ex, ey, ez;
                  if (sizeof(TE) == 8) {
                    ex = (TE)(s_offm[ms][l][0] - s_kw[l][o0 + 3]);
                    ey = (TE)(s_offm[ms][l][1] - s_kw[l][o1 + 3]);
                    ez = (TE)(s_offm[ms][l][2] - s_kw[l][o2 + 3]);
                  } else {
                    ex = from_double<TE>(s_offm[ms][l][0]) - s_kwe[l][o0 + 3];
                    ey = from_double<TE>(s_offm[ms][l][1]) - s_kwe[l][o1 + 3];
                    ez = from_double<TE>(s_offm[ms][l][2]) - s_kwe[l][o2 + 3];
                  }
                  const TE val = legendre_pair<TE>(p, dx, dy, dz, ex, ey, ez);
                  corr += ms ? val : -val;
                }
              }
              corr *= from_double<TE>(mv.q);
            }
            corr += __shfl_xor_sync(0xffffffffu, corr, 1);
            acc += corr;
          }
        }
        const TE accn = __shfl_sync(0xffffffffu, acc, 8);
        const double partial = work ? g.q * to_double(accn - acc) : 0.0;
        if (lane == 0) part[it] = partial;
      } else if (it < PF) {
        // ---- N: Alg. 1 over one near cell, with the pending move applied
        ptype = 1;
        const int k0 = it - PN;
        const int k = same ? k0 : (k0 % 27);
        const int side = same ? 2 : (k0 / 27);  // 0 old, 1 new, 2 both
        const int* cc = (side == 1) ? g.cfn : g.cf;
        const int e0 = cc[0] + k / 9 - 1, e1 = cc[1] + (k / 3) % 3 - 1, e2 = cc[2] + k % 3 - 1;
        const int nL = S.nL;
        bool valid = true;
        int c0, c1, c2, s0 = 0, s1 = 0, s2 = 0;
        if (pbc) {
          c0 = mc_wrap_coord(e0, nL);
          c1 = mc_wrap_coord(e1, nL);
          c2 = mc_wrap_coord(e2, nL);
          s0 = (e0 - c0) / nL;
          s1 = (e1 - c1) / nL;
          s2 = (e2 - c2) / nL;
        } else {
          valid = (e0 >= 0 && e0 < nL && e1 >= 0 && e1 < nL && e2 >= 0 && e2 < nL);
          c0 = e0;
          c1 = e1;
          c2 = e2;
        }
        double partial = 0.0;
        bool ovl = false;
        const int cell = valid ? (c0 * nL + c1) * nL + c2 : 0;
        const int cnt = valid ? __ldcg(&S.ccount[cell]) : 0;
        const bool zero_shift = (s0 == 0 && s1 == 0 && s2 == 0);
        const int mj = have_mv ? mv.j : -1;
        // the moved charge's new cell is this one: it is added here
        const bool add_mv = have_mv && valid &&
                            ((mv.cfn[0] * nL + mv.cfn[1]) * nL + mv.cfn[2]) == cell;
        if (sizeof(TE) == 8) {
          const double sx = s0 * S.a, sy = s1 * S.a, sz = s2 * S.a;
          const double ox = g.r[0] - sx, oy = g.r[1] - sy, oz = g.r[2] - sz;
          const double nx = g.rn[0] - sx, ny = g.rn[1] - sy, nz = g.rn[2] - sz;
          double acc = 0.0;
          for (int s = lane; s < cnt + 1; s += 32) {
            double4 xi;
            int pid;
            if (s < cnt) {
              xi = ldcg4(&S.cpos[(size_t)cell * S.cap + s]);
              pid = __ldcg(&S.cpid[(size_t)cell * S.cap + s]);
              if (pid == mj) continue;
            } else {
              if (!add_mv) continue;
              xi = make_double4(mv.rn[0], mv.rn[1], mv.rn[2], mv.q);
              pid = mj;
            }
            if (!work) continue;
            if (side != 1 && !(pid == g.j && zero_shift)) {
              const double ax = ox - xi.x, ay = oy - xi.y, az = oz - xi.z;
              acc -= g.q * xi.w * rsqrt(ax * ax + ay * ay + az * az);
            }
            if (side != 0) {
              const double bx = nx - xi.x, by = ny - xi.y, bz = nz - xi.z;
              const double d2 = bx * bx + by * by + bz * bz;
              if (d2 == 0.0) ovl = true;
              acc += g.q * xi.w * rsqrt(d2);
            }
          }
          partial = warp_sum(acc);
        } else {
          const int oo0 = e0 - g.cf[0], oo1 = e1 - g.cf[1], oo2 = e2 - g.cf[2];
          const int on0 = e0 - g.cfn[0], on1 = e1 - g.cfn[1], on2 = e2 - g.cfn[2];
          const double wL = S.lev_w[L];
          const float ox = d2f_int(s_off[0][L][0] - oo0 * wL), oy = d2f_int(s_off[0][L][1] - oo1 * wL),
                      oz = d2f_int(s_off[0][L][2] - oo2 * wL);
          const float nx = d2f_int(s_off[1][L][0] - on0 * wL), ny = d2f_int(s_off[1][L][1] - on1 * wL),
                      nz = d2f_int(s_off[1][L][2] - on2 * wL);
          const float qf = d2f_int(g.q);
          float acc = 0.0f;
          for (int s = lane; s < cnt + 1; s += 32) {
            float4 xi;
            int pid;
            if (s < cnt) {
              xi = __ldcg(&S.cpos32[(size_t)cell * S.cap + s]);
              pid = __ldcg(&S.cpid[(size_t)cell * S.cap + s]);
              if (pid == mj) continue;
            } else {
              if (!add_mv) continue;
              xi = make_float4(d2f_int(s_offm[1][L][0]), d2f_int(s_offm[1][L][1]),
                               d2f_int(s_offm[1][L][2]), d2f_int(mv.q));
              pid = mj;
            }
            if (!work) continue;
            if (side != 1 && !(pid == g.j && zero_shift)) {
              const float ax = ox - xi.x, ay = oy - xi.y, az = oz - xi.z;
              acc -= qf * xi.w * rsqrtf(ax * ax + ay * ay + az * az);
            }
            if (side != 0) {
              const float bx = nx - xi.x, by = ny - xi.y, bz = nz - xi.z;
              const float d2 = bx * bx + by * by + bz * bz;
              if (d2 == 0.0f) ovl = true;
              acc += qf * xi.w * rsqrtf(d2);
            }
          }
          partial = f2d_int(warp_sum(acc));
        }
        if (__any_sync(0xffffffffu, ovl)) partial = kInfP;
        // this cell's list has been read: the pending move may now update lists
        __syncwarp();
        if (lane == 0) {
          __threadfence();
          atomicAdd(ncount, 1ULL);
          part[it] = work ? partial : 0.0;
        }
      } else if (it < PX) {
        // ---- F: far lattice (Sec. 3.3 iv, factored), H after the pending move
        ptype = 2;
        const int f = it - PF;
        const int rb = f / nfc, cb = f % nfc;
        double* st = stage[warp];
        double contrib = 0.0;
        if (work) {
          const double c1 = 0.5 * S.a;
          const TE qe = from_double<TE>(g.q);
          const double* xg = (grp & 1) ? g.rn : g.r;
          const TE dx = from_double<TE>(xg[0] - c1), dy = from_double<TE>(xg[1] - c1),
                   dz = from_double<TE>(xg[2] - c1);
          regular_group<TE>(&tabs, p, dx, dy, dz, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
            const TE nr = __shfl_xor_sync(0xffffffffu, vr, 8);
            const TE ni = __shfl_xor_sync(0xffffffffu, vi, 8);
            if (grp == 0 && v) {
              const int k = rl_re(n, m);
              st[k] = to_double(qe * (nr - vr));
              if (m) st[k + 1] = to_double(-qe * (ni - vi));
            }
          });
          __syncwarp();
          const int csz = (C + nfc - 1) / nfc;
          const int cbeg = cb * csz, cend = min(C, cbeg + csz);
          const int k = rb * 32 + lane;
          if (k < C) {
            double gk = 0.0;
            for (int c = cbeg; c < cend; c++) gk += S.G[(size_t)c * C + k] * st[c];
            S.gK[(size_t)buf * MC_NF_COLS * C + (size_t)cb * C + k] = gk;
            double hk = 0.0;
            if (cb == 0) {
              hk = __ldcg(&Hb[hv][k]);
              if (have_mv)
                for (int c2 = 0; c2 < nfc; c2++)
                  hk += __ldcg(&S.gK[(size_t)mbuf * MC_NF_COLS * C + (size_t)c2 * C + k]);
            }
            contrib = (sq(k) ? 1.0 : 2.0) * st[k] * (0.5 * gk + hk);
          }
          if (f == 0)
            for (int kk = lane; kk < C; kk += 32) S.dK[(size_t)buf * C + kk] = st[kk];
        }
        const double partial = warp_sum(contrib);
        __syncwarp();
        if (lane == 0) part[it] = partial;
      } else if (it < PD) {
        if (it == PX) {
          // ---- X: periodic self-interaction correction and dipole term
          ptype = 3;
          double partial = 0.0;
          if (g.outside) {
            partial = kInfP;
          } else if (work) {
            const TE q2 = from_double<TE>(g.q * g.q);
            const TE ddx = from_double<TE>(g.rn[0] - g.r[0]), ddy = from_double<TE>(g.rn[1] - g.r[1]),
                     ddz = from_double<TE>(g.rn[2] - g.r[2]);
            const TE ae = from_double<TE>(S.a);
            TE v = TE(0);
            if (pbc) {
              if (lane < 27) {
                const TE ax = ddx - TE(lane / 9 - 1) * ae;
                const TE ay = ddy - TE((lane / 3) % 3 - 1) * ae;
                const TE az = ddz - TE(lane % 3 - 1) * ae;
                v = -q2 * mc_rsqrt(ax * ax + ay * ay + az * az);
              }
            } else if (lane == 0) {
              v = -q2 * mc_rsqrt(ddx * ddx + ddy * ddy + ddz * ddz);
            }
            partial = to_double(warp_sum(v));
            if (pbc) {
              partial += g.q * g.q / S.a * kImageConstP;
              if (S.dip == 0) {
                const double cdip = -2.0 * kPiP / (3.0 * S.V);
                double D2 = 0.0, Dn2 = 0.0;
#pragma unroll
                for (int kk = 0; kk < 3; kk++) {
                  double D = __ldcg(&Db[hv][kk]);
                  if (have_mv) D += mv.q * (mv.rn[kk] - mv.r[kk]);
                  const double Dn = D + g.q * (g.rn[kk] - g.r[kk]);
                  D2 += D * D;
                  Dn2 += Dn * Dn;
                }
                partial += cdip * Dn2 - cdip * D2;
              }
            }
          }
          if (lane == 0) part[it] = partial;
        } else {
          // ---- U: log(u)
          ptype = 3;
          if (lane == 0) {
            part[it] = 0.0;
            part[MC_MAX_ITEMS - 1] = log(u);
          }
        }
      } else if (it < PZ) {
        // ---- D: speculative coarse-level contributions of step t (Alg. L.2
        //      entries 2k and 2k+1 of IL(alpha) and IL(alpha') per warp)
        ptype = 4;
        int rem = it - PD, l = S.lmin;
        while (rem >= 95) {
          rem -= 95;
          l++;
        }
        const int k = rem, sh = L - l, nl = S.lev_n[l];
        const int side = grp & 1;
        const int entry = 2 * k + (grp >> 1);
        const int* cs0 = side ? g.cfn : g.cf;
        const int cs[3] = {cs0[0] >> sh, cs0[1] >> sh, cs0[2] >> sh};
        const int par = ((cs[0] & 1) << 2) | ((cs[1] & 1) << 1) | (cs[2] & 1);
        int ox = 0, oy = 0, oz = 0;
        if (entry < 189) il_unpack(il[par][entry], &ox, &oy, &oz);
        const int e[3] = {cs[0] + ox, cs[1] + oy, cs[2] + oz};
        const bool valid = entry < 189 && (pbc || (e[0] >= 0 && e[0] < nl && e[1] >= 0 &&
                                                   e[1] < nl && e[2] >= 0 && e[2] < nl));
        const int t3[3] = {mc_wrap_coord(e[0], nl), mc_wrap_coord(e[1], nl), mc_wrap_coord(e[2], nl)};
        const TE f = valid ? from_double<TE>(side ? g.q : -g.q) : TE(0);
        TE dx = TE(3), dy = TE(3), dz = TE(3);
        if (valid) {
          if (sizeof(TE) == 8) {
            dx = (TE)(s_off[side][l][0] - s_kw[l][ox + 3]);
            dy = (TE)(s_off[side][l][1] - s_kw[l][oy + 3]);
            dz = (TE)(s_off[side][l][2] - s_kw[l][oz + 3]);
          } else {
            dx = from_double<TE>(s_off[side][l][0]) - s_kwe[l][ox + 3];
            dy = from_double<TE>(s_off[side][l][1]) - s_kwe[l][oy + 3];
            dz = from_double<TE>(s_off[side][l][2]) - s_kwe[l][oz + 3];
          }
        }
        double* Dt = dcur + (size_t)(S.lev_off[l] + (t3[0] * nl + t3[1]) * nl + t3[2]) * C;
        irregular_group<TE>(&tabs, p, dx, dy, dz, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
          if (valid && v) {
            const int kk = rl_re(n, m);
            atomicAdd(&Dt[kk], to_double(f * vr));
            if (m) atomicAdd(&Dt[kk + 1], to_double(-f * vi));
          }
        });
      } else if (it < nProp) {
        // ---- Z: clear the delta buffer of step t+1
        ptype = 4;
        const size_t b0 = (size_t)(it - PZ) * ZCH;
        for (size_t i = b0 + lane; i < min(nsC, b0 + ZCH); i += 32) __stcg(&dzero[i], 0.0);
      } else if (it < AK) {
        // ---- Ap: add the pending move's coarse-level delta to storage once
        //          this step's coarse-level expansion items have read it
        ptype = 5;
        bool ok = true;
        if (do_prop && lane == 0)
          for (int l = S.lmin; l < ls_end && ok; l++)
            ok = wait_geq(&eflag[l], epoch, S.status, rp.wait_ns);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) {
          const size_t b0 = (size_t)(it - A0) * ZCH;
          for (size_t i = b0 + lane; i < min(nsC, b0 + ZCH); i += 32)
            __stcg(&S.Lhat[i], __ldcg(&S.Lhat[i]) + __ldcg(&dmv[i]));
        }
      } else if (it < AB) {
        // ---- K += dK, H(other buffer) = H + G dK of the pending move
        ptype = 6;
        const int k = (it - AK) * 32 + lane;
        if (k < C) {
          double gv[MC_NF_COLS];
#pragma unroll
          for (int cb = 0; cb < MC_NF_COLS; cb++)
            gv[cb] = cb < nfc ? __ldcg(&S.gK[(size_t)mbuf * MC_NF_COLS * C + (size_t)cb * C + k]) : 0.0;
          const double dk = __ldcg(&S.dK[(size_t)mbuf * C + k]);
          const double kh = __ldcg(&S.Khat[k]), hh = __ldcg(&Hb[hv][k]);
          double gs = 0.0;
#pragma unroll
          for (int cb = 0; cb < MC_NF_COLS; cb++)
            if (cb < nfc) gs += gv[cb];
          __stcg(&S.Khat[k], kh + dk);
          __stcg(&Hb[hv ^ 1][k], hh + gs);
        }
      } else if (it < AT) {
        // ---- bookkeeping of the pending move: waits until every near-cell
        //      item of step t has read its list
        ptype = 6;
        bool ok = true;
        if (lane == 0 && nN) ok = wait_geq(ncount, cumN_now, S.status, rp.wait_ns);
        ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
        if (ok) {
          const int nL = S.nL, cap = S.cap;
          const int co = (mv.cf[0] * nL + mv.cf[1]) * nL + mv.cf[2];
          const int cn = (mv.cfn[0] * nL + mv.cfn[1]) * nL + mv.cfn[2];
          int so = 0, cnt_o = 0, cnt_n = 0;
          if (lane == 0) so = S.pslot[mv.j];
          if (lane == 1) cnt_o = S.ccount[co];
          if (lane == 2) cnt_n = S.ccount[cn];
          so = __shfl_sync(0xffffffffu, so, 0);
          cnt_o = __shfl_sync(0xffffffffu, cnt_o, 1);
          cnt_n = __shfl_sync(0xffffffffu, cnt_n, 2);
          const double4 np = make_double4(mv.rn[0], mv.rn[1], mv.rn[2], mv.q);
          const float4 rel = make_float4(d2f_int(s_offm[1][L][0]), d2f_int(s_offm[1][L][1]),
                                         d2f_int(s_offm[1][L][2]), d2f_int(mv.q));
          if (co == cn) {
            if (lane == 0) S.cpos[so] = np;
            if (lane == 1) S.cpos32[so] = rel;
          } else {
            const int last = cnt_o - 1;
            const int sl = co * cap + last;
            if (so != sl) {
              double4 v4 = make_double4(0, 0, 0, 0);
              float4 f4 = make_float4(0, 0, 0, 0);
              int pid = 0;
              if (lane == 0) v4 = S.cpos[sl];
              if (lane == 1) f4 = S.cpos32[sl];
              if (lane == 2) pid = S.cpid[sl];
              pid = __shfl_sync(0xffffffffu, pid, 2);
              if (lane == 0) S.cpos[so] = v4;
              if (lane == 1) S.cpos32[so] = f4;
              if (lane == 2) {
                S.cpid[so] = pid;
                S.pslot[pid] = so;
              }
            }
            if (lane == 3) S.ccount[co] = last;
            if (cnt_n >= cap) {
              if (lane == 0) atomicExch(S.status, MCD_ERR_CAPACITY);
            } else {
              const int slot = cn * cap + cnt_n;
              if (lane == 0) S.cpos[slot] = np;
              if (lane == 1) S.cpos32[slot] = rel;
              if (lane == 2) S.cpid[slot] = mv.j;
              if (lane == 4) S.pslot[mv.j] = slot;
              if (lane == 5) S.ccount[cn] = cnt_n + 1;
            }
          }
          if (lane == 6) S.ppos[mv.j] = np;
          if (lane == 7) S.energy[0] += mv_dE;
          if (lane >= 8 && lane < 11)
            Db[hv ^ 1][lane - 8] = __ldcg(&Db[hv][lane - 8]) + mv.q * (mv.rn[lane - 8] - mv.r[lane - 8]);
        }
      } else {
        // ---- Alg. L.2 on a finer level: one target cell of the pending move
        ptype = 5;
        int l = L;
        while (l > ls_end && it >= lev_start[l] + lev_items[l]) l--;
        const int k = it - lev_start[l];
        const int sh = L - l, nl = S.lev_n[l];
        const int co[3] = {mv.cf[0] >> sh, mv.cf[1] >> sh, mv.cf[2] >> sh};
        const int cn[3] = {mv.cfn[0] >> sh, mv.cfn[1] >> sh, mv.cfn[2] >> sh};
        int tc[3];
        bool owner = true;
        const bool samel = lev_items[l] == 189;
        const bool from_new = samel || (k < 189);
        int o_known[3];
        {
          const int kk = (k < 189) ? k : k - 189;
          const int* base = from_new ? cn : co;
          const int par = ((base[0] & 1) << 2) | ((base[1] & 1) << 1) | (base[2] & 1);
          int ox, oy, oz;
          il_unpack(il[par][kk], &ox, &oy, &oz);
          o_known[0] = ox;
          o_known[1] = oy;
          o_known[2] = oz;
          const int e[3] = {base[0] + ox, base[1] + oy, base[2] + oz};
          if (!pbc && (e[0] < 0 || e[0] >= nl || e[1] < 0 || e[1] >= nl || e[2] < 0 || e[2] >= nl))
            owner = false;
          for (int d = 0; d < 3; d++) tc[d] = mc_wrap_coord(e[d], nl);
          if (owner && !from_new) {
            for (int s = 0; s < 27 && owner; s++) {
              const int sx = s / 9 - 1, sy = (s / 3) % 3 - 1, sz = s % 3 - 1;
              if (!pbc && (sx || sy || sz)) continue;
              if (in_il(tc[0] + sx * nl - cn[0], tc[1] + sy * nl - cn[1], tc[2] + sz * nl - cn[2],
                        cn[0], cn[1], cn[2]))
                owner = false;
            }
          }
        }
        if (owner) {
          const int side = grp & 1;
          const int* cs = side ? cn : co;
          int ofs[3] = {o_known[0], o_known[1], o_known[2]};
          bool have;
          if (samel || (from_new && side == 1) || (!from_new && side == 0)) {
            have = true;
          } else if (!from_new) {
            have = false;
          } else {
            have = false;
            for (int s = 0; s < 27 && !have; s++) {
              const int sx = s / 9 - 1, sy = (s / 3) % 3 - 1, sz = s % 3 - 1;
              if (!pbc && (sx || sy || sz)) continue;
              const int o0 = tc[0] + sx * nl - cs[0], o1 = tc[1] + sy * nl - cs[1],
                        o2 = tc[2] + sz * nl - cs[2];
              if (in_il(o0, o1, o2, cs[0], cs[1], cs[2])) {
                have = true;
                ofs[0] = o0;
                ofs[1] = o1;
                ofs[2] = o2;
              }
            }
          }
          const TE f = have ? from_double<TE>(side ? mv.q : -mv.q) : TE(0);
          TE dx = TE(3), dy = TE(3), dz = TE(3);
          if (have) {
            if (sizeof(TE) == 8) {
              dx = (TE)(s_offm[side][l][0] - s_kw[l][ofs[0] + 3]);
              dy = (TE)(s_offm[side][l][1] - s_kw[l][ofs[1] + 3]);
              dz = (TE)(s_offm[side][l][2] - s_kw[l][ofs[2] + 3]);
            } else {
              dx = from_double<TE>(s_offm[side][l][0]) - s_kwe[l][ofs[0] + 3];
              dy = from_double<TE>(s_offm[side][l][1]) - s_kwe[l][ofs[1] + 3];
              dz = from_double<TE>(s_offm[side][l][2]) - s_kwe[l][ofs[2] + 3];
            }
          }
          double* st = stage[warp];
          irregular_group<TE>(&tabs, p, dx, dy, dz, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
            const TE cr = f * vr, ci = -f * vi;
            const TE orr = __shfl_xor_sync(0xffffffffu, cr, 8);
            const TE oii = __shfl_xor_sync(0xffffffffu, ci, 8);
            if (grp == 0 && v) {
              const int kk = rl_re(n, m);
              st[kk] = to_double(cr + orr);
              if (m) st[kk + 1] = to_double(ci + oii);
            }
          });
          __syncwarp();
          // a cell that this step's expansion item reads is updated only
          // after that item has read it
          bool ok = true;
          if (do_prop) {
            const int* a0 = g.cf;
            const int* a1 = g.cfn;
            const bool claimed =
                ((a0[0] >> sh) == tc[0] && (a0[1] >> sh) == tc[1] && (a0[2] >> sh) == tc[2]) ||
                ((a1[0] >> sh) == tc[0] && (a1[1] >> sh) == tc[1] && (a1[2] >> sh) == tc[2]);
            if (claimed && lane == 0) ok = wait_geq(&eflag[l], epoch, S.status, rp.wait_ns);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
          }
          if (ok) {
            double* Lt = S.Lhat + (size_t)(S.lev_off[l] + (tc[0] * nl + tc[1]) * nl + tc[2]) * C;
            double vv[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
              const int kk = lane + 32 * i;
              vv[i] = kk < C ? __ldcg(&Lt[kk]) : 0.0;
            }
#pragma unroll
            for (int i = 0; i < 8; i++) {
              const int kk = lane + 32 * i;
              if (kk < C) __stcg(&Lt[kk], vv[i] + st[kk]);
            }
          }
          __syncwarp();
        }
      }
      if (prof_on && lane == 0 && ptype >= 0) p_prof(rp.prof, ptype, t_item);
    }
    cumN = cumN_now;

    if (prof_lead) {
      tp1 = mc_globaltimer();
      rp.prof[0] += tp1 - tp0;
    }
    gen++;
    if (!grid_barrier(S.bar, gen * (unsigned long long)(nCTA + rp.bar_missing), S.status, rp.wait_ns)) break;
    if (prof_lead) {
      tp0 = mc_globaltimer();
      rp.prof[1] += tp0 - tp1;
    }
    if (have_mv) {
      hv ^= 1;
      have_mv = false;
    }
    if (!do_prop) break;

    // ------------------------------------------------ decision of step t
    if (warp == 0) {
      double acc = 0.0;
      for (int i = lane; i < nProp; i += 32) acc += (i < PD) ? __ldcg(&part[i]) : 0.0;
      acc = warp_sum(acc);
      if (lane == 0) {
        s_dE = acc;
        s_logu = __ldcg(&part[MC_MAX_ITEMS - 1]);
      }
    }
    __syncthreads();
    const double dE = s_dE;
    bool accept;
    if (dE <= 0.0) {
      accept = true;
    } else {
      const double t2 = -rp.beta * dE;
      accept = s_logu < t2;
      if (fabs(s_logu - t2) < 1e-9 * fmax(1.0, fabs(t2))) n_border++;
    }
    if (cta == 0 && threadIdx.x == 0 && rp.log_j) {
      rp.log_j[t] = g.j;
      rp.log_dE[t] = dE;
      rp.log_acc[t] = accept ? 1 : 0;
    }
    steps_done++;
    if (prof_lead) {
      rp.prof[2] += mc_globaltimer() - tp0;
      rp.prof[5] += 1;
    }
    if (accept) {
      n_acc++;
      if (!nomove) {
        have_mv = true;
        mv_dE = dE;
        if (threadIdx.x == 0) smv = sg;
        for (int i = threadIdx.x; i < 2 * (MC_MAXLEV + 2) * 3; i += blockDim.x)
          (&s_offm[0][0][0])[i] = (&s_off[0][0][0])[i];
        if (prof_lead) rp.prof[6] += 1;
      }
      if (rp.stop_after_accepts > 0 && n_acc >= rp.stop_after_accepts) stop = true;
    }
    __syncthreads();
  }
  // leave the current H and dipole in the first buffers for the other paths
  if (hv == 1 && cta == 0) {
    __syncthreads();
    for (int k = threadIdx.x; k < C; k += blockDim.x) S.Hhat[k] = __ldcg(&S.Hhat2[k]);
    if (threadIdx.x < 3) S.dipv[threadIdx.x] = __ldcg(&S.dipv2[threadIdx.x]);
  }
  if (cta == 0 && threadIdx.x == 0) {
    S.stats[0] = steps_done;
    S.stats[1] = n_acc;
    S.stats[2] = n_border;
    S.stats[3] = (long long)(mc_globaltimer() - t_begin);
  }
}

template <typename TE>
__global__ void __launch_bounds__(MC_THREADS, 1)
    mc_pipe_kernel(const McSys* __restrict__ sysp, RunParams rp) {
  chain_body_pipe<TE>(sysp, rp, (int)gridDim.x, (int)blockIdx.x);
}

template <typename TE>
__global__ void __launch_bounds__(MC_THREADS, MC_BATCH_CTAS_PER_SM(TE))
    mc_batch_pipe_kernel(const McSys* const* __restrict__ systems, RunParams* __restrict__ rps,
                         const int* __restrict__ cta_chain, const int* __restrict__ cta_rank,
                         const int* __restrict__ chain_ctas) {
  const int ch = cta_chain[blockIdx.x];
  RunParams rp = rps[ch];
  const McSys* sys = systems[ch];
  chain_body_pipe<TE>(sys, rp, chain_ctas[ch], cta_rank[blockIdx.x]);
  if (cta_rank[blockIdx.x] == 0 && threadIdx.x == 0) {
    const long long done = sys->stats[0];
    if (done > 0) rps[ch].step0 = rp.step0 + done;
  }
}

cudaError_t mc_launch_pipe(const McSys* d_sys, const RunParams& rp, int prec, int nCTA,
                           cudaStream_t stream) {
  void* args[] = {(void*)&d_sys, (void*)&rp};
  const void* fn = prec ? (const void*)mc_pipe_kernel<float> : (const void*)mc_pipe_kernel<double>;
  return cudaLaunchCooperativeKernel(fn, dim3(nCTA), dim3(MC_THREADS), args, 0, stream);
}

cudaError_t mc_launch_batch_pipe(const McSys* const* d_systems, RunParams* d_rps,
                                 const int* d_cta_chain, const int* d_cta_rank,
                                 const int* d_chain_ctas, int prec, int nCTA, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nCTA);
  cfg.blockDim = dim3(MC_THREADS);
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (prec)
    return cudaLaunchKernelEx(&cfg, mc_batch_pipe_kernel<float>, d_systems, d_rps, d_cta_chain,
                              d_cta_rank, d_chain_ctas);
  return cudaLaunchKernelEx(&cfg, mc_batch_pipe_kernel<double>, d_systems, d_rps, d_cta_chain,
                            d_cta_rank, d_chain_ctas);
}

// CTAs per SM the pipelined batch kernel of this precision can keep resident
int mc_batch_pipe_ctas_per_sm(int prec) {
  int per = 0;
  const void* fn = prec ? (const void*)mc_batch_pipe_kernel<float> : (const void*)mc_batch_pipe_kernel<double>;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, MC_THREADS, 0) != cudaSuccess) return 0;
  return per;
}
