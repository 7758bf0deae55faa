// Persistent Metropolis-Hastings chain kernel: one cooperative launch runs
// many steps of Alg. L.1 (propose, with Alg. 1 and the periodic terms of
// Sec. 3.3) and Alg. L.2 (accept) for one system on the whole GPU.
//
// One step:
//   1. every thread draws the same Philox proposal (j, r -> r');
//   2. propose items, one warp each, spread over the SMs:
//        E  level expansions (Eq. 1/2) at r and r' on level l
//        N  direct sum over one of the 27 near cells (Alg. 1)
//        F  far lattice term: dK and a 32-row x C/8-column block of G dK
//        X  image self-interaction correction, dipole term, log(u)
//      each writes one partial sum;
//   3. grid barrier;
//   4. every CTA reduces the partials in the same fixed order -> dE and the
//      Metropolis decision (identical in every CTA, no broadcast needed);
//   5. on accept: target items (one warp per updated cell of each level's
//      interaction lists, Alg. L.2) and one bookkeeping item (K, H, dipole,
//      energy, cell lists); then a second grid barrier.
// Template TE is the evaluation type: double (FP64 form) or float (FP32-eval
// form: harmonics and near field in FP32; FP64 accumulators, energy, far
// lattice operator, decision).
#include "mc_dev.cuh"

namespace {

constexpr double kImageConst = 6.0 + 8.0 / 1.7320508075688772 + 12.0 / 1.4142135623730951;
constexpr double kPi = 3.141592653589793;

struct StepGeo {
  int j;
  double q;
  double r[3], rn[3];
  int cf[3], cfn[3];
  bool same;
  bool outside;  // free space: r' left the box
};

__device__ __forceinline__ bool is_square(int k) {
  int s = (int)sqrtf((float)k + 0.5f);
  return s * s == k;
}

}  // namespace

template <typename TE>
__global__ void __launch_bounds__(MC_THREADS, 1)
    mc_chain_kernel(const McSys* __restrict__ sysp, RunParams rp) {
  __shared__ McSys S;
  __shared__ HarmTabs<TE> tabs;
  __shared__ unsigned short il[8][189];
  __shared__ double stage[MC_WARPS][256];
  __shared__ double s_dE, s_logu;

  if (threadIdx.x == 0) S = *sysp;
  harm_tabs_init<TE>(&tabs);
  il_table_init(il);
  __syncthreads();

  const int nCTA = gridDim.x, cta = blockIdx.x;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int half = lane >> 4, hm = lane & 15;
  const int p = S.p, C = S.C, L = S.L;
  const bool pbc = (S.bc == 0);
  const int nWarpsTot = nCTA * MC_WARPS;
  unsigned long long gen = 0;
  long long n_acc = 0, n_border = 0, steps_done = 0;

  for (long long t = 0; t < rp.nsteps; t++) {
    const int buf = (int)(t & 1);
    // ------------------------------------------------------------ proposal
    StepGeo g;
    double u = 0.5;
    if (rp.mode == 0) {
      double d[3];
      mc_proposal(rp.seed, (unsigned long long)(rp.step0 + t), 0u, S.n, rp.h, &g.j, d, &u);
      const double4 pj = ldcg4(&S.ppos[g.j]);
      g.r[0] = pj.x;
      g.r[1] = pj.y;
      g.r[2] = pj.z;
      g.q = pj.w;
      g.outside = false;
#pragma unroll
      for (int k = 0; k < 3; k++) {
        double x = __dadd_rn(g.r[k], d[k]);
        if (pbc) {
          if (x < 0.0) x = __dadd_rn(x, S.a);
          if (x >= S.a) x = __dsub_rn(x, S.a);
        } else if (!(x >= 0.0 && x < S.a)) {
          g.outside = true;
        }
        g.rn[k] = x;
      }
    } else {
      g.j = (int)rp.jg;
      const double4 pj = ldcg4(&S.ppos[g.j]);
      g.r[0] = pj.x;
      g.r[1] = pj.y;
      g.r[2] = pj.z;
      g.q = pj.w;
      g.rn[0] = rp.rx;
      g.rn[1] = rp.ry;
      g.rn[2] = rp.rz;
      g.outside = false;
    }
    const bool nomove = (g.r[0] == g.rn[0] && g.r[1] == g.rn[1] && g.r[2] == g.rn[2]);
#pragma unroll
    for (int k = 0; k < 3; k++) {
      g.cf[k] = finest_coord(g.r[k], S.inv_wL, S.nL);
      g.cfn[k] = g.outside ? g.cf[k] : finest_coord(g.rn[k], S.inv_wL, S.nL);
    }
    g.same = (g.cf[0] == g.cfn[0] && g.cf[1] == g.cfn[1] && g.cf[2] == g.cfn[2]);

    // -------------------------------------------------------- propose items
    const int nE = L - S.lmin + 1;
    const int nN = g.same ? 27 : 54;
    const int nRB = (C + 31) / 32;
    const int nF = pbc ? nRB * MC_NF_COLS : 0;
    const int nItems = nE + nN + nF + 1;
    double* part = S.partials + buf * MC_MAX_ITEMS;

    for (int it = warp * nCTA + cta; it < nItems; it += nWarpsTot) {
      double partial = 0.0;
      if (nomove || g.outside) {
        // no work: dE is 0 (no move) or +inf (left a free-space box)
        if (it == nItems - 1) {
          if (g.outside) partial = __longlong_as_double(0x7ff0000000000000LL);
          if (lane == 0 && rp.mode == 0) part[MC_MAX_ITEMS - 1] = log(u);
        }
      } else if (it < nE) {
        // ---- E: Eq. (2) at r (half 0) and r' (half 1) on level l
        const int l = L - it, sh = L - l;
        const int* cc = half ? g.cfn : g.cf;
        const double* x = half ? g.rn : g.r;
        const int cx = cc[0] >> sh, cy = cc[1] >> sh, cz = cc[2] >> sh;
        const int nl = S.lev_n[l];
        const double w = S.lev_w[l];
        const double dx = x[0] - (cx + 0.5) * w, dy = x[1] - (cy + 0.5) * w,
                     dz = x[2] - (cz + 0.5) * w;
        const double* Lb = S.Lhat + (size_t)(S.lev_off[l] + (cx * nl + cy) * nl + cz) * C;
        const int m = hm;
        TE Lr[MC_PMAX + 1], Li[MC_PMAX + 1];
#pragma unroll
        for (int n = 0; n <= MC_PMAX; n++) {
          Lr[n] = TE(0);
          Li[n] = TE(0);
          if (n <= p && m <= n) {
            const int k = rl_re(n, m);
            Lr[n] = (TE)__ldcg(&Lb[k]);
            if (m) Li[n] = (TE)__ldcg(&Lb[k + 1]);
          }
        }
        TE acc = TE(0);
        regular_columns<TE>(&tabs, p, m, (TE)dx, (TE)dy, (TE)dz, [&](int n, TE cr, TE ci) {
          if (n >= m) acc += Lr[n] * cr - Li[n] * ci;
        });
        if (m > p) acc = TE(0);
        if (m > 0) acc *= TE(2);
        acc = half_sum(acc);
        const double psi = (double)acc;
        const double psin = __shfl_sync(0xffffffffu, psi, 16);
        partial = g.q * (psin - psi);
      } else if (it < nE + nN) {
        // ---- N: Alg. 1 over one near cell (27 cells of the extended domain)
        const int k0 = it - nE;
        const int k = g.same ? k0 : (k0 % 27);
        const int side = g.same ? 2 : (k0 / 27);  // 0 old, 1 new, 2 both
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
        if (valid) {
          const int cell = (c0 * nL + c1) * nL + c2;
          const int cnt = __ldcg(&S.ccount[cell]);
          const bool zero_shift = (s0 == 0 && s1 == 0 && s2 == 0);
          const double sx = s0 * S.a, sy = s1 * S.a, sz = s2 * S.a;
          bool ovl = false;
          if (sizeof(TE) == 8) {
            double acc = 0.0;
            for (int s = lane; s < cnt; s += 32) {
              const double4 xi = ldcg4(&S.cpos[(size_t)cell * S.cap + s]);
              const double xx = xi.x + sx, yy = xi.y + sy, zz = xi.z + sz;
              if (side != 1) {
                const int pid = __ldcg(&S.cpid[(size_t)cell * S.cap + s]);
                if (!(pid == g.j && zero_shift)) {
                  const double ax = g.r[0] - xx, ay = g.r[1] - yy, az = g.r[2] - zz;
                  acc -= g.q * xi.w * rsqrt(ax * ax + ay * ay + az * az);
                }
              }
              if (side != 0) {
                const double bx = g.rn[0] - xx, by = g.rn[1] - yy, bz = g.rn[2] - zz;
                const double d2 = bx * bx + by * by + bz * bz;
                if (d2 == 0.0) ovl = true;
                acc += g.q * xi.w * rsqrt(d2);
              }
            }
            partial = warp_sum(acc);
          } else {
            // positions relative to the (image) cell centre, in FP32
            const double w = S.lev_w[L];
            const double Rx = (c0 + 0.5) * w + sx, Ry = (c1 + 0.5) * w + sy,
                         Rz = (c2 + 0.5) * w + sz;
            const float ox = (float)(g.r[0] - Rx), oy = (float)(g.r[1] - Ry),
                        oz = (float)(g.r[2] - Rz);
            const float nx = (float)(g.rn[0] - Rx), ny = (float)(g.rn[1] - Ry),
                        nz = (float)(g.rn[2] - Rz);
            float acc = 0.0f;
            const float qf = (float)g.q;
            for (int s = lane; s < cnt; s += 32) {
              const float4 xi = __ldcg(&S.cpos32[(size_t)cell * S.cap + s]);
              if (side != 1) {
                const int pid = __ldcg(&S.cpid[(size_t)cell * S.cap + s]);
                if (!(pid == g.j && zero_shift)) {
                  const float ax = ox - xi.x, ay = oy - xi.y, az = oz - xi.z;
                  acc -= qf * xi.w * rsqrtf(ax * ax + ay * ay + az * az);
                }
              }
              if (side != 0) {
                const float bx = nx - xi.x, by = ny - xi.y, bz = nz - xi.z;
                const float d2 = bx * bx + by * by + bz * bz;
                if (d2 == 0.0f) ovl = true;
                acc += qf * xi.w * rsqrtf(d2);
              }
            }
            partial = (double)warp_sum(acc);
          }
          if (__any_sync(0xffffffffu, ovl)) partial = __longlong_as_double(0x7ff0000000000000LL);
        }
      } else if (it < nE + nN + nF) {
        // ---- F: far lattice, Sec. 3.3 (iv) in the factored form
        //   dU_inf = sum_k W_k dK_k (H_k + 1/2 (G dK)_k),  W = 1 (m = 0) or 2
        const int f = it - nE - nN;
        const int rb = f / MC_NF_COLS, cb = f % MC_NF_COLS;
        const int m = hm;
        const double* x = half ? g.rn : g.r;
        const double c1 = 0.5 * S.a;
        double* st = stage[warp];
        const TE dx = (TE)(x[0] - c1), dy = (TE)(x[1] - c1), dz = (TE)(x[2] - c1);
        regular_columns<TE>(&tabs, p, m, dx, dy, dz, [&](int n, TE cr, TE ci) {
          const TE nr = __shfl_xor_sync(0xffffffffu, cr, 16);
          const TE ni = __shfl_xor_sync(0xffffffffu, ci, 16);
          if (half == 0 && m <= p && n >= m) {
            // dK = q (conj Rt(r' - R1) - conj Rt(r - R1))
            const int k = rl_re(n, m);
            st[k] = g.q * ((double)nr - (double)cr);
            if (m) st[k + 1] = -g.q * ((double)ni - (double)ci);
          }
        });
        __syncwarp();
        const int csz = (C + MC_NF_COLS - 1) / MC_NF_COLS;
        const int cbeg = cb * csz, cend = min(C, cbeg + csz);
        const int k = rb * 32 + lane;
        double contrib = 0.0;
        if (k < C) {
          double gk = 0.0;
          for (int c = cbeg; c < cend; c++) gk += S.G[(size_t)c * C + k] * st[c];
          S.gK[(size_t)buf * MC_NF_COLS * C + (size_t)cb * C + k] = gk;
          const double Wk = is_square(k) ? 1.0 : 2.0;
          contrib = Wk * st[k] * (0.5 * gk + (cb == 0 ? __ldcg(&S.Hhat[k]) : 0.0));
        }
        if (f == 0) {
          for (int kk = lane; kk < C; kk += 32) S.dK[(size_t)buf * C + kk] = st[kk];
        }
        partial = warp_sum(contrib);
        __syncwarp();
      } else {
        // ---- X: periodic self-interaction correction (Sec. 3.3, last item),
        //         dipole term (tinfoil reading), log(u)
        double v = 0.0;
        if (pbc) {
          if (lane < 27) {
            const double ax = g.rn[0] - (g.r[0] + (lane / 9 - 1) * S.a);
            const double ay = g.rn[1] - (g.r[1] + ((lane / 3) % 3 - 1) * S.a);
            const double az = g.rn[2] - (g.r[2] + (lane % 3 - 1) * S.a);
            v = -g.q * g.q * rsqrt(ax * ax + ay * ay + az * az);
          }
        } else if (lane == 0) {
          const double ax = g.rn[0] - g.r[0], ay = g.rn[1] - g.r[1], az = g.rn[2] - g.r[2];
          v = -g.q * g.q * rsqrt(ax * ax + ay * ay + az * az);
        }
        partial = warp_sum(v);
        if (pbc) {
          partial += g.q * g.q / S.a * kImageConst;
          if (S.dip == 0) {
            const double cdip = -2.0 * kPi / (3.0 * S.V);
            double D2 = 0.0, Dn2 = 0.0;
#pragma unroll
            for (int k = 0; k < 3; k++) {
              const double D = __ldcg(&S.dipv[k]);
              const double Dn = D + g.q * (g.rn[k] - g.r[k]);
              D2 += D * D;
              Dn2 += Dn * Dn;
            }
            partial += cdip * Dn2 - cdip * D2;
          }
        }
        if (lane == 0 && rp.mode == 0) part[MC_MAX_ITEMS - 1] = log(u);
      }
      if (lane == 0) part[it] = partial;
    }

    gen++;
    if (!grid_barrier(S.bar, gen * (unsigned long long)nCTA, S.status, rp.wait_ns)) break;

    // ------------------------------------------------ decision (every CTA)
    if (warp == 0) {
      double acc = 0.0;
      for (int i = lane; i < nItems; i += 32) acc += __ldcg(&part[i]);
      acc = warp_sum(acc);
      if (lane == 0) {
        s_dE = acc;
        s_logu = (rp.mode == 0) ? __ldcg(&part[MC_MAX_ITEMS - 1]) : 0.0;
      }
    }
    __syncthreads();
    const double dE = s_dE;
    bool accept;
    if (rp.mode == 1) {
      accept = false;
    } else if (rp.mode == 2) {
      accept = true;
    } else if (dE <= 0.0) {
      accept = true;
    } else {
      const double t2 = -rp.beta * dE;
      accept = s_logu < t2;
      if (fabs(s_logu - t2) < 1e-9 * fmax(1.0, fabs(t2))) n_border++;
    }
    const double dE_used = (rp.mode == 2 && rp.has_dE) ? rp.dEg : dE;
    if (cta == 0 && threadIdx.x == 0) {
      if (rp.mode == 1) S.result[0] = dE;
      if (rp.log_j) {
        rp.log_j[t] = g.j;
        rp.log_dE[t] = dE;
        rp.log_acc[t] = accept ? 1 : 0;
      }
    }
    steps_done++;
    if (!accept || nomove) {
      if (accept) n_acc++;
      if (accept && cta == 0 && threadIdx.x == 0) S.energy[0] += dE_used;
      if (rp.stop_after_accepts > 0 && n_acc >= rp.stop_after_accepts) break;
      continue;
    }
    n_acc++;

    // --------------------------------------------------------- accept items
    // level item counts: small levels (<= 4 cells per axis) enumerate every
    // canonical cell, larger ones the interaction lists of alpha' (owners)
    // and of alpha (owners unless also in IL(alpha')).
    int lev_items[MC_MAXLEV + 2], lev_start[MC_MAXLEV + 2];
    int nA = 1;  // item 0: bookkeeping
    for (int l = L; l >= S.lmin; l--) {
      const int sh = L - l, nl = S.lev_n[l];
      const bool samel = ((g.cf[0] >> sh) == (g.cfn[0] >> sh)) &&
                         ((g.cf[1] >> sh) == (g.cfn[1] >> sh)) &&
                         ((g.cf[2] >> sh) == (g.cfn[2] >> sh));
      lev_items[l] = (nl <= 4) ? nl * nl * nl : (samel ? 189 : 378);
      lev_start[l] = nA;
      nA += lev_items[l];
    }
    for (int it = warp * nCTA + cta; it < nA; it += nWarpsTot) {
      if (it == 0) {
        // ---- bookkeeping: K, H, dipole, energy, cell lists
        if (pbc) {
          for (int k = lane; k < C; k += 32) {
            S.Khat[k] += __ldcg(&S.dK[(size_t)buf * C + k]);
            double gs = 0.0;
            for (int cb = 0; cb < MC_NF_COLS; cb++)
              gs += __ldcg(&S.gK[(size_t)buf * MC_NF_COLS * C + (size_t)cb * C + k]);
            S.Hhat[k] += gs;
          }
        }
        if (lane == 0) {
#pragma unroll
          for (int k = 0; k < 3; k++) S.dipv[k] += g.q * (g.rn[k] - g.r[k]);
          S.energy[0] += dE_used;
          const int nL = S.nL, cap = S.cap;
          const int co = (g.cf[0] * nL + g.cf[1]) * nL + g.cf[2];
          const int cn = (g.cfn[0] * nL + g.cfn[1]) * nL + g.cfn[2];
          const double w = S.lev_w[L];
          const float4 rel = make_float4((float)(g.rn[0] - (g.cfn[0] + 0.5) * w),
                                         (float)(g.rn[1] - (g.cfn[1] + 0.5) * w),
                                         (float)(g.rn[2] - (g.cfn[2] + 0.5) * w), (float)g.q);
          const double4 np = make_double4(g.rn[0], g.rn[1], g.rn[2], g.q);
          const int so = S.pslot[g.j];
          if (co == cn) {
            S.cpos[so] = np;
            S.cpos32[so] = rel;
          } else {
            const int last = S.ccount[co] - 1;
            const int sl = co * cap + last;
            if (so != sl) {
              S.cpos[so] = S.cpos[sl];
              S.cpos32[so] = S.cpos32[sl];
              const int pid = S.cpid[sl];
              S.cpid[so] = pid;
              S.pslot[pid] = so;
            }
            S.ccount[co] = last;
            const int sn = S.ccount[cn];
            if (sn >= cap) {
              atomicExch(S.status, MCD_ERR_CAPACITY);
            } else {
              const int slot = cn * cap + sn;
              S.cpos[slot] = np;
              S.cpos32[slot] = rel;
              S.cpid[slot] = g.j;
              S.pslot[g.j] = slot;
              S.ccount[cn] = sn + 1;
            }
          }
          S.ppos[g.j] = np;
        }
        continue;
      }
      // ---- level target item (Alg. L.2)
      int l = L;
      while (l > S.lmin && it >= lev_start[l] + lev_items[l]) l--;
      const int k = it - lev_start[l];
      const int sh = L - l, nl = S.lev_n[l];
      const double w = S.lev_w[l];
      const int co[3] = {g.cf[0] >> sh, g.cf[1] >> sh, g.cf[2] >> sh};
      const int cn[3] = {g.cfn[0] >> sh, g.cfn[1] >> sh, g.cfn[2] >> sh};
      int tc[3];
      bool owner = true;
      if (nl <= 4) {
        tc[0] = k / (nl * nl);
        tc[1] = (k / nl) % nl;
        tc[2] = k % nl;
      } else {
        const bool from_new = (lev_items[l] == 189) || (k < 189);
        const int kk = (k < 189) ? k : k - 189;
        const int* base = from_new ? cn : co;
        const int par = ((base[0] & 1) << 2) | ((base[1] & 1) << 1) | (base[2] & 1);
        int ox, oy, oz;
        il_unpack(il[par][kk], &ox, &oy, &oz);
        const int e[3] = {base[0] + ox, base[1] + oy, base[2] + oz};
        if (!pbc && (e[0] < 0 || e[0] >= nl || e[1] < 0 || e[1] >= nl || e[2] < 0 || e[2] >= nl))
          owner = false;
        for (int d = 0; d < 3; d++) tc[d] = mc_wrap_coord(e[d], nl);
        if (owner && !from_new) {
          // skip targets that the alpha' list owns
          for (int s = 0; s < 27 && owner; s++) {
            const int sx = s / 9 - 1, sy = (s / 3) % 3 - 1, sz = s % 3 - 1;
            if (!pbc && (sx || sy || sz)) continue;
            if (in_il(tc[0] + sx * nl - cn[0], tc[1] + sy * nl - cn[1], tc[2] + sz * nl - cn[2],
                      cn[0], cn[1], cn[2]))
              owner = false;
          }
        }
      }
      if (!owner) continue;
      // contributions of this half's side: bit s of mask = image shift s
      const int* cs = half ? cn : co;
      unsigned mask = 0u;
      for (int s = 0; s < 27; s++) {
        const int sx = s / 9 - 1, sy = (s / 3) % 3 - 1, sz = s % 3 - 1;
        if (!pbc && (sx || sy || sz)) continue;
        if (in_il(tc[0] + sx * nl - cs[0], tc[1] + sy * nl - cs[1], tc[2] + sz * nl - cs[2], cs[0],
                  cs[1], cs[2]))
          mask |= 1u << s;
      }
      const int cnt = __popc(mask);
      const int cnt_o = __shfl_xor_sync(0xffffffffu, cnt, 16);
      const int iters = max(cnt, cnt_o);
      if (iters == 0) continue;
      const double* x = half ? g.rn : g.r;
      const TE sg = (TE)(half ? g.q : -g.q);
      const int m = hm;
      TE ar[MC_PMAX + 1], ai[MC_PMAX + 1];
#pragma unroll
      for (int n = 0; n <= MC_PMAX; n++) {
        ar[n] = TE(0);
        ai[n] = TE(0);
      }
      for (int i = 0; i < iters; i++) {
        const bool act = i < cnt;
        int s = 0;
        if (act) {
          unsigned mm = mask;
          for (int b = 0; b < i; b++) mm &= mm - 1u;
          s = __ffs(mm) - 1;
        }
        const int sx = s / 9 - 1, sy = (s / 3) % 3 - 1, sz = s % 3 - 1;
        const double Rx = (tc[0] + sx * nl + 0.5) * w, Ry = (tc[1] + sy * nl + 0.5) * w,
                     Rz = (tc[2] + sz * nl + 0.5) * w;
        // inactive lanes evaluate a harmless point (never consumed)
        const TE dx = act ? (TE)(x[0] - Rx) : TE(3), dy = act ? (TE)(x[1] - Ry) : TE(3),
                 dz = act ? (TE)(x[2] - Rz) : TE(3);
        const TE f = act ? sg : TE(0);
        irregular_columns<TE>(&tabs, p, m, dx, dy, dz, [&](int n, TE cr, TE ci) {
          ar[n] += f * cr;
          ai[n] -= f * ci;
        });
      }
      double* st = stage[warp];
#pragma unroll
      for (int n = 0; n <= MC_PMAX; n++) {
        const TE orr = __shfl_xor_sync(0xffffffffu, ar[n], 16);
        const TE oii = __shfl_xor_sync(0xffffffffu, ai[n], 16);
        if (half == 0 && n <= p && m <= n) {
          const int kk = rl_re(n, m);
          st[kk] = (double)ar[n] + (double)orr;
          if (m) st[kk + 1] = (double)ai[n] + (double)oii;
        }
      }
      __syncwarp();
      double* Lt = S.Lhat + (size_t)(S.lev_off[l] + (tc[0] * nl + tc[1]) * nl + tc[2]) * C;
      for (int kk = lane; kk < C; kk += 32) __stcg(&Lt[kk], __ldcg(&Lt[kk]) + st[kk]);
      __syncwarp();
    }
    gen++;
    if (!grid_barrier(S.bar, gen * (unsigned long long)nCTA, S.status, rp.wait_ns)) break;
    if (rp.stop_after_accepts > 0 && n_acc >= rp.stop_after_accepts) break;
  }
  if (cta == 0 && threadIdx.x == 0) {
    S.stats[0] = steps_done;
    S.stats[1] = n_acc;
    S.stats[2] = n_border;
  }
}

template __global__ void mc_chain_kernel<double>(const McSys*, RunParams);
template __global__ void mc_chain_kernel<float>(const McSys*, RunParams);

// host-side launcher (cooperative launch: all CTAs co-resident)
cudaError_t mc_launch_chain(const McSys* d_sys, const RunParams& rp, int prec, int nCTA,
                            cudaStream_t stream) {
  void* args[] = {(void*)&d_sys, (void*)&rp};
  const void* fn = prec ? (const void*)mc_chain_kernel<float> : (const void*)mc_chain_kernel<double>;
  return cudaLaunchCooperativeKernel(fn, dim3(nCTA), dim3(MC_THREADS), args, 0, stream);
}

int mc_chain_max_ctas(int prec) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = prec ? (const void*)mc_chain_kernel<float> : (const void*)mc_chain_kernel<double>;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, MC_THREADS, 0);
  if (per < 1) return 0;
  return sms;  // one CTA per SM
}
