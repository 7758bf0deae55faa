// Persistent Metropolis-Hastings chain kernel: one cooperative launch runs
// many steps of Alg. L.1 (propose, with Alg. 1 and the periodic terms of
// Sec. 3.4) and Alg. L.2 (accept) for one system on the whole GPU.
//
// One step:
//   1. warp 0 of every CTA draws the same Philox proposal (j, r -> r') and
//      the offsets of r and r' from the centres of their cells on every
//      level; the CTA reads them from shared memory;
//   2. propose items, one warp each, spread over the SMs:
//        E  level expansions (Eq. 1/2) at r and r' on level l
//        N  direct sum over one of the 27 near cells (Alg. 1)
//        F  far lattice term: dK and a 32-row x C/16-column block of G dK
//        X  image self-interaction correction and dipole term
//        U  log(u) of the Metropolis test
//      each writes one partial sum;
//   3. grid barrier;
//   4. every CTA reduces the partials in the same fixed order -> dE and the
//      Metropolis decision (identical in every CTA, no broadcast needed);
//   5. on accept: Alg. L.2 items (one contribution per half-warp on levels
//      with <= 4 cells per axis, one updated cell per warp above) and one
//      bookkeeping item (K, H, dipole, energy, cell lists); then a second
//      grid barrier.
// Displacements are formed as (offset of the point from its own cell centre)
// minus (integer cell offset) x (cell width), which keeps FP64 work off the
// items and keeps FP32 displacements accurate.
// Template TE is the evaluation type: double (FP64 form) or float (FP32-eval
// form: harmonics and near field in FP32; FP64 accumulators, energy, far
// lattice operator, decision).
#include "mc_items.cuh"

#include <algorithm>

// kVar: MC_VAR_PLAIN (local method, accept computed after the decision),
// MC_VAR_SPEC (local method, speculative accept: MC_SCHEDULE_PHASED) or
// MC_VAR_MM (the multipole method of Alg. M.1/M.2), as separate
// instantiations (smaller code per kernel: the instruction cache is a
// measured limit of this kernel)
template <typename TE, int kVar>
__device__ __forceinline__ void chain_body(const McSys* __restrict__ sysp, RunParams& rp,
                                           const int nCTA, const int cta) {
  // MC_VAR_SPECW: the speculative contributions in the column-scaled form
  // (5 flops per recurrence step, no in-register sum of the two sides: each
  // side its own staged slot, P_n^m applied by the apply's multiply-add):
  // fewer FP64 instructions, for the throughput-bound batched FP64 form
  constexpr bool specw = kVar == MC_VAR_SPECW;
  constexpr bool spec = kVar == MC_VAR_SPEC || specw;
  constexpr bool mm = kVar == MC_VAR_MM;
  __shared__ McSys S;
  __shared__ HarmTabs<TE> tabs;
  __shared__ unsigned short il[8][189];
  __shared__ double stage[MC_WARPS][mm ? 512 : 256];
  __shared__ double s_dE, s_logu, s_u;
  __shared__ double s_wpart[MC_WARPS];  // per-warp partial sums (multipole method)
  __shared__ StepGeo sgeo;
  // offset of r (side 0) / r' (side 1) from its cell centre on level l
  __shared__ double s_off[2][MC_MAXLEV + 2][3];
  // k * width of level l for k = -3..3 (k + 3), and in the evaluation type
  __shared__ double s_kw[MC_MAXLEV + 2][7];
  __shared__ TE s_kwe[MC_MAXLEV + 2][7];
  __shared__ TE s_iW[specw ? MC_PMAX + 1 : 1][16];
  __shared__ double s_P[specw ? (MC_PMAX + 1) * (MC_PMAX + 1) : 1];
  // the contributions in pair-of-floats arithmetic (FP64 form): W, A_k and
  // P_n^m as pairs, n of every real-layout index, and per level the
  // power-of-two unit k_l (2^k_l <= cell width < 2^(k_l + 1))
  __shared__ f2 s_W2[specw ? MC_PMAX + 1 : 1][16];
  __shared__ f2 s_A2[16];
  __shared__ f2 s_P2[specw ? (MC_PMAX + 1) * (MC_PMAX + 1) : 1];
  __shared__ unsigned char s_nn[specw ? (MC_PMAX + 1) * (MC_PMAX + 1) : 1];
  __shared__ int s_kl[MC_MAXLEV + 2];

  if (threadIdx.x == 0) S = *sysp;
  harm_tabs_init<TE>(&tabs);
  if constexpr (specw) irregular_w_tabs<TE>(s_iW, s_P);
  il_table_init(il);
  __syncthreads();
  for (int i = threadIdx.x; i < (MC_MAXLEV + 2) * 7; i += blockDim.x) {
    const int l = i / 7, k = i % 7 - 3;
    const double v = (l >= 1 && l <= S.L) ? k * S.lev_w[l] : 0.0;
    s_kw[l][k + 3] = v;
    s_kwe[l][k + 3] = (TE)v;
  }
  if constexpr (specw) pair_w_tabs<TE>(s_iW, s_P, s_W2, s_A2, s_P2, s_nn, s_kl, S.lev_w, S.L);
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = S.p, C = S.C, L = S.L;
  const bool pbc = (S.bc == 0);
  const int nWarpsTot = nCTA * MC_WARPS;
  const int gw = warp * nCTA + cta;  // this warp's first item of every phase
  unsigned long long gen = 0;
  long long n_acc = 0, n_border = 0, steps_done = 0;
  const bool prof_on = rp.prof != nullptr;
  const bool prof_lead = prof_on && cta == 0 && threadIdx.x == 0;
  unsigned long long tp0 = 0, tp1 = 0;
  const unsigned long long t_begin = mc_globaltimer();

  // Proposal items in the order F, E, N, X, U, K.  The far items come
  // first, so far item f always runs on the warp of slot f, which keeps its
  // block of the constant operator G (32 rows x csz columns) in registers for
  // the launch.  (The items share SMs with the speculative accept items that
  // follow them; measured on GB300, this order leaves the expansion items on
  // the SMs with the fewest of those.)
  const int nRB = (C + 31) / 32;
  const int nfc = rp.nf_cols;
  const int nF = pbc ? nRB * nfc : 0;
  const int csz = (C + nfc - 1) / nfc;
  const int nE = L - S.lmin + 1;
  const bool gpre = nF <= nWarpsTot && csz <= MC_GPRE;
  const int gf = gw;  // far item of this warp's slot
  double gcol[MC_GPRE];
#pragma unroll
  for (int i = 0; i < MC_GPRE; i++) gcol[i] = 0.0;
  if (gpre && gf >= 0 && gf < nF) {
    const int k = (gf / nfc) * 32 + lane, cbeg = (gf % nfc) * csz;
#pragma unroll
    for (int i = 0; i < MC_GPRE; i++) {
      const int c = cbeg + i;
      if (k < C && i < csz && c < C) gcol[i] = __ldcg(&S.G[(size_t)c * C + k]);
    }
  }

  // proposal of the next step, drawn and its particle loaded ahead (warp 0)
  bool pf_ok = false;
  int pf_j = 0;
  double pf_d = 0.0, pf_u = 0.5;
  double4 pf_pos = make_double4(0, 0, 0, 0);
  // geometry of a proposal (warp 0, per lane: r, r' components on lanes
  // 0..2; the offsets from the cell centres for side lane/16, level slot
  // lane%16), formed for the next step at the end of this step's items
  struct PGeo {
    int j, cf, cfn, lo;
    double q, uu, r, rn;
    double off[3];
    bool out;
  } pg;
  pg.j = -1;
  pg.lo = 0;
  bool pg_ok = false;
  // whole warp: j, charge (lanes 0..2), r and d (or r' when !is_d) per axis lane
  auto form_geo = [&](PGeo& G, int j, double q, double r, double dn, bool is_d, double uu) {
    double rn = 0.0;
    bool out = false;
    if (lane < 3) {
      if (is_d) {
        double x = __dadd_rn(r, dn);
        if (pbc) {
          if (x < 0.0) x = __dadd_rn(x, S.a);
          if (x >= S.a) x = __dsub_rn(x, S.a);
        } else if (!(x >= 0.0 && x < S.a)) {
          out = true;
        }
        rn = x;
      } else {
        rn = dn;
      }
    }
    const bool any_out = __any_sync(0xffffffffu, lane < 3 && out);
    int cf = 0, cfn = 0;
    if (lane < 3) {
      cf = finest_coord(r, S.inv_wL, S.nL);
      cfn = any_out ? cf : finest_coord(rn, S.inv_wL, S.nL);
    }
    const int side = lane >> 4, li = lane & 15;
    const int l = L - li;
    const int lo = (l >= 1 && l <= L && li <= L - 1) ? l : 0;
#pragma unroll
    for (int ax = 0; ax < 3; ax++) {
      const double xo = __shfl_sync(0xffffffffu, r, ax), xn = __shfl_sync(0xffffffffu, rn, ax);
      const int co = __shfl_sync(0xffffffffu, cf, ax), cnn = __shfl_sync(0xffffffffu, cfn, ax);
      const double xs = side ? xn : xo;
      const int cs = side ? cnn : co;
      G.off[ax] = lo ? xs - ((double)(cs >> (L - lo)) + 0.5) * S.lev_w[lo] : 0.0;
    }
    G.j = j;
    G.q = __shfl_sync(0xffffffffu, q, 0);
    G.uu = uu;
    G.r = r;
    G.rn = rn;
    G.cf = cf;
    G.cfn = cfn;
    G.lo = lo;
    G.out = any_out;
  };

  // the two previous steps (every thread): moved, particle; warp 0 lanes
  // 0..2 also keep their r' components.  The accept of a step can still be
  // running in other CTAs when this CTA reads ahead (see the split barrier
  // below), so loads made one step ahead are checked against both.
  bool mv1 = false, mv2 = false;
  int j1 = -1, j2 = -1;
  double rn1 = 0.0, rn2 = 0.0;
  // target count of the split barrier that ended the previous step's accept
  // (0: none pending); reads of state the accept writes wait for it
  unsigned long long pend = 0;

  for (long long t = 0; t < rp.nsteps; t++) {
    const int buf = (int)(t & 1);
    if (prof_lead) tp0 = mc_globaltimer();
    // ------------------------------------------------------------ proposal
    if (warp == 0) {
      if (rp.mode == 0) {
        // the geometry formed at the end of the previous step holds unless
        // one of the two previous steps moved this particle (the position was
        // loaded before their accepts); else form it again here
        const bool fast = pg_ok && !(mv1 && pg.j == j1) && !(mv2 && pg.j == j2);
        if (!fast) {
          int j;
          double d = 0.0, uu = 0.5;
          double4 pj;
          if (pf_ok) {
            j = pf_j;
            d = pf_d;
            uu = pf_u;
            pj = pf_pos;
          } else {
            mc_proposal_axis(rp.seed, (unsigned long long)(rp.step0 + t), rp.chain, S.n, rp.h,
                             lane < 3 ? lane : 0, &j, &d, lane == 3 ? &uu : nullptr);
            pj = lane < 3 ? ldcg4(&S.ppos[j]) : make_double4(0, 0, 0, 0);
          }
          double r = lane == 0 ? pj.x : (lane == 1 ? pj.y : pj.z);
          if (pf_ok && lane < 3) {
            if (mv1 && j == j1) {
              r = rn1;
            } else if (mv2 && j == j2) {
              r = rn2;
            }
          }
          form_geo(pg, j, pj.w, r, d, true, uu);
        }
      } else {
        const int j = (int)rp.jg;
        const double4 pj = lane < 3 ? ldcg4(&S.ppos[j]) : make_double4(0, 0, 0, 0);
        const double r = lane == 0 ? pj.x : (lane == 1 ? pj.y : pj.z);
        const double rn = lane == 0 ? rp.rx : (lane == 1 ? rp.ry : rp.rz);
        form_geo(pg, j, pj.w, r, rn, false, 0.5);
      }
      // publish
      if (pg.lo) {
        const int side = lane >> 4;
#pragma unroll
        for (int ax = 0; ax < 3; ax++) s_off[side][pg.lo][ax] = pg.off[ax];
      }
      if (lane < 3) {
        sgeo.r[lane] = pg.r;
        sgeo.rn[lane] = pg.rn;
        sgeo.cf[lane] = pg.cf;
        sgeo.cfn[lane] = pg.cfn;
      }
      if (lane == 0) {
        sgeo.j = pg.j;
        sgeo.q = pg.q;
        sgeo.outside = pg.out;
      }
      if (lane == 3) s_u = pg.uu;
      pg_ok = false;
    }
    __syncthreads();
    const StepGeo g = sgeo;
    if (warp == 0) {
      // draw the next proposal and start loading its particle
      pf_ok = false;
      if (rp.mode == 0 && t + 1 < rp.nsteps) {
        mc_proposal_axis(rp.seed, (unsigned long long)(rp.step0 + t + 1), rp.chain, S.n, rp.h,
                         lane < 3 ? lane : 0, &pf_j, &pf_d, lane == 3 ? &pf_u : nullptr);
        if (lane < 3) pf_pos = ldcg4(&S.ppos[pf_j]);
        pf_ok = true;
      }
    }
    const double u = s_u;
    const bool nomove = (g.r[0] == g.rn[0] && g.r[1] == g.rn[1] && g.r[2] == g.rn[2]);
    const bool same = (g.cf[0] == g.cfn[0] && g.cf[1] == g.cfn[1] && g.cf[2] == g.cfn[2]);
    const bool idle = nomove || g.outside;

    // accept items per level: on small levels (<= 4 cells per axis) item k
    // takes entries 2k, 2k+1 of IL(alpha) and IL(alpha') (4 contributions);
    // on larger levels one item per updated target cell
    int lev_items[MC_MAXLEV + 2], lev_start[MC_MAXLEV + 2];
    int nD = 0;
    for (int l = L; l >= S.lmin; l--) {
      const int sh = L - l, nl = S.lev_n[l];
      const bool samel = ((g.cf[0] >> sh) == (g.cfn[0] >> sh)) &&
                         ((g.cf[1] >> sh) == (g.cfn[1] >> sh)) &&
                         ((g.cf[2] >> sh) == (g.cfn[2] >> sh));
      lev_items[l] = (nl <= 4) ? 95 : (samel ? 189 : 378);
      lev_start[l] = nD;
      nD += lev_items[l];
    }
    // speculative accept: phase-A items per level (small levels: as above,
    // adding into the step's small-level delta buffer; large levels: two
    // targets per item, staged in the level's block of MC_DSLOTS x C doubles
    // at slot k) and phase-B apply items (one per small-level cell, two
    // large-level targets per item)
    int sp_items[MC_MAXLEV + 2], sp_start[MC_MAXLEV + 2];
    int nDs = 0, nLB = 0;
    for (int l = L; l >= S.lmin; l--) {
      sp_items[l] = (S.lev_n[l] <= 4) ? 95 : (lev_items[l] + 1) / 2;
      sp_start[l] = nDs;
      nDs += sp_items[l];
      if (S.lev_n[l] > 4) nLB += lev_items[l];
    }
    // (staged slots by step parity, small-level deltas in three rotating
    // buffers: the accept of the previous step may still read its own)
    const int nlev = L - S.lmin + 1;
    auto dslot = [&](int l, int slot, int side) -> double* {
      if constexpr (specw)
        return S.dacc + ((((size_t)(t & 1) * nlev + (L - l)) * 2 + side) * MC_DSLOTS + slot) * C;
      return S.dacc + (((size_t)(t & 1) * nlev + (L - l)) * MC_DSLOTS + slot) * C;
    };
    const size_t nsC = (size_t)S.nsmall * C;
    double* dsm = S.dsmall + (size_t)(t % 3) * nsC;             // this step's
    double* dsm_next = S.dsmall + (size_t)((t + 1) % 3) * nsC;  // zeroed now
    // wait of one warp for the previous step's accept (all CTAs)
    auto need_state = [&]() {
      if (pend) warp_wait(S.bar, pend, S.status, rp.wait_ns);
    };

    // ------------------------------------- phase A: propose (+ accept deltas)
    // near items: near_parts per cell and side (slot blocks of the cell
    // round robin), 2 near_parts per cell when r and r' share their finest
    // cell (27 items at near_parts = 1)
    const int nNP = S.near_parts;
    const int nNsame = nNP == 1 ? 1 : 2 * nNP;
    const int nN = same ? 27 * nNsame : 54 * nNP;
    // the multipole method's P items: 95 per level (entries 2k, 2k+1 of
    // IL(alpha) and IL(alpha') per item, one per 8-lane group)
    const int nEx = mm ? 95 * nlev : nE;
    // K: the far-field change dK of the next proposal, which depends on
    // positions only, is formed one step ahead; this step's far items use
    // the one formed in the previous step unless that step moved the
    // particle this proposal picks
    const bool k_next = pbc && rp.mode == 0 && t + 1 < rp.nsteps;
    const bool dk_pre = pbc && rp.mode == 0 && t > 0 && !(mv1 && g.j == j1) && !(mv2 && g.j == j2);
    const int iF = 0, iE = nF, iN = iE + nEx, iX = iN + nN, iU = iX + 1, iK = iU + 1;
    const int nProp = k_next ? iK + 1 : iU + 1;
    const int nPhaseA = nProp + ((spec && !idle) ? nDs : 0);
    double* part = S.partials + buf * MC_MAX_ITEMS;

    double wsum = 0.0;  // this warp's items, in item order (multipole method)
    for (int it = gw; it < nPhaseA; it += nWarpsTot) {
      const unsigned long long t_item = prof_on ? mc_globaltimer() : 0ULL;
      int ptype = 7;
      if (it >= nProp) {
        // ---- speculative Alg. L.2 contributions of the proposed move
        const int dk = it - nProp;
        int l = L;
        while (l > S.lmin && dk >= sp_start[l] + sp_items[l]) l--;
        const int k = dk - sp_start[l];
        const int sh = L - l, nl = S.lev_n[l];
        const int co[3] = {g.cf[0] >> sh, g.cf[1] >> sh, g.cf[2] >> sh};
        const int cn[3] = {g.cfn[0] >> sh, g.cfn[1] >> sh, g.cfn[2] >> sh};
        const int grp = lane >> 3, side = grp & 1;
        if (nl <= 4) {
          // entries 2k, 2k+1 of both lists, added into the step's delta
          // buffer of the small levels (image copies make targets repeat)
          const SmallEntry se = small_entry(il, side ? cn : co, nl, pbc, 2 * k + (grp >> 1));
          const TE f = se.valid ? from_double<TE>(side ? g.q : -g.q) : TE(0);
          TE dx = TE(3), dy = TE(3), dz = TE(3);
          if (se.valid) {
            if (sizeof(TE) == 8) {
              dx = (TE)(s_off[side][l][0] - s_kw[l][se.o[0] + 3]);
              dy = (TE)(s_off[side][l][1] - s_kw[l][se.o[1] + 3]);
              dz = (TE)(s_off[side][l][2] - s_kw[l][se.o[2] + 3]);
            } else {
              dx = from_double<TE>(s_off[side][l][0]) - s_kwe[l][se.o[0] + 3];
              dy = from_double<TE>(s_off[side][l][1]) - s_kwe[l][se.o[1] + 3];
              dz = from_double<TE>(s_off[side][l][2]) - s_kwe[l][se.o[2] + 3];
            }
          }
          double* Dt = dsm + (size_t)(S.lev_off[l] + (se.t3[0] * nl + se.t3[1]) * nl + se.t3[2]) * C;
          auto add = [&](int t2, int n, int m, bool v, TE vr, TE vi) {
            if (se.valid && v) {
              const int kk = rl_re(n, m);
              atomicAdd(&Dt[kk], to_double(vr));
              if (m) atomicAdd(&Dt[kk + 1], to_double(neg_bits(vi)));
            }
          };
          if constexpr (specw && sizeof(TE) == 8) {
            // pair-of-floats recurrence in units of 2^k_l, back to the
            // true scale (2^(-k_l (n + 1))) for the atomic adds
            const int kl = s_kl[l];
            irregular_group_w2(s_A2, s_W2, p, f2_from_double((double)dx, -kl), f2_from_double((double)dy, -kl),
                               f2_from_double((double)dz, -kl), f2_from_double((double)f, 0),
                               [&](int t2, int n, int m, bool v, f2 vr, f2 vi) {
                                 if (se.valid && v) {
                                   const int kk = rl_re(n, m), e = -kl * (n + 1);
                                   atomicAdd(&Dt[kk], f2_to_double(vr, e));
                                   if (m) atomicAdd(&Dt[kk + 1], f2_to_double(f2_neg(vi), e));
                                 }
                               });
          } else if constexpr (specw) {
            irregular_group_w<TE>(&tabs, s_iW, p, dx, dy, dz, f, add);
          } else {
            irregular_group_s<TE>(&tabs, p, dx, dy, dz, f, add);
          }
        } else {
          // targets 2k (groups 0, 1) and 2k+1 (groups 2, 3); group 0/2 the
          // alpha side, 1/3 the alpha' side
          const int kt = 2 * k + (grp >> 1);
          const bool samel = lev_items[l] == 189;
          const bool exists = kt < lev_items[l];
          const LargeItem li = large_item(il, co, cn, nl, pbc, samel, exists ? kt : 0);
          const bool own = exists && li.owner;
          const int* cs = side ? cn : co;
          int ofs[3] = {li.ofs[0], li.ofs[1], li.ofs[2]};
          bool have = false;
          if (own) {
            if (samel || (li.from_new && side == 1) || (!li.from_new && side == 0)) {
              have = true;
            } else if (li.from_new) {
              list_offset(li.tc, cs, nl, pbc, ofs);
              have = in_il(ofs[0], ofs[1], ofs[2], cs[0], cs[1], cs[2]);
            }  // else: the target is not in IL(alpha') (else not owner)
          }
          const TE f = have ? from_double<TE>(side ? g.q : -g.q) : TE(0);
          TE dx = TE(3), dy = TE(3), dz = TE(3);
          if (have) {
            if (sizeof(TE) == 8) {
              dx = (TE)(s_off[side][l][0] - s_kw[l][ofs[0] + 3]);
              dy = (TE)(s_off[side][l][1] - s_kw[l][ofs[1] + 3]);
              dz = (TE)(s_off[side][l][2] - s_kw[l][ofs[2] + 3]);
            } else {
              dx = from_double<TE>(s_off[side][l][0]) - s_kwe[l][ofs[0] + 3];
              dy = from_double<TE>(s_off[side][l][1]) - s_kwe[l][ofs[1] + 3];
              dz = from_double<TE>(s_off[side][l][2]) - s_kwe[l][ofs[2] + 3];
            }
          }
          if constexpr (specw && sizeof(TE) == 8) {
            // each side in its own slot, column-scaled, as the pair (hi, lo)
            // of the value in units of 2^k_l (the apply rescales)
            double* Ds = dslot(l, exists ? kt : 0, side);
            const int kl = s_kl[l];
            irregular_group_w2(s_A2, s_W2, p, f2_from_double((double)dx, -kl), f2_from_double((double)dy, -kl),
                               f2_from_double((double)dz, -kl), f2_from_double((double)f, 0),
                               [&](int t2, int n, int m, bool v, f2 vr, f2 vi) {
                                 if (own && v) {
                                   const int kk = rl_re(n, m);
                                   __stcg(reinterpret_cast<float2*>(&Ds[kk]), make_float2(vr.h, vr.l));
                                   if (m) __stcg(reinterpret_cast<float2*>(&Ds[kk + 1]), make_float2(-vi.h, -vi.l));
                                 }
                               });
          } else if constexpr (specw) {
            double* Ds = dslot(l, exists ? kt : 0, side);
            irregular_group_w<TE>(&tabs, s_iW, p, dx, dy, dz, f, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
              if (own && v) {
                const int kk = rl_re(n, m);
                __stcg(&Ds[kk], to_double(vr));
                if (m) __stcg(&Ds[kk + 1], to_double(neg_bits(vi)));
              }
            });
          } else {
            double* Ds = dslot(l, exists ? kt : 0, 0);
            irregular_group_s<TE>(&tabs, p, dx, dy, dz, f, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
              const TE cr = vr, ci = neg_bits(vi);
              const TE orr = __shfl_xor_sync(0xffffffffu, cr, 8);
              const TE oii = __shfl_xor_sync(0xffffffffu, ci, 8);
              if (side == 0 && own && v) {
                const int kk = rl_re(n, m);
                __stcg(&Ds[kk], to_double(cr + orr));
                if (m) __stcg(&Ds[kk + 1], to_double(ci + oii));
              }
            });
          }
        }
        if (prof_on && lane == 0) prof_item(rp.prof, nl <= 4 ? 7 : 8, t_item);
        continue;
      }
      if (spec) {
        // clear the other small-level delta buffer (used again next step)
        const size_t zc = (nsC + nProp - 1) / nProp, z0 = (size_t)it * zc;
        const size_t z1 = z0 + zc < nsC ? z0 + zc : nsC;
        for (size_t zi = z0 + lane; zi < z1; zi += 32) __stcg(&dsm_next[zi], 0.0);
      }
      double partial = 0.0;
      if (k_next && it == iK) {
        // ---- K: dK of the next proposal (drawn and moved exactly as the
        //         proposal code of the next step does); runs on idle steps too
        ptype = 2;
        item_dk<TE>(S, &tabs, rp, t + 1, lane, S.dKpre + (size_t)((t + 1) & 1) * C);
      } else if (idle) {
        // no work: dE is 0 (no move) or +inf (left a free-space box)
        if (it == iX && g.outside) partial = kInf;
        if (it == iU && lane == 0 && rp.mode == 0) part[MC_MAX_ITEMS - 1] = log(u);
        ptype = 3;
      } else if (mm && it >= iE && it < iN) {
        // ---- P: Alg. M.1, the multipole expansions (Eq. multipole
        //      expansion) of entry 2k + grp/2 of IL(alpha) (groups 0, 2) and
        //      IL(alpha') (groups 1, 3) on level l at r and r'
        ptype = 0;
        const int pi = it - iE, lvi = pi / 95, k = pi % 95;
        const int l = L - lvi, sh = L - l, nl = S.lev_n[l];
        const int grp = lane >> 3, side = grp & 1;
        const int co[3] = {g.cf[0] >> sh, g.cf[1] >> sh, g.cf[2] >> sh};
        const int cn[3] = {g.cfn[0] >> sh, g.cfn[1] >> sh, g.cfn[2] >> sh};
        const SmallEntry se = small_entry(il, side ? cn : co, nl, pbc, 2 * k + (grp >> 1));
        TE dx = TE(3), dy = TE(3), dz = TE(3);
        if (se.valid) {
          if (sizeof(TE) == 8) {
            dx = (TE)(s_off[side][l][0] - s_kw[l][se.o[0] + 3]);
            dy = (TE)(s_off[side][l][1] - s_kw[l][se.o[1] + 3]);
            dz = (TE)(s_off[side][l][2] - s_kw[l][se.o[2] + 3]);
          } else {
            dx = from_double<TE>(s_off[side][l][0]) - s_kwe[l][se.o[0] + 3];
            dy = from_double<TE>(s_off[side][l][1]) - s_kwe[l][se.o[1] + 3];
            dz = from_double<TE>(s_off[side][l][2]) - s_kwe[l][se.o[2] + 3];
          }
        }
        const double* Mb =
            S.Mhat + (size_t)(S.lev_off[l] + (se.t3[0] * nl + se.t3[1]) * nl + se.t3[2]) * C;
        // the column polynomials of the irregular sets first (positions
        // only), then the multipoles, which the previous accept may still be
        // writing
        TE qsv[MC_PMAX + 2];
        TE D1r, D1i, D2r, D2i;
        irregular_group_q<TE>(&tabs, p, dx, dy, dz, &D1r, &D1i, &D2r, &D2i,
                              [&](int t2, int n, int m, bool v, bool c1, TE qv) {
                                qsv[t2] = v ? qv : TE(0);
                              });
        need_state();
        double ld[MC_PMAX + 2], lid[MC_PMAX + 2];
#pragma unroll
        for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
          int n, m;
          bool v;
          group_nm(p, t2, &n, &m, &v);
          const int kk = rl_re(n, m);
          ld[t2] = (se.valid && v) ? __ldcg(&Mb[kk]) : 0.0;
          lid[t2] = (se.valid && v && m) ? __ldcg(&Mb[kk + 1]) : 0.0;
        }
        const int m1 = lane & 7, len1 = p - m1 + 1;
        TE SR = TE(0), SI = TE(0), SR1 = TE(0), SI1 = TE(0);
#pragma unroll
        for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
          if (t2 <= p + 1) {
            const bool sw = t2 == len1;  // first step of column 2
            SR1 = sw ? SR : SR1;
            SI1 = sw ? SI : SI1;
            SR = sw ? TE(0) : SR;
            SI = sw ? TE(0) : SI;
            SR += from_double<TE>(ld[t2]) * qsv[t2];
            SI += from_double<TE>(lid[t2]) * qsv[t2];
          }
        }
        TE acc = (m1 ? TE(2) : TE(1)) * (D1r * SR1 - D1i * SI1) + TE(2) * (D2r * SR - D2i * SI);
        acc = group_sum(acc);
        // r' side counts +, r side -; the four groups summed
        TE sv = se.valid ? (side ? acc : -acc) : TE(0);
        sv += __shfl_xor_sync(0xffffffffu, sv, 8);
        sv += __shfl_xor_sync(0xffffffffu, sv, 16);
        partial = g.q * to_double(sv);
      } else if (it >= iE && it < iN) {
        // ---- E: Eq. (2) at r (group 0) and r' (group 1) on level l
        ptype = 0;
        const int l = L - (it - iE), sh = L - l;
        const int grp = lane >> 3, side = grp & 1;
        const int* cc = side ? g.cfn : g.cf;
        const int cx = cc[0] >> sh, cy = cc[1] >> sh, cz = cc[2] >> sh;
        const int nl = S.lev_n[l];
        const double* Lb = S.Lhat + (size_t)(S.lev_off[l] + (cx * nl + cy) * nl + cz) * C;
        const TE dx = from_double<TE>(s_off[side][l][0]), dy = from_double<TE>(s_off[side][l][1]),
                 dz = from_double<TE>(s_off[side][l][2]);
        // the column polynomials first (positions only), then the
        // expansion, which the previous accept may still be writing: each
        // lane contracts its two columns, then applies their diagonal values
        TE qsv[MC_PMAX + 2];
        TE D1r, D1i, D2r, D2i;
        regular_group_q<TE>(&tabs, p, dx, dy, dz, &D1r, &D1i, &D2r, &D2i,
                            [&](int t2, int n, int m, bool v, bool c1, TE qv) {
                              qsv[t2] = v ? qv : TE(0);
                            });
        need_state();
        double ld[MC_PMAX + 2], lid[MC_PMAX + 2];
#pragma unroll
        for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
          int n, m;
          bool v;
          group_nm(p, t2, &n, &m, &v);
          const int k = rl_re(n, m);
          ld[t2] = v ? __ldcg(&Lb[k]) : 0.0;
          lid[t2] = (v && m) ? __ldcg(&Lb[k + 1]) : 0.0;
        }
        const int m1 = lane & 7, len1 = p - m1 + 1;
        TE SR = TE(0), SI = TE(0), SR1 = TE(0), SI1 = TE(0);
#pragma unroll
        for (int t2 = 0; t2 <= MC_PMAX + 1; t2++) {
          if (t2 <= p + 1) {
            const bool sw = t2 == len1;  // first step of column 2
            SR1 = sw ? SR : SR1;
            SI1 = sw ? SI : SI1;
            SR = sw ? TE(0) : SR;
            SI = sw ? TE(0) : SI;
            SR += from_double<TE>(ld[t2]) * qsv[t2];
            SI += from_double<TE>(lid[t2]) * qsv[t2];
          }
        }
        TE acc = (m1 ? TE(2) : TE(1)) * (D1r * SR1 - D1i * SI1) + TE(2) * (D2r * SR - D2i * SI);
        acc = group_sum(acc);
        const TE accn = __shfl_sync(0xffffffffu, acc, 8);
        partial = g.q * to_double(accn - acc);
      } else if (it < iE) {
        // ---- F: far lattice, Sec. 3.4 (iv) in the factored form
        //   dU_inf = sum_k W_k dK_k (H_k + 1/2 (G dK)_k),  W = 1 (m = 0) or 2
        ptype = 2;
        const int f = it - iF;
        const int rb = f / nfc, cb = f % nfc;
        const double c1 = 0.5 * S.a;
        double* st = stage[warp];
        const TE qe = from_double<TE>(g.q);
        const int grp = lane >> 3;
        const double* xg = (grp & 1) ? g.rn : g.r;
        const int k = rb * 32 + lane;
        need_state();
        const double hk = (cb == 0 && k < C) ? __ldcg(&S.Hhat[k]) : 0.0;
        if (dk_pre) {
          const double* src = S.dKpre + (size_t)(t & 1) * C;
          for (int kk = lane; kk < C; kk += 32) st[kk] = __ldcg(&src[kk]);
        } else {
          const TE dx = from_double<TE>(xg[0] - c1), dy = from_double<TE>(xg[1] - c1),
                   dz = from_double<TE>(xg[2] - c1);
          regular_group_s<TE>(&tabs, p, dx, dy, dz, qe, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
            const TE nr = __shfl_xor_sync(0xffffffffu, vr, 8);
            const TE ni = __shfl_xor_sync(0xffffffffu, vi, 8);
            if (grp == 0 && v) {
              // dK = q (conj Rt(r' - R1) - conj Rt(r - R1)), q folded into the sets
              const int kk = rl_re(n, m);
              st[kk] = to_double(nr - vr);
              if (m) st[kk + 1] = to_double(vi - ni);
            }
          });
        }
        __syncwarp();
        const int cbeg = cb * csz, cend = min(C, cbeg + csz);
        double contrib = 0.0;
        if (k < C) {
          double gk = 0.0;
          if (gpre && it == gw) {
#pragma unroll
            for (int i = 0; i < MC_GPRE; i++)
              if (cbeg + i < cend) gk += gcol[i] * st[cbeg + i];
          } else {
            for (int c = cbeg; c < cend; c++) gk += __ldcg(&S.G[(size_t)c * C + k]) * st[c];
          }
          S.gK[(size_t)buf * MC_NF_COLS * C + (size_t)cb * C + k] = gk;
          const double Wk = is_square(k) ? 1.0 : 2.0;
          contrib = Wk * st[k] * (0.5 * gk + hk);
        }
        if (f == 0) {
          for (int kk = lane; kk < C; kk += 32) S.dK[(size_t)buf * C + kk] = st[kk];
        }
        partial = warp_sum(contrib);
        __syncwarp();
      } else if (it < iX) {
        // ---- N: Alg. 1 over one near cell (27 cells of the extended domain)
        ptype = 1;
        const int k0 = it - iN;
        const NearPart np = near_part(k0, same, nNP, nNsame);
        const int k = np.k, side = np.side, part = np.part, nparts = np.nparts;
        item_near<TE>(S, g, s_off, k, side, part, nparts, pbc, lane,
                      [&](int, int, int) {
                        need_state();
                        return true;
                      },
                      &partial);
      } else if (it == iX) {
        // ---- X: periodic self-interaction correction (Sec. 3.4, last item)
        //         and the dipole term (tinfoil reading)
        ptype = 3;
        item_image<TE>(S, g, pbc, lane,
                       [&]() {
                         need_state();
                         return true;
                       },
                       &partial);
      } else if (it == iU) {
        // ---- U: log(u) for the Metropolis test
        ptype = 3;
        if (lane == 0 && rp.mode == 0) part[MC_MAX_ITEMS - 1] = log(u);
      }
      if (mm) {
        wsum += partial;
      } else if (lane == 0) {
        part[it] = partial;
      }
      if (prof_on && lane == 0) prof_item(rp.prof, ptype, t_item);
    }
    if (warp == 0 && pf_ok) {
      // the next proposal's geometry, while the other items still run
      form_geo(pg, pf_j, pf_pos.w, lane == 0 ? pf_pos.x : (lane == 1 ? pf_pos.y : pf_pos.z), pf_d,
               true, pf_u);
      pg_ok = true;
    }
    if (mm) {
      // the multipole method has more items than partial slots: one partial
      // per CTA, summed over its warps in a fixed order
      if (lane == 0) s_wpart[warp] = wsum;
      __syncthreads();
      if (threadIdx.x == 0) {
        double cs = 0.0;
#pragma unroll
        for (int w2 = 0; w2 < MC_WARPS; w2++) cs += s_wpart[w2];
        part[cta] = cs;
      }
    }

    if (prof_lead) {
      tp1 = mc_globaltimer();
      rp.prof[0] += tp1 - tp0;
    }
    gen++;
    if (!grid_barrier(S.bar, gen * (unsigned long long)(nCTA + rp.bar_missing), S.status, rp.wait_ns)) break;
    pend = 0;  // the full barrier covers the previous accept
    if (prof_lead) {
      tp0 = mc_globaltimer();
      rp.prof[1] += tp0 - tp1;
    }

    // ------------------------------------------------ decision (every CTA)
    if (warp == 0) {
      // the partials in one fixed order (loads issued together)
      double v[MC_MAX_ITEMS / 32];
#pragma unroll
      for (int i = 0; i < MC_MAX_ITEMS / 32; i++) {
        const int ii = lane + 32 * i;
        v[i] = ii < (mm ? nCTA : nProp) ? __ldcg(&part[ii]) : 0.0;
      }
      const double lu = (rp.mode == 0 && lane == 0) ? __ldcg(&part[MC_MAX_ITEMS - 1]) : 0.0;
      // only the rows that hold slots (warp-uniform count)
      const int nRows = ((mm ? nCTA : nProp) + 31) / 32;
      double acc = v[0];
#pragma unroll
      for (int i = 1; i < MC_MAX_ITEMS / 32; i++)
        if (i < nRows) acc += v[i];
      acc = warp_sum(acc);
      if (lane == 0) {
        s_dE = acc;
        s_logu = lu;
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
    if (prof_lead) {
      tp1 = mc_globaltimer();
      rp.prof[2] += tp1 - tp0;
      rp.prof[5] += 1;
    }
    mv2 = mv1;
    j2 = j1;
    rn2 = rn1;
    mv1 = accept && !nomove;
    j1 = g.j;
    if (warp == 0 && lane < 3) rn1 = g.rn[lane];
    if (!accept || nomove) {
      if (accept) n_acc++;
      if (accept && cta == 0 && threadIdx.x == 0) S.energy[0] += dE_used;
      if (rp.stop_after_accepts > 0 && n_acc >= rp.stop_after_accepts) break;
      continue;
    }
    n_acc++;

    // ----------------------------------------------- phase B: accept items
    // item 0: bookkeeping; items 1..nKH: K and H += G dK, 32 entries each;
    // then the Alg. L.2 items (applied from the staged contributions, or
    // computed here when not speculating)
    const int nKH = pbc ? (C + 31) / 32 : 0;
    const int nB = 1 + nKH + (mm ? nlev : (spec ? S.nsmall + nLB : nD));
    for (int it = gw; it < nB; it += nWarpsTot) {
      const unsigned long long t_item = prof_on ? mc_globaltimer() : 0ULL;
      if (it == 0) {
        // ---- bookkeeping: dipole, energy, cell lists
        item_bookkeeping(S, g, s_off[1][L], dE_used, lane);
        if (prof_on && lane == 0) prof_item(rp.prof, 6, t_item);
        continue;
      }
      if (it <= nKH) {
        // ---- K += dK, H += G dK (sum of the column-block partials)
        item_kh(S, it - 1, nfc, S.gK + (size_t)buf * MC_NF_COLS * C, S.dK + (size_t)buf * C, lane);
        if (prof_on && lane == 0) prof_item(rp.prof, 6, t_item);
        continue;
      }
      if (mm) {
        // ---- Alg. M.2 on level l: Mhat(alpha) -= q conj Rt(r - R_alpha)
        //      (group 0), Mhat(alpha') += q conj Rt(r' - R_alpha') (group 1)
        const int l = L - (it - 1 - nKH), sh = L - l, nl = S.lev_n[l];
        const int co[3] = {g.cf[0] >> sh, g.cf[1] >> sh, g.cf[2] >> sh};
        const int cn[3] = {g.cfn[0] >> sh, g.cfn[1] >> sh, g.cfn[2] >> sh};
        const int grp = lane >> 3, side = grp & 1;
        const TE f = grp < 2 ? from_double<TE>(side ? g.q : -g.q) : TE(0);
        const TE dx = from_double<TE>(s_off[side][l][0]), dy = from_double<TE>(s_off[side][l][1]),
                 dz = from_double<TE>(s_off[side][l][2]);
        double* st = stage[warp];
        regular_group_s<TE>(&tabs, p, dx, dy, dz, f, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
          if (grp < 2 && v) {
            const int kk = side * 256 + rl_re(n, m);
            st[kk] = to_double(vr);
            if (m) st[kk + 1] = to_double(neg_bits(vi));
          }
        });
        __syncwarp();
        const bool samel = co[0] == cn[0] && co[1] == cn[1] && co[2] == cn[2];
        double* M0 = S.Mhat + (size_t)(S.lev_off[l] + (co[0] * nl + co[1]) * nl + co[2]) * C;
        double* M1 = S.Mhat + (size_t)(S.lev_off[l] + (cn[0] * nl + cn[1]) * nl + cn[2]) * C;
        double v0[8], v1[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const int kk = lane + 32 * i;
          v0[i] = kk < C ? __ldcg(&M0[kk]) : 0.0;
          v1[i] = (kk < C && !samel) ? __ldcg(&M1[kk]) : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const int kk = lane + 32 * i;
          if (kk < C) {
            if (samel) {
              __stcg(&M0[kk], v0[i] + (st[kk] + st[256 + kk]));
            } else {
              __stcg(&M0[kk], v0[i] + st[kk]);
              __stcg(&M1[kk], v1[i] + st[256 + kk]);
            }
          }
        }
        __syncwarp();
        if (prof_on && lane == 0) prof_item(rp.prof, 5, t_item);
        continue;
      }
      // ---- Alg. L.2 items
      if (spec) {
        const int a = it - 1 - nKH;
        if (a < S.nsmall) {
          // small-level cell a (levels with <= 4 cells per axis are the
          // first cells of Lhat): add the step's delta and clear it
          double* Lt = S.Lhat + (size_t)a * C;
          double* Dt = dsm + (size_t)a * C;
          double v[8], w[8];
#pragma unroll
          for (int i = 0; i < 8; i++) {
            const int kk = lane + 32 * i;
            v[i] = kk < C ? __ldcg(&Lt[kk]) : 0.0;
            w[i] = kk < C ? __ldcg(&Dt[kk]) : 0.0;
          }
#pragma unroll
          for (int i = 0; i < 8; i++) {
            const int kk = lane + 32 * i;
            if (kk < C) {
              __stcg(&Lt[kk], specw ? fma(s_P[specw ? kk : 0], w[i], v[i]) : v[i] + w[i]);
              __stcg(&Dt[kk], 0.0);
            }
          }
          if (prof_on && lane == 0) prof_item(rp.prof, 4, t_item);
          continue;
        }
        // large levels: staged target b of level l
        int b = a - S.nsmall, l = L;
        while (l > S.lmin && b >= lev_items[l]) {
          b -= lev_items[l];
          l--;
        }
        const int sh = L - l, nl = S.lev_n[l];
        const int co[3] = {g.cf[0] >> sh, g.cf[1] >> sh, g.cf[2] >> sh};
        const int cn[3] = {g.cfn[0] >> sh, g.cfn[1] >> sh, g.cfn[2] >> sh};
        const LargeItem li = large_item(il, co, cn, nl, pbc, lev_items[l] == 189, b);
        if (li.owner) {
          const double* Ds = dslot(l, b, 0);
          const double* Ds1 = dslot(l, b, 1);
          double* Lt = S.Lhat + (size_t)(S.lev_off[l] + (li.tc[0] * nl + li.tc[1]) * nl + li.tc[2]) * C;
          if constexpr (specw && sizeof(TE) == 8) {
            // L += P_n^m (w + w') 2^(-k_l (n + 1)): the two sides' pairs
            // summed and scaled in pair arithmetic, one FP64 add into L
            const int kl = s_kl[l];
            double v[8];
            float2 w0[8], w1[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
              const int kk = lane + 32 * i;
              v[i] = kk < C ? __ldcg(&Lt[kk]) : 0.0;
              w0[i] = kk < C ? __ldcg(reinterpret_cast<const float2*>(&Ds[kk])) : make_float2(0.0f, 0.0f);
              w1[i] = kk < C ? __ldcg(reinterpret_cast<const float2*>(&Ds1[kk])) : make_float2(0.0f, 0.0f);
            }
#pragma unroll
            for (int i = 0; i < 8; i++) {
              const int kk = lane + 32 * i;
              if (kk < C) {
                const f2 t = f2_mul(s_P2[kk], f2_add({w0[i].x, w0[i].y}, {w1[i].x, w1[i].y}));
                __stcg(&Lt[kk], v[i] + f2_to_double(t, -kl * (s_nn[kk] + 1)));
              }
            }
          } else {
            double v[8], w[8];
#pragma unroll
            for (int i = 0; i < 8; i++) {
              const int kk = lane + 32 * i;
              v[i] = kk < C ? __ldcg(&Lt[kk]) : 0.0;
              w[i] = kk < C ? __ldcg(&Ds[kk]) : 0.0;
              if constexpr (specw) w[i] += kk < C ? __ldcg(&Ds1[kk]) : 0.0;
            }
#pragma unroll
            for (int i = 0; i < 8; i++) {
              const int kk = lane + 32 * i;
              if (kk < C) __stcg(&Lt[kk], specw ? fma(s_P[specw ? kk : 0], w[i], v[i]) : v[i] + w[i]);
            }
          }
        }
        if (prof_on && lane == 0) prof_item(rp.prof, 5, t_item);
        continue;
      }
      const int dk = it - 1 - nKH;
      int l = L;
      while (l > S.lmin && dk >= lev_start[l] + lev_items[l]) l--;
      const int k = dk - lev_start[l];
      const int sh = L - l, nl = S.lev_n[l];
      const int co[3] = {g.cf[0] >> sh, g.cf[1] >> sh, g.cf[2] >> sh};
      const int cn[3] = {g.cfn[0] >> sh, g.cfn[1] >> sh, g.cfn[2] >> sh};
      const int grp = lane >> 3, side = grp & 1;
      if (nl <= 4) {
        // entries 2k (groups 0, 1) and 2k+1 (groups 2, 3) of IL(alpha)
        // (groups 0, 2) and IL(alpha') (groups 1, 3), atomic adds
        const SmallEntry se = small_entry(il, side ? cn : co, nl, pbc, 2 * k + (grp >> 1));
        const TE f = se.valid ? from_double<TE>(side ? g.q : -g.q) : TE(0);
        TE dx = TE(3), dy = TE(3), dz = TE(3);
        if (se.valid) {
          if (sizeof(TE) == 8) {
            dx = (TE)(s_off[side][l][0] - s_kw[l][se.o[0] + 3]);
            dy = (TE)(s_off[side][l][1] - s_kw[l][se.o[1] + 3]);
            dz = (TE)(s_off[side][l][2] - s_kw[l][se.o[2] + 3]);
          } else {
            dx = from_double<TE>(s_off[side][l][0]) - s_kwe[l][se.o[0] + 3];
            dy = from_double<TE>(s_off[side][l][1]) - s_kwe[l][se.o[1] + 3];
            dz = from_double<TE>(s_off[side][l][2]) - s_kwe[l][se.o[2] + 3];
          }
        }
        double* Lt = S.Lhat + (size_t)(S.lev_off[l] + (se.t3[0] * nl + se.t3[1]) * nl + se.t3[2]) * C;
        irregular_group_s<TE>(&tabs, p, dx, dy, dz, f, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
          if (se.valid && v) {
            const int kk = rl_re(n, m);
            red_add_f64(&Lt[kk], to_double(vr));
            if (m) red_add_f64(&Lt[kk + 1], to_double(neg_bits(vi)));
          }
        });
        if (prof_on && lane == 0) prof_item(rp.prof, 4, t_item);
        continue;
      }
      const bool samel = lev_items[l] == 189;
      const LargeItem li = large_item(il, co, cn, nl, pbc, samel, k);
      if (!li.owner) continue;
      const int* cs = side ? cn : co;
      int ofs[3] = {li.ofs[0], li.ofs[1], li.ofs[2]};
      bool have;
      if (samel || (li.from_new && side == 1) || (!li.from_new && side == 0)) {
        have = true;
      } else if (!li.from_new) {
        have = false;  // the target is not in IL(alpha') (else not owner)
      } else {
        list_offset(li.tc, cs, nl, pbc, ofs);
        have = in_il(ofs[0], ofs[1], ofs[2], cs[0], cs[1], cs[2]);
      }
      const TE f = have ? from_double<TE>(side ? g.q : -g.q) : TE(0);
      TE dx = TE(3), dy = TE(3), dz = TE(3);
      if (have) {
        if (sizeof(TE) == 8) {
          dx = (TE)(s_off[side][l][0] - s_kw[l][ofs[0] + 3]);
          dy = (TE)(s_off[side][l][1] - s_kw[l][ofs[1] + 3]);
          dz = (TE)(s_off[side][l][2] - s_kw[l][ofs[2] + 3]);
        } else {
          dx = from_double<TE>(s_off[side][l][0]) - s_kwe[l][ofs[0] + 3];
          dy = from_double<TE>(s_off[side][l][1]) - s_kwe[l][ofs[1] + 3];
          dz = from_double<TE>(s_off[side][l][2]) - s_kwe[l][ofs[2] + 3];
        }
      }
      double* st = stage[warp];
      irregular_group_s<TE>(&tabs, p, dx, dy, dz, f, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
        const TE cr = vr, ci = neg_bits(vi);
        const TE orr = __shfl_xor_sync(0xffffffffu, cr, 8);
        const TE oii = __shfl_xor_sync(0xffffffffu, ci, 8);
        if (grp == 0 && v) {
          const int kk = rl_re(n, m);
          st[kk] = to_double(cr + orr);
          if (m) st[kk + 1] = to_double(ci + oii);
        }
      });
      __syncwarp();
      double* Lt = S.Lhat + (size_t)(S.lev_off[l] + (li.tc[0] * nl + li.tc[1]) * nl + li.tc[2]) * C;
      {
        double v[8];
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const int kk = lane + 32 * i;
          v[i] = kk < C ? __ldcg(&Lt[kk]) : 0.0;
        }
#pragma unroll
        for (int i = 0; i < 8; i++) {
          const int kk = lane + 32 * i;
          if (kk < C) __stcg(&Lt[kk], v[i] + st[kk]);
        }
      }
      __syncwarp();
      if (prof_on && lane == 0) prof_item(rp.prof, 5, t_item);
    }
    if (prof_lead) {
      tp0 = mc_globaltimer();
      rp.prof[3] += tp0 - tp1;
      rp.prof[6] += 1;
    }
    // split barrier: arrive and go on with the next proposal; its reads of
    // the state written above wait for the count (need_state)
    gen++;
    grid_arrive(S.bar);
    pend = gen * (unsigned long long)(nCTA + rp.bar_missing);
    if (prof_lead) rp.prof[4] += mc_globaltimer() - tp0;
    if (rp.stop_after_accepts > 0 && n_acc >= rp.stop_after_accepts) break;
  }
  if (cta == 0 && threadIdx.x == 0) {
    S.stats[0] = steps_done;
    S.stats[1] = n_acc;
    S.stats[2] = n_border;
    S.stats[3] = (long long)(mc_globaltimer() - t_begin);  // this launch's wall time, ns
  }
}

// one chain on the whole grid
template <typename TE, int kVar>
__global__ void __launch_bounds__(MC_THREADS, 1)
    mc_chain_kernel(const McSys* __restrict__ sysp, RunParams rp) {
  chain_body<TE, kVar>(sysp, rp, (int)gridDim.x, (int)blockIdx.x);
}

// many independent chains: CTA b runs chain cta_chain[b] as rank cta_rank[b]
// of that chain's group of chain_ctas[chain] CTAs (each chain has its own
// barrier counter, partials and status in its McSys); per-chain parameters
// in device memory, step counter advanced in place so that a replayed graph
// continues every chain's proposal stream
template <typename TE, int kVar>
__global__ void __launch_bounds__(MC_THREADS, MC_BATCH_CTAS_PER_SM(TE))
    mc_batch_kernel(const McSys* const* __restrict__ systems, RunParams* __restrict__ rps,
                    const int* __restrict__ cta_chain, const int* __restrict__ cta_rank,
                    const int* __restrict__ chain_ctas) {
  const int ch = cta_chain[blockIdx.x];
  RunParams rp = rps[ch];
  const McSys* sys = systems[ch];
  chain_body<TE, kVar>(sys, rp, chain_ctas[ch], cta_rank[blockIdx.x]);
  if (cta_rank[blockIdx.x] == 0 && threadIdx.x == 0) {
    // every CTA of the group read rps[ch] before the group's first barrier
    const long long done = sys->stats[0];
    if (done > 0) rps[ch].step0 = rp.step0 + done;
  }
}

template __global__ void mc_chain_kernel<double, MC_VAR_PLAIN>(const McSys*, RunParams);
template __global__ void mc_chain_kernel<float, MC_VAR_PLAIN>(const McSys*, RunParams);
template __global__ void mc_chain_kernel<double, MC_VAR_SPEC>(const McSys*, RunParams);
template __global__ void mc_chain_kernel<float, MC_VAR_SPEC>(const McSys*, RunParams);
template __global__ void mc_chain_kernel<double, MC_VAR_MM>(const McSys*, RunParams);
template __global__ void mc_chain_kernel<float, MC_VAR_MM>(const McSys*, RunParams);

namespace {
template <int V>
const void* chain_fn(int prec) {
  return prec ? (const void*)mc_chain_kernel<float, V> : (const void*)mc_chain_kernel<double, V>;
}
template <int V>
cudaError_t batch_launch(const cudaLaunchConfig_t* cfg, int prec, const McSys* const* d_systems,
                         RunParams* d_rps, const int* d_cta_chain, const int* d_cta_rank,
                         const int* d_chain_ctas) {
  if (prec)
    return cudaLaunchKernelEx(cfg, mc_batch_kernel<float, V>, d_systems, d_rps, d_cta_chain,
                              d_cta_rank, d_chain_ctas);
  return cudaLaunchKernelEx(cfg, mc_batch_kernel<double, V>, d_systems, d_rps, d_cta_chain,
                            d_cta_rank, d_chain_ctas);
}
}  // namespace

// host-side launchers (cooperative launches: all CTAs co-resident)
cudaError_t mc_launch_chain(const McSys* d_sys, const RunParams& rp, int prec, int var, int nCTA,
                            cudaStream_t stream) {
  void* args[] = {(void*)&d_sys, (void*)&rp};
  const void* fn = var == MC_VAR_MM     ? chain_fn<MC_VAR_MM>(prec)
                   : var == MC_VAR_SPEC ? chain_fn<MC_VAR_SPEC>(prec)
                                        : chain_fn<MC_VAR_PLAIN>(prec);
  return cudaLaunchCooperativeKernel(fn, dim3(nCTA), dim3(MC_THREADS), args, 0, stream);
}

cudaError_t mc_launch_batch(const McSys* const* d_systems, RunParams* d_rps, const int* d_cta_chain,
                            const int* d_cta_rank, const int* d_chain_ctas, int prec, int var,
                            int nCTA, cudaStream_t stream) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(nCTA);
  cfg.blockDim = dim3(MC_THREADS);
  cfg.dynamicSmemBytes = 0;
  cfg.stream = stream;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (var == MC_VAR_MM)
    return batch_launch<MC_VAR_MM>(&cfg, prec, d_systems, d_rps, d_cta_chain, d_cta_rank, d_chain_ctas);
  if (var == MC_VAR_SPECW && !prec)  // (FP64 only)
    return cudaLaunchKernelEx(&cfg, mc_batch_kernel<double, MC_VAR_SPECW>, d_systems, d_rps, d_cta_chain,
                              d_cta_rank, d_chain_ctas);
  if (var == MC_VAR_SPECW)
    return batch_launch<MC_VAR_SPEC>(&cfg, prec, d_systems, d_rps, d_cta_chain, d_cta_rank, d_chain_ctas);
  if (var == MC_VAR_SPEC)
    return batch_launch<MC_VAR_SPEC>(&cfg, prec, d_systems, d_rps, d_cta_chain, d_cta_rank,
                                     d_chain_ctas);
  return batch_launch<MC_VAR_PLAIN>(&cfg, prec, d_systems, d_rps, d_cta_chain, d_cta_rank,
                                    d_chain_ctas);
}

// CTAs the batched form can keep co-resident (its kernels' occupancy x SMs)
int mc_batch_max_ctas(int prec) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fns[4][2] = {
      {(const void*)mc_batch_kernel<double, MC_VAR_PLAIN>, (const void*)mc_batch_kernel<float, MC_VAR_PLAIN>},
      {(const void*)mc_batch_kernel<double, MC_VAR_SPEC>, (const void*)mc_batch_kernel<float, MC_VAR_SPEC>},
      {(const void*)mc_batch_kernel<double, MC_VAR_MM>, (const void*)mc_batch_kernel<float, MC_VAR_MM>},
      {(const void*)mc_batch_kernel<double, MC_VAR_SPECW>, (const void*)mc_batch_kernel<float, MC_VAR_SPEC>}};
  int best = 1 << 30;
  for (int v = 0; v < 4; v++) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fns[v][prec ? 1 : 0], MC_THREADS, 0) !=
        cudaSuccess)
      return 0;
    best = std::min(best, per);
  }
  const int cap = prec ? MC_BATCH_CTAS_PER_SM(float) : MC_BATCH_CTAS_PER_SM(double);
  return best < 1 ? 0 : sms * std::min(best, cap);
}

int mc_chain_max_ctas(int prec) {
  int dev = 0, sms = 0, per = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const void* fn = chain_fn<MC_VAR_SPEC>(prec);
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, fn, MC_THREADS, 0);
  if (per < 1) return 0;
  return sms;  // one CTA per SM
}
