// Asynchronous persistent chain kernel (MC_SCHEDULE_ASYNC): the steps of
// Alg. L.1 (propose, with Alg. 1 and the periodic terms of Sec. 3.4) and
// Alg. L.2 (accept, its contributions computed speculatively) for one
// system, with no grid or CTA barrier inside the step loop.  Warps meet
// only through data:
//   * one control warp per CTA (warp 0) publishes the proposal geometry of
//     step t in a 4-deep shared-memory ring, then polls the partial sums of
//     step t (4-deep ring of slots in global memory, each slot reset to a
//     sentinel before its reuse), makes the Metropolis decision (the same
//     slots summed in the same order in every CTA) and publishes it;
//   * heavy warps (1..3, one per SM sub-partition, then warp 4 beside the
//     control warp) run the FP64-heavy items: K (dK of the next proposal),
//     E (Eq. 2 at r and r' per level) and the speculative Alg. L.2
//     contributions;
//   * light warps (5..7) run the near-field (Alg. 1), far-lattice, image and
//     log(u) items and the apply items (bookkeeping, K/H, the staged Alg.
//     L.2 contributions added into the expansions): an apply item loads its
//     operands once the contributions and the previous accepts are complete,
//     and after an accepting decision only adds, stores and counts itself on
//     an arrival counter.
// Reads of state that an accept writes (expansions, cell lists, H, dipole)
// wait for the arrival count of all earlier accepts; the apply of step t
// waits for the contribution counter of step t; the decision of step t also
// waits for the contributions of step t-1, which bounds how far the
// speculative work lags behind (at most one step), so every step-indexed
// buffer (4 deep by step) is free before the step that reuses it starts.
// Heavy items never wait for a decision: the geometry of step t+1 is
// published before decision t (unless both steps draw the same particle),
// so its contributions run while step t is still being decided and applied.
// Every wait is bounded by wall time; on expiry the status word is set and
// all warps leave the loop.
#include "mc_items.cuh"

#include <algorithm>

#define MC_ASYNC_CTRL 0   // control warp (sub-partition 0)
#define MC_ASYNC_HEAVY 4  // warps 1..4: 1..3 first (sub-partitions 1..3), 4 beside the control warp
#define MC_ASYNC_LIGHT 3  // warps 5..7

namespace {

constexpr unsigned long long kSentinel = 0xFFFFFFFFFFFFFFFFull;
constexpr double kInfA = __builtin_huge_val();

__device__ __forceinline__ void st_release_f64(double* p, double v) {
  unsigned long long b = (unsigned long long)__double_as_longlong(v);
  if (b == kSentinel) b = 0x7FF8000000000000ull;  // a computed NaN never reads as "not yet"
  asm volatile("st.release.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(b) : "memory");
}

__device__ __forceinline__ unsigned long long ld_relaxed_b64(const void* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// four relaxed loads in one statement: all four are in flight together
// (one L2 round trip), the results are waited for where they are used
__device__ __forceinline__ void ld_relaxed_x4(const void* p0, const void* p1, const void* p2, const void* p3,
                                              unsigned long long* v) {
  asm volatile(
      "ld.relaxed.gpu.global.b64 %0, [%4];\n\t"
      "ld.relaxed.gpu.global.b64 %1, [%5];\n\t"
      "ld.relaxed.gpu.global.b64 %2, [%6];\n\t"
      "ld.relaxed.gpu.global.b64 %3, [%7];"
      : "=l"(v[0]), "=l"(v[1]), "=l"(v[2]), "=l"(v[3])
      : "l"(p0), "l"(p1), "l"(p2), "l"(p3)
      : "memory");
}

__device__ __forceinline__ void red_release_add(unsigned long long* p, unsigned long long v) {
  asm volatile("red.release.gpu.global.add.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// shared-memory flag: writer fences the block then stores; reader polls
// (lane 0), fences, and the warp synchronises
__device__ __forceinline__ void flag_publish(volatile long long* f, long long v) {
  __threadfence_block();
  *f = v;
}

// one warp waits until *f >= v; false on abort, error status or timeout
__device__ __forceinline__ bool flag_wait(volatile long long* f, long long v, volatile int* abort_flag,
                                          int* status, long long wait_ns) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    if (*f < v) {
      const unsigned long long t0 = mc_globaltimer();
      unsigned spins = 0;
      while (*f < v) {
        if (*abort_flag) {
          ok = 0;
          break;
        }
        // back off: a spinning warp takes issue slots from the warps that
        // share its sub-partition
        if (spins >= 4u) __nanosleep(100);
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
    __threadfence_block();
  }
  ok = __shfl_sync(0xffffffffu, ok, 0);
  __syncwarp();
  return ok != 0;
}

// one warp waits for a global counter to reach target (lane 0 polls with
// relaxed loads and back-off, bounded by wait_ns; an acquire-only fence once
// reached: it orders the warp's later accesses after the writes released
// with the counted arrivals, without waiting for the warp's own earlier
// writes as an acq_rel fence would); false on timeout or when another CTA
// has set an error status
__device__ __forceinline__ bool counter_wait(unsigned long long* ctr, unsigned long long target,
                                             int* status, long long wait_ns) {
  int ok = 1;
  if ((threadIdx.x & 31) == 0) {
    unsigned long long v = ld_relaxed_b64(ctr);
    if (v < target) {
      const unsigned long long t0 = mc_globaltimer();
      unsigned spins = 0;
      while (true) {
        // a few polls back to back, then a short back-off (measured on
        // GB300: +0.4 % over backing off from the third poll; longer
        // back-offs delay these waits, which are on the step's critical path)
        if (spins >= 8u) __nanosleep(100);
        v = ld_relaxed_b64(ctr);
        if (v >= target) break;
        if ((++spins & 31u) == 0u) {
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

}  // namespace

template <typename TE>
__device__ __forceinline__ void async_body(const McSys* __restrict__ sysp, RunParams& rp,
                                           const int nCTA, const int cta) {
  __shared__ McSys S;
  __shared__ HarmTabs<TE> tabs;
  __shared__ unsigned short il[8][189];
  __shared__ double stage[MC_WARPS][256];
  __shared__ TE s_iW[MC_PMAX + 1][16];
  __shared__ double s_P[(MC_PMAX + 1) * (MC_PMAX + 1)];
  __shared__ double s_kw[MC_MAXLEV + 2][7];
  __shared__ TE s_kwe[MC_MAXLEV + 2][7];
  // rings by step (t & 3): geometry, offsets of r / r' from their cell
  // centres per level, u; decision
  __shared__ StepGeo s_geo[4];
  __shared__ double s_off[4][2][MC_MAXLEV + 2][3];
  __shared__ double s_u[4];
  __shared__ unsigned long long s_tpub[4];  // publication times (profiling)
  // decision ring, 8 deep: a warp reads decisions of its steps t-2..t, and
  // no warp is more than 4 steps behind a published geometry
  __shared__ double s_dEu[8];
  __shared__ int s_acc[8];
  __shared__ unsigned long long s_cumB[8];  // apply items of the accepted steps through step s
  __shared__ volatile long long s_gstep;  // last published geometry step
  __shared__ volatile long long s_dstep;  // last published decision step
  __shared__ volatile long long s_stop;   // steps of this launch (set when the chain stops)
  __shared__ volatile long long s_wdone[MC_WARPS];
  __shared__ volatile int s_abort;
  __shared__ long long s_stats[3];

  const unsigned long long t_begin = mc_globaltimer();
  if (threadIdx.x == 0) {
    S = *sysp;
    s_gstep = -1;
    s_dstep = -1;
    s_stop = rp.nsteps;
    s_abort = 0;
  }
  if (threadIdx.x < MC_WARPS) s_wdone[threadIdx.x] = -1;
  harm_tabs_init<TE>(&tabs);
  irregular_w_tabs<TE>(s_iW, s_P);
  il_table_init(il);
  __syncthreads();
  for (int i = threadIdx.x; i < (MC_MAXLEV + 2) * 7; i += blockDim.x) {
    const int l = i / 7, k = i % 7 - 3;
    const double v = (l >= 1 && l <= S.L) ? k * S.lev_w[l] : 0.0;
    s_kw[l][k + 3] = v;
    s_kwe[l][k + 3] = (TE)v;
  }
  __syncthreads();

  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int p = S.p, C = S.C, L = S.L;
  const bool pbc = (S.bc == 0);
  const bool prof_on = rp.prof != nullptr;
  const int nlev = L - S.lmin + 1;
  const int nRB = (C + 31) / 32;
  const int nfc = rp.nf_cols;
  const int nF = pbc ? nRB * nfc : 0;
  const int csz = (C + nfc - 1) / nfc;
  const int nE = 4 * nlev;  // E items: four quarter contractions per level
  // light phase-A slots: F, N (54 x near_parts), X, U; heavy slots: K, E,
  // contributions
  const int nNP = S.near_parts, nNI = 54 * nNP;
  const int iN = nF, iX = nF + nNI, iU = iX + 1, nLA = iX + 2;
  const int slotE = nLA;  // partial slots of the E items
  const int nSlots = nLA + nE;
  const int hK = 0, hE = 1, hD = 1 + nE;
  const int nHw = MC_ASYNC_HEAVY * nCTA, nLw = MC_ASYNC_LIGHT * nCTA;
  const bool heavy = warp >= 1 && warp <= MC_ASYNC_HEAVY;
  const bool light = warp > MC_ASYNC_HEAVY;
  const int hw = (warp - 1) * nCTA + cta;
  const int lw = (warp - MC_ASYNC_HEAVY - 1) * nCTA + cta;
  const int bstart = nLw - 1 - lw;  // first apply item of a light warp
  const size_t nsC = (size_t)S.nsmall * C;
  // counters on their own 128-byte lines (sync[16 i]): [1..4] contributions
  // done by step mod 4, [5] K item of step s done (s + 1), [6] decisions made
  unsigned long long* dcnt = S.sync + 16;      // dcnt[16 i]: step mod 4 = i
  unsigned long long* ktag = S.sync + 16 * 5;
  unsigned long long* decdone = S.sync + 16 * 6;

  // far operator columns kept in registers by the light warp of F item lw
  const bool gpre = nF <= nLw && csz <= MC_GPRE;
  double gcol[MC_GPRE];
#pragma unroll
  for (int i = 0; i < MC_GPRE; i++) gcol[i] = 0.0;
  if (light && gpre && lw < nF) {
    const int k = (lw / nfc) * 32 + lane, cbeg = (lw % nfc) * csz;
#pragma unroll
    for (int i = 0; i < MC_GPRE; i++) {
      const int c = cbeg + i;
      if (k < C && i < csz && c < C) gcol[i] = __ldcg(&S.G[(size_t)c * C + k]);
    }
  }

  if (warp == MC_ASYNC_CTRL) {
    // ================================================= control warp
    long long n_acc = 0, n_border = 0, steps_done = 0;
    bool mv1 = false, mv2 = false;
    int j1 = -1, j2 = -1;
    double rn1 = 0.0, rn2 = 0.0;
    unsigned long long cumD[4] = {0ull, 0ull, 0ull, 0ull};  // contributions by step mod 4
    struct PGeo {
      int j, cf, cfn, lo;
      double q, uu, r, rn;
      double off[3];
      bool out;
    } pg;
    pg.j = -1;
    // whole warp: j, charge, r (lanes 0..2), displacement; offsets from the
    // cell centres per level (side lane/16, level slot lane%16)
    auto form_geo = [&](PGeo& G, int j, double q, double r, double dn, double uu) {
      double rn = 0.0;
      bool out = false;
      if (lane < 3) {
        double x = __dadd_rn(r, dn);
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
    auto draw = [&](long long s, int* j, double* d, double* uu, double4* pos) {
      mc_proposal_axis(rp.seed, (unsigned long long)(rp.step0 + s), rp.chain, S.n, rp.h,
                       lane < 3 ? lane : 0, j, d, lane == 3 ? uu : nullptr);
      *uu = __shfl_sync(0xffffffffu, *uu, 3);
      *pos = lane < 3 ? ldcg4(&S.ppos[*j]) : make_double4(0, 0, 0, 0);
      const double w = __shfl_sync(0xffffffffu, pos->w, 0);
      pos->w = w;
    };
    auto axis = [&](const double4& v) { return lane == 0 ? v.x : (lane == 1 ? v.y : v.z); };
    // publication of the geometry of step s (ring slot s & 3, whose
    // previous step s - 4 every item warp has finished)
    long long published = -1;
    auto publish = [&](long long s) -> bool {
      if (s >= 4) {
        for (int w2 = 0; w2 < MC_WARPS; w2++)
          if (w2 != MC_ASYNC_CTRL && !flag_wait(&s_wdone[w2], s - 4, &s_abort, S.status, rp.wait_ns))
            return false;
      }
      const int si = (int)(s & 3);
      if (pg.lo) {
        const int side = lane >> 4;
#pragma unroll
        for (int ax = 0; ax < 3; ax++) s_off[si][side][pg.lo][ax] = pg.off[ax];
      }
      if (lane < 3) {
        s_geo[si].r[lane] = pg.r;
        s_geo[si].rn[lane] = pg.rn;
        s_geo[si].cf[lane] = pg.cf;
        s_geo[si].cfn[lane] = pg.cfn;
      }
      if (lane == 0) {
        s_geo[si].j = pg.j;
        s_geo[si].q = pg.q;
        s_geo[si].outside = pg.out;
        s_u[si] = pg.uu;
      }
      __syncwarp();
      if (lane == 0) {
        s_tpub[si] = prof_on ? mc_globaltimer() : 0ull;
        flag_publish(&s_gstep, s);
      }
      __syncwarp();
      published = s;
      return true;
    };
    double pf_d = 0.0;
    double4 pf_pos = make_double4(0, 0, 0, 0);
    long long t = 0;
    bool ok = true;
    unsigned long long cumB = 0ull;  // apply items of the accepted steps so far
    // proposal 0
    {
      double uu = 0.5;
      int j;
      draw(0, &j, &pf_d, &uu, &pf_pos);
      form_geo(pg, j, pf_pos.w, axis(pf_pos), pf_d, uu);
      if (rp.nsteps > 0) ok = publish(0);
    }
    for (; t < rp.nsteps && ok; t++) {
      const int gi = (int)(t & 3);
      if (published < t) {
        // held back: its particle was the previous step's; the position
        // with the moves of steps t-2 and t-1 (decided now) applied
        double r = axis(pf_pos);
        if (lane < 3) {
          if (mv2 && pg.j == j2) r = rn2;
          if (mv1 && pg.j == j1) r = rn1;
        }
        form_geo(pg, pg.j, pf_pos.w, r, pf_d, pg.uu);
        if (!publish(t)) {
          ok = false;
          break;
        }
      }
      const unsigned long long t_pub = s_tpub[gi];
      // step quantities the decision needs (as every warp forms them)
      const StepGeo g = s_geo[gi];
      const bool nomove = (g.r[0] == g.rn[0] && g.r[1] == g.rn[1] && g.r[2] == g.rn[2]);
      const bool idle = nomove || g.outside;
      int nDs = 0, nLB2 = 0;
      for (int l = L; l >= S.lmin; l--) {
        const int sh = L - l;
        const bool samel = ((g.cf[0] >> sh) == (g.cfn[0] >> sh)) &&
                           ((g.cf[1] >> sh) == (g.cfn[1] >> sh)) &&
                           ((g.cf[2] >> sh) == (g.cfn[2] >> sh));
        const int it_l = (S.lev_n[l] <= 4) ? 95 : (samel ? 95 : 189);
        nDs += it_l;
        if (S.lev_n[l] > 4) nLB2 += it_l;
      }
      const int nB = 1 + (pbc ? (C + 31) / 32 : 0) + S.nsmall + nLB2;
      // ---- proposal t+1: its position load holds every move up to step
      //      t-2 (their applies preceded this warp's last decision); the
      //      decided move of step t-1 is put in here.  Published at once
      //      unless it draws the particle of step t, whose move is not
      //      decided yet
      if (t + 1 < rp.nsteps) {
        int j;
        double uu = 0.5;
        draw(t + 1, &j, &pf_d, &uu, &pf_pos);
        double r = axis(pf_pos);
        if (lane < 3 && mv1 && j == j1) r = rn1;
        form_geo(pg, j, pf_pos.w, r, pf_d, uu);
        if (j != g.j && !publish(t + 1)) {
          ok = false;
          break;
        }
      }
      if (prof_on && cta == 0 && lane == 0) rp.prof[1] += mc_globaltimer() - t_pub;
      // ---- decision of step t: the partial slots of this step, log(u),
      //      and the contributions of step t-1 (bounded lag)
      const double* part = S.partials + (size_t)gi * MC_MAX_ITEMS;
      const unsigned long long dprev = t > 0 ? cumD[(t - 1) & 3] : 0ull;
      constexpr int kRows = MC_MAX_ITEMS / 32;
      static_assert(kRows % 4 == 0, "the poll loads rows in groups of four");
      unsigned long long bb[kRows];
      double lu = 0.0;
      const int nRows = (nSlots + 31) / 32;  // warp-uniform
      {
        // slot of row i that this lane polls (a row past the slots repeats
        // the lane's slot of row 0: loaded, never used); lane 0 also polls
        // log u and the contribution counter of step t-1.  Each poll is one
        // round trip for every row at once; the back-off between polls
        // (measured on GB300: 50 ns slowed the step's items, 150-500 ns
        // gave +3-4 % over the row-by-row poll) keeps the polling loads of
        // 152 control warps from crowding the memory pipes of the items
        auto slot = [&](int i) -> const void* {
          return &part[lane + 32 * i < nSlots ? lane + 32 * i : lane];
        };
        const void* dc = t > 0 ? (const void*)&dcnt[16 * ((t - 1) & 3)] : (const void*)&part[lane];
        const unsigned long long t0 = mc_globaltimer();
        unsigned spins = 0;
        while (true) {
          unsigned long long bx[4] = {0ull, 0ull, 0ull, 0ull};
#pragma unroll
          for (int g4 = 0; g4 < kRows; g4 += 4) {
            if (g4 == 0 || g4 < nRows) {
              ld_relaxed_x4(slot(g4), slot(g4 + 1), slot(g4 + 2), slot(g4 + 3), &bb[g4]);
            } else {
              bb[g4] = bb[g4 + 1] = bb[g4 + 2] = bb[g4 + 3] = 0ull;
            }
          }
          if (lane == 0) ld_relaxed_x4(&part[MC_MAX_ITEMS - 1], dc, slot(0), slot(0), bx);
          bool all = true;
#pragma unroll
          for (int i = 0; i < kRows; i++) all = all && (lane + 32 * i >= nSlots || bb[i] != kSentinel);
          if (lane == 0) {
            all = all && (bx[0] != kSentinel);
            lu = __longlong_as_double((long long)bx[0]);
            if (t > 0) all = all && (bx[1] >= dprev);
            if (rp.bar_missing) all = false;  // failure-path test: never complete
          }
          if (__all_sync(0xffffffffu, all)) break;
          __nanosleep(350);
          int bad = 0;
          if (lane == 0 && (++spins & 63u) == 0u) {
            if ((long long)(mc_globaltimer() - t0) > rp.wait_ns) {
              atomicExch(S.status, MCD_ERR_TIMEOUT);
              bad = 1;
            } else if (*((volatile int*)S.status) != MCD_OK) {
              bad = 1;
            }
          }
          if (__shfl_sync(0xffffffffu, bad, 0)) {
            ok = false;
            break;
          }
        }
        if (!ok) break;
        asm volatile("fence.acquire.gpu;" ::: "memory");
      }
      // the same fixed order in every CTA; only the rows that hold slots
      // (every FP64 add here is on the step's critical path)
      double acc = __longlong_as_double((long long)(lane < nSlots ? bb[0] : 0ull));
#pragma unroll
      for (int i = 1; i < kRows; i++)
        if (i < nRows) acc += lane + 32 * i < nSlots ? __longlong_as_double((long long)bb[i]) : 0.0;
      const double dE = warp_sum(acc);
      lu = __shfl_sync(0xffffffffu, lu, 0);
      const double t2 = -rp.beta * dE;
      const bool accept = dE <= 0.0 || lu < t2;
      if (accept && !nomove) cumB += (unsigned long long)nB;
      if (lane == 0) {
        s_dEu[t & 7] = dE;
        s_acc[t & 7] = accept ? 1 : 0;
        s_cumB[t & 7] = cumB;
        flag_publish(&s_dstep, t);
        red_release_add(decdone, 1ull);
        if (cta == 0) {
          if (rp.log_j) {
            rp.log_j[t] = g.j;
            rp.log_dE[t] = dE;
            rp.log_acc[t] = accept ? 1 : 0;
          }
          if (accept && nomove) S.energy[0] += dE;
          if (prof_on) {
            rp.prof[0] += mc_globaltimer() - t_pub;
            rp.prof[5] += 1;
            if (accept && !nomove) rp.prof[6] += 1;
          }
        }
      }
      __syncwarp();
      // decisions within 1e-9 of the threshold (counted after publishing)
      if (dE > 0.0 && fabs(lu - t2) < 1e-9 * fmax(1.0, fabs(t2))) n_border++;
      if (!idle) cumD[t & 3] += (unsigned long long)nDs;
      steps_done++;
      if (accept) n_acc++;
      mv2 = mv1;
      j2 = j1;
      rn2 = rn1;
      mv1 = accept && !nomove;
      j1 = g.j;
      if (lane < 3) rn1 = g.rn[lane];
      if (rp.stop_after_accepts > 0 && n_acc >= rp.stop_after_accepts) {
        t++;
        break;
      }
    }
    if (lane == 0) {
      // the item warps leave at the first wait past the last decided step
      // (a step published early but not decided is left undone)
      s_stop = t;
      flag_publish(&s_gstep, 1ll << 62);
      flag_publish(&s_dstep, 1ll << 62);
      if (!ok) s_abort = 1;
      s_stats[0] = steps_done;
      s_stats[1] = n_acc;
      s_stats[2] = n_border;
    }
    __syncwarp();
  } else {
    // ================================================= item warps
    unsigned long long cumD[4] = {0ull, 0ull, 0ull, 0ull};  // contributions by step mod 4
    // particle and no-move flag of the two previous steps
    int j_prev = -1, j_prev2 = -1;
    bool nomove_prev = true, nomove_prev2 = true;
    for (long long t = 0;; t++) {
      if (!flag_wait(&s_gstep, t, &s_abort, S.status, rp.wait_ns)) {
        s_abort = 1;
        break;
      }
      if (t >= s_stop) break;
      const int gi = (int)(t & 3);
      const StepGeo g = s_geo[gi];
      const double(*off)[MC_MAXLEV + 2][3] = s_off[gi];
      const bool nomove = (g.r[0] == g.rn[0] && g.r[1] == g.rn[1] && g.r[2] == g.rn[2]);
      const bool same = (g.cf[0] == g.cfn[0] && g.cf[1] == g.cfn[1] && g.cf[2] == g.cfn[2]);
      const bool idle = nomove || g.outside;
      int lev_items[MC_MAXLEV + 2], sp_start[MC_MAXLEV + 2];
      int nDs = 0, nLB2 = 0;
      for (int l = L; l >= S.lmin; l--) {
        const int sh = L - l;
        const bool samel = ((g.cf[0] >> sh) == (g.cfn[0] >> sh)) &&
                           ((g.cf[1] >> sh) == (g.cfn[1] >> sh)) &&
                           ((g.cf[2] >> sh) == (g.cfn[2] >> sh));
        lev_items[l] = (S.lev_n[l] <= 4) ? 95 : (samel ? 189 : 378);
        sp_start[l] = nDs;
        nDs += (S.lev_n[l] <= 4) ? 95 : (lev_items[l] + 1) / 2;
        if (S.lev_n[l] > 4) nLB2 += (lev_items[l] + 1) / 2;
      }
      const int nHeavy = hD + (idle ? 0 : nDs);
      if (!idle) cumD[t & 3] += (unsigned long long)nDs;
      const int nKH = pbc ? (C + 31) / 32 : 0;
      const int nB = 1 + nKH + S.nsmall + nLB2;
      // the geometry of step t can be published before the decision of step
      // t-1: state reads first wait for that decision, then for the apply
      // items of every accepted step through t-1
      bool have_prev = t == 0, halt = false;
      unsigned long long pend = 0ull;
      auto sync_prev = [&]() -> bool {
        if (!have_prev) {
          if (!flag_wait(&s_dstep, t - 1, &s_abort, S.status, rp.wait_ns)) return false;
          if (t - 1 >= s_stop) {
            halt = true;
            return false;
          }
          pend = s_cumB[(t - 1) & 7];
          have_prev = true;
        }
        return true;
      };
      auto need_state = [&]() -> bool {
        if (!sync_prev()) return false;
        return pend == 0ull || counter_wait(S.bar, pend, S.status, rp.wait_ns);
      };
      // staged contributions: by step mod 4, level and side, MC_DSLOTS x C
      auto dslot = [&](int l, int slot, int side) -> double* {
        return S.dacc + ((((size_t)(t & 3) * nlev + (L - l)) * 2 + side) * MC_DSLOTS + slot) * C;
      };
      double* dsm = S.dsmall + (size_t)(t & 3) * nsC;
      double* dsm_clear = S.dsmall + (size_t)((t + 2) & 3) * nsC;
      double* part = S.partials + (size_t)gi * MC_MAX_ITEMS;
      double* part_next = S.partials + (size_t)((t + 1) & 3) * MC_MAX_ITEMS;
      bool fail = false;
      // the owner of a partial slot resets its next-step entry (last read by
      // the decisions of step t-3, which every CTA has made)
      auto reset_next = [&](int slot) -> bool {
        if (t >= 3 && !counter_wait(decdone, (unsigned long long)nCTA * (unsigned long long)(t - 2), S.status,
                                 rp.wait_ns))
          return false;
        if (lane == 0) {
          *(unsigned long long*)&part_next[slot] = kSentinel;
          if (slot == iU) *(unsigned long long*)&part_next[MC_MAX_ITEMS - 1] = kSentinel;
        }
        return true;
      };
      auto put = [&](int slot, double v) {
        __syncwarp();
        if (lane == 0) st_release_f64(&part[slot], v);
      };

      if (heavy) {
        // ------------------------------------------------ heavy items
        for (int it = hw; it < nHeavy && !fail; it += nHw) {
          const unsigned long long t_item = prof_on ? mc_globaltimer() : 0ULL;
          if (it == hK) {
            // ---- K: dK of the next proposal (drawn and moved exactly as
            //      the control warp will), for the far items of step t+1
            if (t + 1 < rp.nsteps && pbc) {
              // the position load holds every move up to step t-2 (the far
              // items of step t+1 use this dK only if steps t-1 and t did not
              // move the particle)
              if (t >= 2) {
                if (!flag_wait(&s_dstep, t - 2, &s_abort, S.status, rp.wait_ns) ||
                    !counter_wait(S.bar, s_cumB[(t - 2) & 7], S.status, rp.wait_ns)) {
                  fail = true;
                  break;
                }
              }
              item_dk<TE>(S, &tabs, rp, t + 1, lane, S.dKpre + (size_t)((t + 1) & 3) * C);
              __syncwarp();
              if (lane == 0) {
                asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(ktag),
                             "l"((unsigned long long)(t + 1)) : "memory");
              }
            }
            if (prof_on && lane == 0) prof_item(rp.prof, 2, t_item);
            continue;
          }
          if (it < hD) {
            // ---- E: Eq. (2) at r (group 0) and r' (group 1) on level l,
            //      quarter qd of the recurrence steps of every lane
            const int e = it - hE;
            const int lv = e >> 2, qd = e & 3;
            if (!reset_next(slotE + e)) {
              fail = true;
              break;
            }
            double partial = 0.0;
            if (!idle) {
              const int l = L - lv, sh = L - l;
              const int grp = lane >> 3, side = grp & 1;
              const int* cc = side ? g.cfn : g.cf;
              const int cx = cc[0] >> sh, cy = cc[1] >> sh, cz = cc[2] >> sh;
              const int nl = S.lev_n[l];
              const double* Lb = S.Lhat + (size_t)(S.lev_off[l] + (cx * nl + cy) * nl + cz) * C;
              const TE dx = from_double<TE>(off[side][l][0]), dy = from_double<TE>(off[side][l][1]),
                       dz = from_double<TE>(off[side][l][2]);
              constexpr int kQ = (MC_PMAX + 2 + 3) / 4;  // recurrence steps per quarter
              TE qsv[4 * kQ];
#pragma unroll
              for (int i = 0; i < 4 * kQ; i++) qsv[i] = TE(0);  // steps past p + 1 stay 0
              TE D1r, D1i, D2r, D2i;
              regular_group_q<TE>(&tabs, p, dx, dy, dz, &D1r, &D1i, &D2r, &D2i,
                                  [&](int t2, int n, int m, bool v, bool c1, TE qv) {
                                    qsv[t2] = v ? qv : TE(0);
                                  });
              // this quarter's steps t2 = qd kQ + i (columns m1 then m2 of
              // the lane), their polynomials selected out of the registers
              TE qq[kQ];
#pragma unroll
              for (int i = 0; i < kQ; i++)
                qq[i] = qd == 0 ? qsv[i] : (qd == 1 ? qsv[kQ + i] : (qd == 2 ? qsv[2 * kQ + i] : qsv[3 * kQ + i]));
              if (!need_state()) {
                fail = true;
                break;
              }
              if (prof_on && lane == 0) prof_item(rp.prof, 9, s_tpub[gi]);
              const int m1 = lane & 7, len1 = p - m1 + 1;
              double ld[kQ], lid[kQ];
              bool col1[kQ];
#pragma unroll
              for (int i = 0; i < kQ; i++) {
                const int t2 = qd * kQ + i;
                int n, m;
                bool v;
                group_nm(p, t2, &n, &m, &v);
                v = v && t2 <= p + 1;
                const int k = rl_re(n, m);
                ld[i] = v ? __ldcg(&Lb[k]) : 0.0;
                lid[i] = (v && m) ? __ldcg(&Lb[k + 1]) : 0.0;
                col1[i] = t2 < len1;
              }
              TE SR = TE(0), SI = TE(0), SR1 = TE(0), SI1 = TE(0);
#pragma unroll
              for (int i = 0; i < kQ; i++) {
                const TE pr = from_double<TE>(ld[i]) * qq[i], pi = from_double<TE>(lid[i]) * qq[i];
                SR1 += col1[i] ? pr : TE(0);
                SI1 += col1[i] ? pi : TE(0);
                SR += col1[i] ? TE(0) : pr;
                SI += col1[i] ? TE(0) : pi;
              }
              TE acc = (m1 ? TE(2) : TE(1)) * (D1r * SR1 - D1i * SI1) + TE(2) * (D2r * SR - D2i * SI);
              acc = group_sum(acc);
              const TE accn = __shfl_sync(0xffffffffu, acc, 8);
              partial = g.q * to_double(accn - acc);
            }
            // on a step without a move too: decision t then implies that
            // every apply of step t-1 is complete, which the reuse of the
            // step-indexed buffers relies on
            if (idle && !need_state()) {
              fail = true;
              break;
            }
            put(slotE + e, partial);
            if (prof_on && lane == 0) {
              prof_item(rp.prof, 0, t_item);
              prof_item(rp.prof, 10, s_tpub[gi]);
            }
            continue;
          }
          // ---- speculative Alg. L.2 contributions of the proposed move,
          //      column-scaled (the apply multiplies by P_n^m)
          const int dk = it - hD;
          int l = L;
          while (l > S.lmin && dk >= sp_start[l] + ((S.lev_n[l] <= 4) ? 95 : (lev_items[l] + 1) / 2)) l--;
          const int k = dk - sp_start[l];
          const int sh = L - l, nl = S.lev_n[l];
          const int co[3] = {g.cf[0] >> sh, g.cf[1] >> sh, g.cf[2] >> sh};
          const int cn[3] = {g.cfn[0] >> sh, g.cfn[1] >> sh, g.cfn[2] >> sh};
          const int grp = lane >> 3, side = grp & 1;
          if (nl <= 4) {
            // entries 2k, 2k+1 of both lists, added into this step's
            // small-level buffer (image copies make targets repeat)
            const SmallEntry se = small_entry(il, side ? cn : co, nl, pbc, 2 * k + (grp >> 1));
            const TE f = se.valid ? from_double<TE>(side ? g.q : -g.q) : TE(0);
            TE dx = TE(3), dy = TE(3), dz = TE(3);
            if (se.valid) {
              if (sizeof(TE) == 8) {
                dx = (TE)(off[side][l][0] - s_kw[l][se.o[0] + 3]);
                dy = (TE)(off[side][l][1] - s_kw[l][se.o[1] + 3]);
                dz = (TE)(off[side][l][2] - s_kw[l][se.o[2] + 3]);
              } else {
                dx = from_double<TE>(off[side][l][0]) - s_kwe[l][se.o[0] + 3];
                dy = from_double<TE>(off[side][l][1]) - s_kwe[l][se.o[1] + 3];
                dz = from_double<TE>(off[side][l][2]) - s_kwe[l][se.o[2] + 3];
              }
            }
            double* Dt = dsm + (size_t)(S.lev_off[l] + (se.t3[0] * nl + se.t3[1]) * nl + se.t3[2]) * C;
            irregular_group_w<TE>(&tabs, s_iW, p, dx, dy, dz, f, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
              if (se.valid && v) {
                const int kk = rl_re(n, m);
                red_add_f64(&Dt[kk], to_double(vr));
                if (m) red_add_f64(&Dt[kk + 1], to_double(neg_bits(vi)));
              }
            });
          } else {
            // targets 2k (groups 0, 1) and 2k+1 (groups 2, 3); each side in
            // its own slot (the apply adds both)
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
              }
            }
            const TE f = have ? from_double<TE>(side ? g.q : -g.q) : TE(0);
            TE dx = TE(3), dy = TE(3), dz = TE(3);
            if (have) {
              if (sizeof(TE) == 8) {
                dx = (TE)(off[side][l][0] - s_kw[l][ofs[0] + 3]);
                dy = (TE)(off[side][l][1] - s_kw[l][ofs[1] + 3]);
                dz = (TE)(off[side][l][2] - s_kw[l][ofs[2] + 3]);
              } else {
                dx = from_double<TE>(off[side][l][0]) - s_kwe[l][ofs[0] + 3];
                dy = from_double<TE>(off[side][l][1]) - s_kwe[l][ofs[1] + 3];
                dz = from_double<TE>(off[side][l][2]) - s_kwe[l][ofs[2] + 3];
              }
            }
            double* Ds = dslot(l, exists ? kt : 0, side);
            irregular_group_w<TE>(&tabs, s_iW, p, dx, dy, dz, f, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
              if (own && v) {
                const int kk = rl_re(n, m);
                __stcg(&Ds[kk], to_double(vr));
                if (m) __stcg(&Ds[kk + 1], to_double(neg_bits(vi)));
              }
            });
          }
          __syncwarp();
          if (lane == 0) red_release_add(&dcnt[16 * (t & 3)], 1ull);
          if (prof_on && lane == 0) prof_item(rp.prof, nl <= 4 ? 7 : 8, t_item);
        }
      } else if (light) {
        // ------------------------------------------------ light items
        for (int it = lw; it < nLA && !fail; it += nLw) {
          const unsigned long long t_item = prof_on ? mc_globaltimer() : 0ULL;
          if (!reset_next(it) || !sync_prev()) {
            fail = true;
            break;
          }
          // clear the small-level buffer of step t+2 (last used by step t-2,
          // whose contributions and apply preceded the decision of step t-1)
          {
            const size_t zc = (nsC + nLA - 1) / nLA, z0 = (size_t)it * zc;
            const size_t z1 = z0 + zc < nsC ? z0 + zc : nsC;
            for (size_t zi = z0 + lane; zi < z1; zi += 32) __stcg(&dsm_clear[zi], 0.0);
          }
          double partial = 0.0;
          int ptype = 3;
          if (it < iN) {
            // ---- F: far lattice, Sec. 3.4 (iv) in the factored form
            //   dU_inf = sum_k W_k dK_k (H_k + 1/2 (G dK)_k),  W = 1 (m = 0) or 2
            ptype = 2;
            const int f = it;
            const int rb = f / nfc, cb = f % nfc;
            const double c1 = 0.5 * S.a;
            double* st = stage[warp];
            const int k = rb * 32 + lane;
            // dK formed one step ahead holds unless step t-1 or t-2 moved
            // this proposal's particle
            const bool mv1 = t >= 1 && s_acc[(t - 1) & 7] != 0 && !nomove_prev && j_prev == g.j;
            const bool mv2 = t >= 2 && s_acc[(t - 2) & 7] != 0 && !nomove_prev2 && j_prev2 == g.j;
            const bool dk_pre = pbc && t > 0 && !mv1 && !mv2;
            if (!idle) {
              if (dk_pre) {
                if (!counter_wait(ktag, (unsigned long long)t, S.status, rp.wait_ns)) {
                  fail = true;
                  break;
                }
                const double* src = S.dKpre + (size_t)(t & 3) * C;
                for (int kk = lane; kk < C; kk += 32) st[kk] = __ldcg(&src[kk]);
              } else {
                const TE qe = from_double<TE>(g.q);
                const int grp = lane >> 3;
                const double* xg = (grp & 1) ? g.rn : g.r;
                const TE dx = from_double<TE>(xg[0] - c1), dy = from_double<TE>(xg[1] - c1),
                         dz = from_double<TE>(xg[2] - c1);
                regular_group_s<TE>(&tabs, p, dx, dy, dz, qe, [&](int t2, int n, int m, bool v, TE vr, TE vi) {
                  const TE nr = __shfl_xor_sync(0xffffffffu, vr, 8);
                  const TE ni = __shfl_xor_sync(0xffffffffu, vi, 8);
                  if (grp == 0 && v) {
                    const int kk = rl_re(n, m);
                    st[kk] = to_double(nr - vr);
                    if (m) st[kk + 1] = to_double(vi - ni);
                  }
                });
              }
              if (!need_state()) {
                fail = true;
                break;
              }
              const double hk = (cb == 0 && k < C) ? __ldcg(&S.Hhat[k]) : 0.0;
              __syncwarp();
              const int cbeg = cb * csz, cend = min(C, cbeg + csz);
              double contrib = 0.0;
              if (k < C) {
                double gk = 0.0;
                if (gpre && it == lw) {
#pragma unroll
                  for (int i = 0; i < MC_GPRE; i++)
                    if (cbeg + i < cend) gk += gcol[i] * st[cbeg + i];
                } else {
                  for (int c = cbeg; c < cend; c++) gk += __ldcg(&S.G[(size_t)c * C + k]) * st[c];
                }
                S.gK[(size_t)(t & 3) * MC_NF_COLS * C + (size_t)cb * C + k] = gk;
                const double Wk = is_square(k) ? 1.0 : 2.0;
                contrib = Wk * st[k] * (0.5 * gk + hk);
              }
              if (f == 0) {
                for (int kk = lane; kk < C; kk += 32) S.dK[(size_t)(t & 3) * C + kk] = st[kk];
              }
              partial = warp_sum(contrib);
              __syncwarp();
            }
          } else if (it < iX) {
            // ---- N: Alg. 1 over one near cell (27 cells of the extended
            //      domain), part of its slots: near_parts items per cell and
            //      side, or 2 near_parts per cell when both sides share it
            ptype = 1;
            const int k0 = it - iN;
            if (!idle) {
              const NearPart np = near_part(k0, same, nNP, 2 * nNP);
              const int k = np.k, side = np.side, part = np.part, nparts = np.nparts;
              if (!item_near<TE>(S, g, off, k, side, part, nparts, pbc, lane,
                                 [&](int, int, int) {
                                   const bool okw = need_state();
                                   if (okw && prof_on && lane == 0) prof_item(rp.prof, 14, s_tpub[gi]);
                                   return okw;
                                 },
                                 &partial)) {
                fail = true;
                break;
              }
            }
          } else if (it == iX) {
            // ---- X: periodic self-interaction correction (Sec. 3.4, last
            //      item) and the dipole term (tinfoil reading); +inf when r'
            //      left a free-space box
            if (g.outside) {
              partial = kInfA;
            } else if (!nomove && !item_image<TE>(S, g, pbc, lane, need_state, &partial)) {
              fail = true;
              break;
            }
          } else {
            // ---- U: log(u) for the Metropolis test
            if (lane == 0) st_release_f64(&part[MC_MAX_ITEMS - 1], log(s_u[gi]));
          }
          put(it, partial);
          if (prof_on && lane == 0) {
            prof_item(rp.prof, ptype, t_item);
            prof_item(rp.prof, 15, s_tpub[gi]);
          }
        }
        // ------------------------------------------------ apply items
        // (none on a step without a move; the staged contributions' operands
        // are loaded before the decision is known)
        if (!fail && bstart < nB && !idle) {
          bool decided = false, accepted = false;
          for (int b = bstart; b < nB && !fail; b += nLw) {
            const unsigned long long t_item = prof_on ? mc_globaltimer() : 0ULL;
            int ptype = 6;
            const int a = b - 1 - nKH;  // staged-contribution item (a >= 0)
            // operands of a staged-contribution item: this step's
            // contributions complete, every earlier accept applied
            double v[2][8], w[2][8], w1[2][8];
            double* Lt[2] = {nullptr, nullptr};
            bool own[2] = {false, false};
            int lsm = 0;  // large level of the item (0: small level)
            if (a >= 0) {
              if (!counter_wait(&dcnt[16 * (t & 3)], cumD[t & 3], S.status, rp.wait_ns) || !need_state()) {
                fail = true;
                break;
              }
              if (prof_on && lane == 0) prof_item(rp.prof, 12, s_tpub[gi]);
              if (a < S.nsmall) {
                // small-level cell a
                Lt[0] = S.Lhat + (size_t)a * C;
                own[0] = true;
                const double* Dt = dsm + (size_t)a * C;
#pragma unroll
                for (int i = 0; i < 8; i++) {
                  const int kk = lane + 32 * i;
                  v[0][i] = kk < C ? __ldcg(&Lt[0][kk]) : 0.0;
                  w[0][i] = kk < C ? __ldcg(&Dt[kk]) : 0.0;
                  w1[0][i] = 0.0;
                }
              } else {
                // large levels: targets 2c and 2c+1 of level l, both
                // targets' loads in flight together
                int c2 = a - S.nsmall, l = L;
                while (l > S.lmin && c2 >= (lev_items[l] + 1) / 2) {
                  c2 -= (lev_items[l] + 1) / 2;
                  l--;
                }
                lsm = l;
                const int sh = L - l, nl = S.lev_n[l];
                const int co[3] = {g.cf[0] >> sh, g.cf[1] >> sh, g.cf[2] >> sh};
                const int cn[3] = {g.cfn[0] >> sh, g.cfn[1] >> sh, g.cfn[2] >> sh};
                const bool samel = lev_items[l] == 189;
                const double* Ds0[2];
                const double* Ds1[2];
#pragma unroll
                for (int h2 = 0; h2 < 2; h2++) {
                  const int tb = 2 * c2 + h2;
                  const bool ex = tb < lev_items[l];
                  const LargeItem li = large_item(il, co, cn, nl, pbc, samel, ex ? tb : 0);
                  own[h2] = ex && li.owner;
                  Ds0[h2] = dslot(l, ex ? tb : 0, 0);
                  Ds1[h2] = dslot(l, ex ? tb : 0, 1);
                  Lt[h2] = S.Lhat + (size_t)(S.lev_off[l] + (li.tc[0] * nl + li.tc[1]) * nl + li.tc[2]) * C;
                }
#pragma unroll
                for (int h2 = 0; h2 < 2; h2++) {
#pragma unroll
                  for (int i = 0; i < 8; i++) {
                    const int kk = lane + 32 * i;
                    const bool in = own[h2] && kk < C;
                    v[h2][i] = in ? __ldcg(&Lt[h2][kk]) : 0.0;
                    w[h2][i] = in ? __ldcg(&Ds0[h2][kk]) : 0.0;
                    w1[h2][i] = in ? __ldcg(&Ds1[h2][kk]) : 0.0;
                  }
                }
              }
            }
            if (a >= 0) {
              // the accepted values, formed before the decision is known: an
              // accept then only stores them
#pragma unroll
              for (int h2 = 0; h2 < 2; h2++) {
#pragma unroll
                for (int i = 0; i < 8; i++) {
                  const int kk = lane + 32 * i;
                  if (own[h2] && kk < C) v[h2][i] = fma(s_P[kk], w[h2][i] + w1[h2][i], v[h2][i]);
                }
              }
            }
            if (!decided) {
              if (!flag_wait(&s_dstep, t, &s_abort, S.status, rp.wait_ns)) {
                fail = true;
                break;
              }
              if (t >= s_stop) {
                halt = fail = true;
                break;
              }
              decided = true;
              accepted = s_acc[t & 7] != 0;
              if (prof_on && lane == 0) prof_item(rp.prof, 11, s_tpub[gi]);
            }
            if (!accepted) break;  // rejected: nothing to apply
            const double dE_used = s_dEu[t & 7];
            if (b == 0) {
              // ---- bookkeeping: energy, dipole, positions, cell lists
              item_bookkeeping(S, g, off[1][L], dE_used, lane);
            } else if (b <= nKH) {
              // ---- K += dK, H += G dK (sum of the column-block partials)
              item_kh(S, b - 1, nfc, S.gK + (size_t)(t & 3) * MC_NF_COLS * C, S.dK + (size_t)(t & 3) * C, lane);
            } else {
              // L += P (sum of the contributions), formed above
              ptype = lsm ? 5 : 4;
#pragma unroll
              for (int h2 = 0; h2 < 2; h2++) {
#pragma unroll
                for (int i = 0; i < 8; i++) {
                  const int kk = lane + 32 * i;
                  if (own[h2] && kk < C) __stcg(&Lt[h2][kk], v[h2][i]);
                }
              }
            }
            __syncwarp();
            if (lane == 0) red_release_add(S.bar, 1ull);
            if (prof_on && lane == 0) {
              prof_item(rp.prof, ptype, t_item);
              prof_item(rp.prof, 13, s_tpub[gi]);
            }
          }
        }
      }
      if (fail) {
        if (!halt) s_abort = 1;
        break;
      }
      j_prev2 = j_prev;
      nomove_prev2 = nomove_prev;
      j_prev = g.j;
      nomove_prev = nomove;
      if (lane == 0) flag_publish(&s_wdone[warp], t);
      __syncwarp();
    }
  }
  __syncthreads();
  if (cta == 0 && threadIdx.x == 0) {
    S.stats[0] = s_stats[0];
    S.stats[1] = s_stats[1];
    S.stats[2] = s_stats[2];
    S.stats[3] = (long long)(mc_globaltimer() - t_begin);  // this launch's wall time, ns
  }
}

template <typename TE>
__global__ void __launch_bounds__(MC_THREADS, 1) mc_async_kernel(const McSys* __restrict__ sysp, RunParams rp) {
  async_body<TE>(sysp, rp, (int)gridDim.x, (int)blockIdx.x);
}

template __global__ void mc_async_kernel<double>(const McSys*, RunParams);
template __global__ void mc_async_kernel<float>(const McSys*, RunParams);

cudaError_t mc_launch_async(const McSys* d_sys, const RunParams& rp, int prec, int nCTA, cudaStream_t stream) {
  void* args[] = {(void*)&d_sys, (void*)&rp};
  const void* fn = prec ? (const void*)mc_async_kernel<float> : (const void*)mc_async_kernel<double>;
  return cudaLaunchCooperativeKernel(fn, dim3(nCTA), dim3(MC_THREADS), args, 0, stream);
}
