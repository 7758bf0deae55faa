// Work-item building blocks shared by the chain kernels (mc_chain.cu and
// mc_async.cu): the proposal geometry, item timers, and the target cells of
// the Alg. L.2 contributions on small and large levels.
#pragma once
#include "mc_dev.cuh"

namespace {

constexpr double kImageConst = 6.0 + 8.0 / 1.7320508075688772 + 12.0 / 1.4142135623730951;
constexpr double kPi = 3.141592653589793;

struct StepGeo {
  int j;
  double q;
  double r[3], rn[3];
  int cf[3], cfn[3];
  bool outside;  // free space: r' left the box
};

// Optional timers (RunParams.prof, 56 counters, globaltimer ns):
//   [0..4] CTA 0 thread 0: own propose items, barrier-1 wait, decision,
//          own accept items, barrier-2 wait; [5] steps, [6] accepted steps;
//   [8+t] summed duration, [24+t] count, [40+t] max duration of items of
//   type t: 0 E, 1 N, 2 F, 3 X/U, 4 small-level accept (or apply),
//   5 target accept (or apply), 6 bookkeeping and K/H, 7 speculative
//   small-level contribution, 8 speculative large-level contribution.
__device__ __forceinline__ void prof_item(unsigned long long* prof, int type,
                                          unsigned long long t0) {
  const unsigned long long d = mc_globaltimer() - t0;
  atomicAdd(&prof[8 + type], d);
  atomicAdd(&prof[24 + type], 1ULL);
  atomicMax(&prof[40 + type], d);
}

__device__ __forceinline__ bool is_square(int k) {
  int s = (int)sqrtf((float)k + 0.5f);
  return s * s == k;
}

constexpr double kInf = __builtin_huge_val();

}  // namespace



// ----------------------------------------------------------- shared items
// Work items that both chain kernels run unchanged; each is executed by one
// whole warp.  `wait` callbacks order the item's reads of state that the
// accepts write (each kernel has its own mechanism) and return false when
// the wait gave up (the item then stops and returns false).

// Alg. 1 over one near cell: the neighbour at offset k (0..26) of the
// finest cell of r (side 0), of r' (side 1), or of both (side 2, same
// cell): the Coulomb (and Lennard-Jones) change of the moving charge with
// the cell's charges; +inf when r' falls on a charge.  The item takes the
// slot blocks part, part + nparts, ... (32 slots each) of the cell, so
// nparts items together cover it.  wait(c0, c1, c2) is called with the
// (wrapped) cell before its list is read.
template <typename TE, typename Wait>
__device__ __forceinline__ bool item_near(const McSys& S, const StepGeo& g,
                                          const double (*off)[MC_MAXLEV + 2][3], int k, int side,
                                          int part, int nparts, bool pbc, int lane, Wait&& wait,
                                          double* partial_out) {
  const int L = S.L;
  const int* cc = (side == 1) ? g.cfn : g.cf;
  const int d0 = k / 9 - 1, d1 = (k / 3) % 3 - 1, d2 = k % 3 - 1;
  const int e0 = cc[0] + d0, e1 = cc[1] + d1, e2 = cc[2] + d2;
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
  if (!wait(c0, c1, c2)) return false;
  double partial = 0.0;
  if (valid) {
    const int cell = (c0 * nL + c1) * nL + c2;
    const int cnt = __ldcg(&S.ccount[cell]);
    const bool zero_shift = (s0 == 0 && s1 == 0 && s2 == 0);
    bool ovl = false;
    const bool lj = S.lj_on != 0;
    if (sizeof(TE) == 8) {
      // query points moved by minus the image shift
      const double sx = s0 * S.a, sy = s1 * S.a, sz = s2 * S.a;
      const double ox = g.r[0] - sx, oy = g.r[1] - sy, oz = g.r[2] - sz;
      const double nx = g.rn[0] - sx, ny = g.rn[1] - sy, nz = g.rn[2] - sz;
      double acc = 0.0;
      for (int s = 32 * part + lane; s < cnt; s += 32 * nparts) {
        const double4 xi = ldcg4(&S.cpos[(size_t)cell * S.cap + s]);
        const int pid = (side != 1 || lj) ? __ldcg(&S.cpid[(size_t)cell * S.cap + s]) : -1;
        if (side != 1) {
          if (!(pid == g.j && zero_shift)) {
            const double ax = ox - xi.x, ay = oy - xi.y, az = oz - xi.z;
            const double d2 = ax * ax + ay * ay + az * az;
            const double ir = rsqrt(d2);
            acc -= g.q * xi.w * ir;
            if (lj && pid != g.j) acc -= lj_energy(ir * ir, d2, S.lj_eps4, S.lj_s6, S.lj_s12, S.lj_rc2);
          }
        }
        if (side != 0) {
          const double bx = nx - xi.x, by = ny - xi.y, bz = nz - xi.z;
          const double d2 = bx * bx + by * by + bz * bz;
          if (d2 == 0.0) ovl = true;
          const double ir = rsqrt(d2);
          acc += g.q * xi.w * ir;
          // the moving particle's old copy (and its images, beyond the
          // cutoff) has no Lennard-Jones term
          if (lj && pid != g.j) acc += lj_energy(ir * ir, d2, S.lj_eps4, S.lj_s6, S.lj_s12, S.lj_rc2);
        }
      }
      partial = warp_sum(acc);
    } else {
      // FP32: slot positions are stored relative to their cell centre; the
      // query points relative to this (image) cell's centre follow from
      // their finest-cell offsets and the integer cell offset
      const int oo0 = e0 - g.cf[0], oo1 = e1 - g.cf[1], oo2 = e2 - g.cf[2];
      const int on0 = e0 - g.cfn[0], on1 = e1 - g.cfn[1], on2 = e2 - g.cfn[2];
      const double wL = S.lev_w[L];
      const float ox = d2f_int(off[0][L][0] - oo0 * wL), oy = d2f_int(off[0][L][1] - oo1 * wL),
                  oz = d2f_int(off[0][L][2] - oo2 * wL);
      const float nx = d2f_int(off[1][L][0] - on0 * wL), ny = d2f_int(off[1][L][1] - on1 * wL),
                  nz = d2f_int(off[1][L][2] - on2 * wL);
      float acc = 0.0f;
      const float qf = d2f_int(g.q);
      const float e4 = d2f_int(S.lj_eps4), s6 = d2f_int(S.lj_s6), s12 = d2f_int(S.lj_s12),
                  rc2 = d2f_int(S.lj_rc2);
      // close pairs: the FP32 cell-relative coordinates carry an absolute
      // error of ~1e-7 w (w the finest cell width), which a pair at distance
      // d turns into ~1e-7 w / d^2 of energy; pairs closer than w/8 are
      // therefore summed in FP64 from the absolute positions (rare: ~0.4 per
      // step at 24 charges per cell), which bounds the FP32 pair error by
      // ~1e-5 w^-1, and an exact overlap is decided in FP64 as in the FP64 form
      const float close2 = d2f_int(wL * wL * (1.0 / 64.0));
      double acc64 = 0.0;
      bool any_close = false;
      for (int s = 32 * part + lane; s < cnt; s += 32 * nparts) {
        const float4 xi = __ldcg(&S.cpos32[(size_t)cell * S.cap + s]);
        const int pid = (side != 1 || lj) ? __ldcg(&S.cpid[(size_t)cell * S.cap + s]) : -1;
        bool close_o = false, close_n = false;
        if (side != 1) {
          if (!(pid == g.j && zero_shift)) {
            const float ax = ox - xi.x, ay = oy - xi.y, az = oz - xi.z;
            const float d2 = ax * ax + ay * ay + az * az;
            if (d2 < close2) {
              close_o = true;
            } else {
              const float ir = rsqrtf(d2);
              acc -= qf * xi.w * ir;
              if (lj && pid != g.j) acc -= lj_energy(ir * ir, d2, e4, s6, s12, rc2);
            }
          }
        }
        if (side != 0) {
          const float bx = nx - xi.x, by = ny - xi.y, bz = nz - xi.z;
          const float d2 = bx * bx + by * by + bz * bz;
          if (d2 < close2) {
            close_n = true;
          } else {
            const float ir = rsqrtf(d2);
            acc += qf * xi.w * ir;
            if (lj && pid != g.j) acc += lj_energy(ir * ir, d2, e4, s6, s12, rc2);
          }
        }
        if (close_o || close_n) {
          any_close = true;
          const double4 x64 = ldcg4(&S.cpos[(size_t)cell * S.cap + s]);
          const double sx = s0 * S.a, sy = s1 * S.a, sz = s2 * S.a;
          if (close_o) {
            const double ax = (g.r[0] - sx) - x64.x, ay = (g.r[1] - sy) - x64.y, az = (g.r[2] - sz) - x64.z;
            const double d2 = ax * ax + ay * ay + az * az;
            const double ir = rsqrt(d2);
            acc64 -= g.q * x64.w * ir;
            if (lj && pid != g.j) acc64 -= lj_energy(ir * ir, d2, S.lj_eps4, S.lj_s6, S.lj_s12, S.lj_rc2);
          }
          if (close_n) {
            const double bx = (g.rn[0] - sx) - x64.x, by = (g.rn[1] - sy) - x64.y, bz = (g.rn[2] - sz) - x64.z;
            const double d2 = bx * bx + by * by + bz * bz;
            if (d2 == 0.0) ovl = true;
            const double ir = rsqrt(d2);
            acc64 += g.q * x64.w * ir;
            if (lj && pid != g.j) acc64 += lj_energy(ir * ir, d2, S.lj_eps4, S.lj_s6, S.lj_s12, S.lj_rc2);
          }
        }
      }
      partial = f2d_int(warp_sum(acc));
      if (__any_sync(0xffffffffu, any_close)) partial += warp_sum(acc64);
    }
    if (__any_sync(0xffffffffu, ovl)) partial = kInf;
  }
  *partial_out = partial;
  return true;
}

// Periodic self-interaction correction (Sec. 3.4, last item: the moving
// charge's images) and, with tinfoil boundary conditions, the dipole term;
// free space: the charge's interaction with its old position.  wait() is
// called before the dipole sum is read.
template <typename TE, typename Wait>
__device__ __forceinline__ bool item_image(const McSys& S, const StepGeo& g, bool pbc, int lane,
                                           Wait&& wait, double* partial_out) {
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
  double partial = to_double(warp_sum(v));
  if (pbc) {
    partial += g.q * g.q / S.a * kImageConst;
    if (S.dip == 0) {
      if (!wait()) return false;
      const double cdip = -2.0 * kPi / (3.0 * S.V);
      double D2 = 0.0, Dn2 = 0.0;
#pragma unroll
      for (int kk = 0; kk < 3; kk++) {
        const double D = __ldcg(&S.dipv[kk]);
        const double Dn = D + g.q * (g.rn[kk] - g.r[kk]);
        D2 += D * D;
        Dn2 += Dn * Dn;
      }
      partial += cdip * Dn2 - cdip * D2;
    }
  }
  *partial_out = partial;
  return true;
}

// dK of the proposal of step s (drawn and moved exactly as the proposal code
// of that step does), from the particle position as loaded now, into dst
// (C doubles): dK = q (conj Rt(r' - R1) - conj Rt(r - R1)), R1 the box centre.
template <typename TE>
__device__ __forceinline__ void item_dk(const McSys& S, const HarmTabs<TE>* tabs, const RunParams& rp,
                                        long long s, int lane, double* dst) {
  int jn;
  double dn = 0.0;
  mc_proposal_axis(rp.seed, (unsigned long long)(rp.step0 + s), rp.chain, S.n, rp.h, lane < 3 ? lane : 0,
                   &jn, &dn, nullptr);
  const double4 pj = ldcg4(&S.ppos[jn]);
  double x0 = 0.0, x1 = 0.0;
  if (lane < 3) {
    x0 = lane == 0 ? pj.x : (lane == 1 ? pj.y : pj.z);
    double x = __dadd_rn(x0, dn);
    if (x < 0.0) x = __dadd_rn(x, S.a);
    if (x >= S.a) x = __dsub_rn(x, S.a);
    x1 = x;
  }
  const int grp = lane >> 3, side = grp & 1;
  const double c1 = 0.5 * S.a;
  double xs[3];
#pragma unroll
  for (int ax = 0; ax < 3; ax++) {
    const double a0 = __shfl_sync(0xffffffffu, x0, ax), a1 = __shfl_sync(0xffffffffu, x1, ax);
    xs[ax] = side ? a1 : a0;
  }
  const TE dx = from_double<TE>(xs[0] - c1), dy = from_double<TE>(xs[1] - c1), dz = from_double<TE>(xs[2] - c1);
  regular_group_s<TE>(tabs, S.p, dx, dy, dz, from_double<TE>(pj.w), [&](int t2, int n, int m, bool v, TE vr, TE vi) {
    const TE nr = __shfl_xor_sync(0xffffffffu, vr, 8);
    const TE ni = __shfl_xor_sync(0xffffffffu, vi, 8);
    if (grp == 0 && v) {
      const int kk = rl_re(n, m);
      __stcg(&dst[kk], to_double(nr - vr));
      if (m) __stcg(&dst[kk + 1], to_double(vi - ni));
    }
  });
}

// Accept bookkeeping of a move: cell lists (slot moved within or between
// finest cells), position, running energy, dipole sum; off_new = offset of
// r' from the centre of its finest cell (the FP32 slot record).
__device__ __forceinline__ void item_bookkeeping(const McSys& S, const StepGeo& g, const double* off_new,
                                                 double dE_used, int lane) {
  const int nL = S.nL, cap = S.cap;
  const int co = (g.cf[0] * nL + g.cf[1]) * nL + g.cf[2];
  const int cn = (g.cfn[0] * nL + g.cfn[1]) * nL + g.cfn[2];
  // the loads the move needs, issued together by lanes 0..2
  int so = 0, cnt_o = 0, cnt_n = 0;
  if (lane == 0) so = S.pslot[g.j];
  if (lane == 1) cnt_o = S.ccount[co];
  if (lane == 2) cnt_n = S.ccount[cn];
  so = __shfl_sync(0xffffffffu, so, 0);
  cnt_o = __shfl_sync(0xffffffffu, cnt_o, 1);
  cnt_n = __shfl_sync(0xffffffffu, cnt_n, 2);
  const double4 np = make_double4(g.rn[0], g.rn[1], g.rn[2], g.q);
  const float4 rel = make_float4(d2f_int(off_new[0]), d2f_int(off_new[1]), d2f_int(off_new[2]), d2f_int(g.q));
  if (co == cn) {
    if (lane == 0) S.cpos[so] = np;
    if (lane == 1) S.cpos32[so] = rel;
  } else {
    const int last = cnt_o - 1;
    const int sl = co * cap + last;
    if (so != sl) {
      // move the cell's last slot into the freed one
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
      if (lane == 2) S.cpid[slot] = g.j;
      if (lane == 4) S.pslot[g.j] = slot;
      if (lane == 5) S.ccount[cn] = cnt_n + 1;
    }
  }
  if (lane == 6) S.ppos[g.j] = np;
  if (lane == 7) S.energy[0] += dE_used;
  if (lane >= 8 && lane < 11) S.dipv[lane - 8] += g.q * (g.rn[lane - 8] - g.r[lane - 8]);
}

// K += dK, H += G dK for 32 entries (block b, 0-based): the sum of the
// column-block partials gK (nfc blocks of C) and dK of the accepted move.
__device__ __forceinline__ void item_kh(const McSys& S, int b, int nfc, const double* gK, const double* dK,
                                        int lane) {
  const int C = S.C;
  const int k = b * 32 + lane;
  if (k < C) {
    double gv[MC_NF_COLS];
#pragma unroll
    for (int cb = 0; cb < MC_NF_COLS; cb++) gv[cb] = cb < nfc ? __ldcg(&gK[(size_t)cb * C + k]) : 0.0;
    const double dk = __ldcg(&dK[k]);
    const double kh = __ldcg(&S.Khat[k]), hh = __ldcg(&S.Hhat[k]);
    double gs = 0.0;
#pragma unroll
    for (int cb = 0; cb < MC_NF_COLS; cb++)
      if (cb < nfc) gs += gv[cb];
    __stcg(&S.Khat[k], kh + dk);
    __stcg(&S.Hhat[k], hh + gs);
  }
}
