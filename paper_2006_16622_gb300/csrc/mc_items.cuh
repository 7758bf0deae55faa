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

// Offset of target cell tc from list centre c on a level with nl >= 8 cells
// per axis: with periodic images the one image of the target within
// [-nl/2, nl/2) per axis (an interaction-list offset lies in [-3, 3], so no
// other image can be in the list).
__device__ __forceinline__ void list_offset(const int* tc, const int* c, int nl, bool pbc, int* o) {
#pragma unroll
  for (int d = 0; d < 3; d++) {
    int v = tc[d] - c[d];
    if (pbc) {
      if (v >= nl / 2) v -= nl;
      if (v < -nl / 2) v += nl;
    }
    o[d] = v;
  }
}

// Target cell of large-level accept item k and whether the item owns it:
// the interaction list of alpha' (items k < 189, or every item when alpha =
// alpha' on this level) owns its targets; an item of the alpha list
// (k >= 189) owns its target unless the target is also in IL(alpha').
struct LargeItem {
  int tc[3];
  int ofs[3];  // offset of the target from the centre of the item's own list
  bool owner, from_new;
};

__device__ __forceinline__ LargeItem large_item(const unsigned short (*il)[189], const int* co,
                                                const int* cn, int nl, bool pbc, bool samel,
                                                int k) {
  LargeItem it;
  it.owner = true;
  it.from_new = samel || (k < 189);
  const int kk = (k < 189) ? k : k - 189;
  const int* base = it.from_new ? cn : co;
  const int par = ((base[0] & 1) << 2) | ((base[1] & 1) << 1) | (base[2] & 1);
  int ox, oy, oz;
  il_unpack(il[par][kk], &ox, &oy, &oz);
  it.ofs[0] = ox;
  it.ofs[1] = oy;
  it.ofs[2] = oz;
  const int e[3] = {base[0] + ox, base[1] + oy, base[2] + oz};
  if (!pbc && (e[0] < 0 || e[0] >= nl || e[1] < 0 || e[1] >= nl || e[2] < 0 || e[2] >= nl))
    it.owner = false;
  for (int d = 0; d < 3; d++) it.tc[d] = mc_wrap_coord(e[d], nl);
  if (it.owner && !it.from_new) {
    int o[3];
    list_offset(it.tc, cn, nl, pbc, o);
    if (in_il(o[0], o[1], o[2], cn[0], cn[1], cn[2])) it.owner = false;
  }
  return it;
}

// Small-level accept entry (levels with <= 4 cells per axis): entry `entry`
// of IL(alpha) (side 0) or IL(alpha') (side 1); image copies make targets
// repeat across entries, so updates of these levels are atomic adds.
struct SmallEntry {
  int t3[3];
  int o[3];
  bool valid;
};

__device__ __forceinline__ SmallEntry small_entry(const unsigned short (*il)[189], const int* cs,
                                                  int nl, bool pbc, int entry) {
  SmallEntry se;
  const int par = ((cs[0] & 1) << 2) | ((cs[1] & 1) << 1) | (cs[2] & 1);
  int ox = 0, oy = 0, oz = 0;
  if (entry < 189) il_unpack(il[par][entry], &ox, &oy, &oz);
  se.o[0] = ox;
  se.o[1] = oy;
  se.o[2] = oz;
  const int e[3] = {cs[0] + ox, cs[1] + oy, cs[2] + oz};
  se.valid = entry < 189 && (pbc || (e[0] >= 0 && e[0] < nl && e[1] >= 0 && e[1] < nl &&
                                     e[2] >= 0 && e[2] < nl));
  for (int d = 0; d < 3; d++) se.t3[d] = mc_wrap_coord(e[d], nl);
  return se;
}

