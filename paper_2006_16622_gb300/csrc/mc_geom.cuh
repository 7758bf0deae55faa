// Octree geometry of the interaction lists (Sec. 3.1) and of the Alg. L.2
// targets: the per-parity offset table, list membership, the offset of a
// target from a list centre with periodic images, and the target cells and
// owners of the accept contributions on small and large levels.  Integer
// code only (CUDA thread index for the table fill), so it also compiles for
// host tests.
#pragma once

// Interaction-list offsets (Sec. 3.1) for the 8 parity classes of a cell:
// children of the parent's 27 neighbours span [-2-b, 3-b] per axis (b the
// cell's parity on that axis); the 27 near offsets are removed.  Built per
// CTA in shared memory: il[parity][k] = packed (ox+4) | (oy+4)<<4 | (oz+4)<<8.
__device__ __forceinline__ void il_table_init(unsigned short (*il)[189]) {
  for (int t = threadIdx.x; t < 8 * 216; t += blockDim.x) {
    const int par = t / 216, b = t % 216;
    const int bx = (par >> 2) & 1, by = (par >> 1) & 1, bz = par & 1;
    const int i = b / 36, jj = (b / 6) % 6, l = b % 6;
    const int ox = i - 2 - bx, oy = jj - 2 - by, oz = l - 2 - bz;
    const bool inner = (ox >= -1 && ox <= 1 && oy >= -1 && oy <= 1 && oz >= -1 && oz <= 1);
    if (inner) continue;
    // rank of b among the non-inner entries of this parity class
    int k = 0;
    for (int bb = 0; bb < b; bb++) {
      const int ii = bb / 36, j2 = (bb / 6) % 6, l2 = bb % 6;
      const int px = ii - 2 - bx, py = j2 - 2 - by, pz = l2 - 2 - bz;
      if (!(px >= -1 && px <= 1 && py >= -1 && py <= 1 && pz >= -1 && pz <= 1)) k++;
    }
    il[par][k] = (unsigned short)((ox + 4) | ((oy + 4) << 4) | ((oz + 4) << 8));
  }
}
__device__ __forceinline__ void il_unpack(unsigned short v, int* ox, int* oy, int* oz) {
  *ox = (int)(v & 15) - 4;
  *oy = (int)((v >> 4) & 15) - 4;
  *oz = (int)((v >> 8) & 15) - 4;
}

__device__ __forceinline__ int mc_wrap_coord(int e, int n) { return ((e % n) + n) % n; }

__device__ __forceinline__ bool in_il(int ox, int oy, int oz, int cx, int cy, int cz) {
  const int bx = cx & 1, by = cy & 1, bz = cz & 1;
  if (ox < -2 - bx || ox > 3 - bx || oy < -2 - by || oy > 3 - by || oz < -2 - bz || oz > 3 - bz)
    return false;
  return (ox < -1 || ox > 1 || oy < -1 || oy > 1 || oz < -1 || oz > 1);
}

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

// Near-field items of a step (Alg. 1 split over several items per near
// cell): item k0 takes near cell k (0..26) of the side `side` (0: r, 1: r',
// 2: both, when r and r' share their finest cell) and the slot blocks part,
// part + nparts, ... (32 slots each) of that cell.  With different cells the
// 54 nparts items are (cell, side) x nparts; with a shared cell the first
// 27 nsame items are cell x nsame (items beyond get k = -1, no work).
struct NearPart {
  int k, side, part, nparts;
};

__device__ __forceinline__ NearPart near_part(int k0, bool same, int nparts, int nsame) {
  NearPart r;
  if (same) {
    r.k = k0 % 27;
    r.side = 2;
    r.part = k0 / 27;
    r.nparts = nsame;
    if (r.part >= nsame) r.k = -1;
  } else {
    const int kb = k0 % 54;
    r.k = kb % 27;
    r.side = kb / 27;
    r.part = k0 / 54;
    r.nparts = nparts;
  }
  return r;
}
