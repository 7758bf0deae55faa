// One group of 8 lanes computes one set of column-scaled irregular solid
// harmonics in pair-of-floats arithmetic (mc_df64.cuh); the FP64 form of the
// same group (irregular_group_w, harm_group) lives in mc_dev.cuh.  Depends
// only on the pair helpers, threadIdx.x and the warp shuffles.
#pragma once
#include "mc_df64.cuh"

// irregular_group_w in pair-of-floats arithmetic (mc_df64.cuh, FP32 pipe,
// ~46 significant bits): the displacement comes in units of 2^k, so value
// (n, m) comes out multiplied by 2^(k (n + 1)) (the harmonics are
// homogeneous of degree -(n + 1)); with |x| near 1 every value and its low
// part stay inside the normal float range.  A2[k] = A_k, the diagonal
// factors of the irregular tables; W2 the W table of irregular_w_tabs.
template <typename F>
__device__ __forceinline__ void irregular_group_w2(const f2* A2, const f2 (*W2)[16], int p, f2 x, f2 y,
                                                   f2 z, f2 s, F&& use) {
  const f2 zero = {0.0f, 0.0f};
  const f2 r2 = f2_add(f2_mul_add(x, x, y, y), f2_mul(z, z));
  const f2 ir = f2_rsqrt(r2);
  const f2 Q = f2_mul(ir, ir);
  const f2 X = f2_mul(x, Q), Y = f2_mul(y, Q), Z = f2_mul(z, Q);
  const f2 start = f2_mul(ir, s);
  const int g = threadIdx.x & 7;
  const int k0 = 2 * g, k1 = 2 * g + 1;
  const f2 a0 = A2[k0], a1 = A2[k1];
  const f2 f0r = (k0 == 0) ? start : f2_mul(X, a0), f0i = (k0 == 0) ? zero : f2_mul(Y, a0);
  const f2 f1r = f2_mul(X, a1), f1i = f2_mul(Y, a1);
  // inclusive product scan of f_{2g} f_{2g+1} over the 8 lanes of the group
  f2 Ir = f2_mul_sub(f0r, f1r, f0i, f1i), Ii = f2_mul_add(f0r, f1i, f0i, f1r);
#pragma unroll
  for (int d = 1; d < 8; d <<= 1) {
    const f2 ur = f2_shfl_up(Ir, d, 8), ui = f2_shfl_up(Ii, d, 8);
    if (g >= d) {
      const f2 nr = f2_mul_sub(ur, Ir, ui, Ii), ni = f2_mul_add(ur, Ii, ui, Ir);
      Ir = nr;
      Ii = ni;
    }
  }
  f2 Er = f2_shfl_up(Ir, 1, 8), Ei = f2_shfl_up(Ii, 1, 8);
  if (g == 0) {
    Er = f2_make(1.0f);
    Ei = zero;
  }
  const f2 D0r = f2_mul_sub(Er, f0r, Ei, f0i), D0i = f2_mul_add(Er, f0i, Ei, f0r);  // X_{2g}^{2g}
  const f2 D1r = Ir, D1i = Ii;                                                       // X_{2g+1}^{2g+1}
  const int m1 = g, m2 = p - g;
  const bool active = m1 <= m2;
  const bool two = m2 > m1;
  const f2 e1r = f2_shfl(D0r, m1 >> 1, 8), e1i = f2_shfl(D0i, m1 >> 1, 8);
  const f2 o1r = f2_shfl(D1r, m1 >> 1, 8), o1i = f2_shfl(D1i, m1 >> 1, 8);
  const int m2c = (m2 >= 0 && m2 <= 15) ? m2 : 0;
  const f2 e2r = f2_shfl(D0r, m2c >> 1, 8), e2i = f2_shfl(D0i, m2c >> 1, 8);
  const f2 o2r = f2_shfl(D1r, m2c >> 1, 8), o2i = f2_shfl(D1i, m2c >> 1, 8);
  const f2 d1r = f2_sel(m1 & 1, o1r, e1r), d1i = f2_sel(m1 & 1, o1i, e1i);
  const f2 d2r = f2_sel(m2c & 1, o2r, e2r), d2i = f2_sel(m2c & 1, o2i, e2i);
  const int len1 = p - m1 + 1;
  f2 p1r = zero, p1i = zero, p2r = zero, p2i = zero;
#pragma unroll 1
  for (int t = 0; t <= p + 1; t++) {
    const bool c1 = t < len1;
    const int m = c1 ? m1 : m2c;
    const int n = c1 ? (m1 + t) : (m2c + t - len1);
    const bool valid = active && (c1 || two) && n <= p;
    const bool st = (n == m);
    const int nn = n > 15 ? 15 : n;
    const f2 b = f2_mul(Q, W2[nn][m]);
    f2 vr = f2_mul_sub(Z, p1r, b, p2r), vi = f2_mul_sub(Z, p1i, b, p2i);
    vr = f2_sel(st, c1 ? d1r : d2r, vr);
    vi = f2_sel(st, c1 ? d1i : d2i, vi);
    p2r = f2_sel(st, zero, p1r);
    p2i = f2_sel(st, zero, p1i);
    p1r = vr;
    p1i = vi;
    use(t, n, m, valid, vr, vi);
  }
}
