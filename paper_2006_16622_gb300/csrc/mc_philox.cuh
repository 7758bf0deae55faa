// The proposal stream: Philox4x32-10 and the step's draws (particle,
// displacement, acceptance uniform).  Needs only <stdint.h> and CUDA's
// integer and round-to-nearest intrinsics, so it also compiles for host
// tests.
#pragma once
#include <stdint.h>

// ------------------------------------------------------------ Philox4x32-10
// Salmon et al. (SC'11): two 32x32 multiplies per round, Weyl key bumps.
__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; r++) {
    if (r) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    uint32_t lo0 = 0xD2511F53u * c[0], hi0 = __umulhi(0xD2511F53u, c[0]);
    uint32_t lo1 = 0xCD9E8D57u * c[2], hi1 = __umulhi(0xCD9E8D57u, c[2]);
    uint32_t n0 = hi1 ^ c[1] ^ k0, n2 = hi0 ^ c[3] ^ k1;
    c[0] = n0;
    c[1] = lo1;
    c[2] = n2;
    c[3] = lo0;
  }
}

// Proposal of global step s: j = floor(A0 n / 2^32); delta_k = h (2u_k - 1),
// u_k = (A_k + 1/2) 2^-32; acceptance uniform ((B0>>5) 2^26 + (B1>>6)) 2^-53.
// Written with explicit round-to-nearest intrinsics so that no contraction
// changes the bits of the displacement.
__device__ __forceinline__ void mc_proposal(unsigned long long seed, unsigned long long s,
                                            uint32_t chain, int n, double h, int* j,
                                            double d[3], double* u) {
  uint32_t A[4] = {(uint32_t)s, (uint32_t)(s >> 32), chain, 0u};
  uint32_t B[4] = {(uint32_t)s, (uint32_t)(s >> 32), chain, 1u};
  philox4x32_10(A, (uint32_t)seed, (uint32_t)(seed >> 32));
  philox4x32_10(B, (uint32_t)seed, (uint32_t)(seed >> 32));
  *j = (int)(((unsigned long long)A[0] * (unsigned long long)n) >> 32);
#pragma unroll
  for (int k = 0; k < 3; k++) {
    double uk = __dmul_rn(__dadd_rn((double)A[k + 1], 0.5), 2.3283064365386963e-10);
    d[k] = __dmul_rn(h, __dsub_rn(__dmul_rn(2.0, uk), 1.0));
  }
  *u = __dmul_rn(__dadd_rn(__dmul_rn((double)(B[0] >> 5), 67108864.0), (double)(B[1] >> 6)),
                 1.1102230246251565e-16);
}

// One axis of the proposal: every lane runs both Philox blocks (integer
// work), the FP64 arithmetic of the displacement is per axis, u only where
// requested.
__device__ __forceinline__ void mc_proposal_axis(unsigned long long seed, unsigned long long s,
                                                 uint32_t chain, int n, double h, int axis, int* j,
                                                 double* d, double* u) {
  uint32_t A[4] = {(uint32_t)s, (uint32_t)(s >> 32), chain, 0u};
  uint32_t B[4] = {(uint32_t)s, (uint32_t)(s >> 32), chain, 1u};
  philox4x32_10(A, (uint32_t)seed, (uint32_t)(seed >> 32));
  philox4x32_10(B, (uint32_t)seed, (uint32_t)(seed >> 32));
  *j = (int)(((unsigned long long)A[0] * (unsigned long long)n) >> 32);
  const uint32_t w = axis == 0 ? A[1] : (axis == 1 ? A[2] : A[3]);
  const double uk = __dmul_rn(__dadd_rn((double)w, 0.5), 2.3283064365386963e-10);
  *d = __dmul_rn(h, __dsub_rn(__dmul_rn(2.0, uk), 1.0));
  if (u)
    *u = __dmul_rn(__dadd_rn(__dmul_rn((double)(B[0] >> 5), 67108864.0), (double)(B[1] >> 6)),
                   1.1102230246251565e-16);
}
