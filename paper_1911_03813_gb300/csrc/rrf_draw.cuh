// The Gaussian test matrix of eq. rrf, drawn where it is used (never stored).
#pragma once

#include <cstdint>

namespace stmf {

// Philox4x32-10 (Salmon et al., SC 2011) and a Box-Muller normal: entry (l, j) of the test matrix
// of eq. rrf uses counter (l mod 2^32, l div 2^32, j, 0) and key (seed mod 2^32, seed div 2^32);
// words x0, x1 give u_k = (x_k + 1/2) 2^-32 and omega = sqrt(-2 ln u1) cos(2 pi u2).
__device__ __forceinline__ void rrf_philox(int64_t l, int j, uint64_t seed, uint32_t& x0,
                                           uint32_t& x1) {
  uint32_t c0 = (uint32_t)(uint64_t)l, c1 = (uint32_t)((uint64_t)l >> 32), c2 = (uint32_t)j, c3 = 0;
  uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, c0), lo0 = 0xD2511F53u * c0;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, c2), lo1 = 0xCD9E8D57u * c2;
    const uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
  }
  x0 = c0;
  x1 = c1;
}

__device__ __forceinline__ double rrf_omega(int64_t l, int j, uint64_t seed) {
  uint32_t x0, x1;
  rrf_philox(l, j, seed, x0, x1);
  const double u1 = ((double)x0 + 0.5) * 0x1p-32;
  const double u2 = ((double)x1 + 0.5) * 0x1p-32;
  return sqrt(-2.0 * log(u1)) * cos(6.283185307179586 * u2);
}

// The same draw with u_k and the normal in FP32 (the range finder for reduced-precision samples,
// whose products and sums are FP32 too): cos(2 pi u2) as cospi(2 u2). Within a few FP32 ulps of
// the FP64 draw; A0 is a random start, so that rounding does not matter to the method.
__device__ __forceinline__ float rrf_omega_f32(int64_t l, int j, uint64_t seed) {
  uint32_t x0, x1;
  rrf_philox(l, j, seed, x0, x1);
  const float u1 = fmaf(__uint2float_rn(x0), 0x1p-32f, 0x1p-33f);
  const float u2 = fmaf(__uint2float_rn(x1), 0x1p-32f, 0x1p-33f);
  return sqrtf(-2.f * logf(u1)) * cospif(2.f * u2);
}

}  // namespace stmf
