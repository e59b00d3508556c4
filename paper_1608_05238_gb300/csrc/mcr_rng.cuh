// mcr_rng.cuh -- the counter-based random numbers of the transport kernels (2D and 3D).
#pragma once

namespace mcr {

// Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11): ten rounds of two 32x32->64 products and
// xors, Weyl-incremented key, on a 4-word counter.
__device__ __forceinline__ uint4 philox4x32_10_block(uint4 c, unsigned k0, unsigned k1) {
  unsigned c0 = c.x, c1 = c.y, c2 = c.z, c3 = c.w;
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const unsigned lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    const unsigned lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    const unsigned n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return make_uint4(c0, c1, c2, c3);
}

// The block of event `event` of packet `pid`: counter (pid_lo, pid_hi, event, 0).
__device__ __forceinline__ uint4 philox4x32_10(unsigned long long pid, unsigned event, unsigned k0,
                                               unsigned k1) {
  return philox4x32_10_block(make_uint4((unsigned)pid, (unsigned)(pid >> 32), event, 0u), k0, k1);
}

// Uniform in (0,1): ((x >> 9) + 1/2) 2^-23, exact in FP32.  Built from the bits: 1 + m 2^-23
// (m = x >> 9 as the mantissa) minus (1 - 2^-24) is exactly (2m + 1) 2^-24, a 24-bit value, so
// the subtraction is exact and no integer-to-float conversion is needed.
__device__ __forceinline__ float u01(unsigned x) { return __uint_as_float(0x3F800000u | (x >> 9)) - 0x1.fffffep-1f; }

}  // namespace mcr
