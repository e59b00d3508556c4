// mcr_harmonics.cuh -- the harmonic row of a direction, shared by every kernel that deposits into
// the 2D tally, so that all of them multiply a track weight by bit-identical coefficients.
#pragma once

namespace mcr {

// h = (1, cos theta, sin theta, ..., cos K theta, sin K theta) of the direction
// (s_x, s_z) = (sin theta, cos theta), from (s_z + i s_x)^n by K complex products (Eqs. 9-11
// without trigonometry).  Channel c goes to my[1 + c], so each (cos n theta, sin n theta) pair is
// one 8-byte aligned store at word 2n.
__device__ __forceinline__ void harmonic_row(float *my, float sx, float sz, int K) {
  my[1] = 1.f;
  float c = sz, s = sx;
  float2 *pairs = reinterpret_cast<float2 *>(my);
#pragma unroll 4
  for (int n = 1; n <= K; ++n) {
    pairs[n] = make_float2(c, s);
    const float cn = fmaf(c, sz, -s * sx);
    const float sn = fmaf(s, sz, c * sx);
    c = cn;
    s = sn;
  }
}

}  // namespace mcr
