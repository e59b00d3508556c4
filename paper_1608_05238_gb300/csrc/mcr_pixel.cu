// mcr_pixel.cu -- the per-pixel kernels around the transport (all memory-bound, one pass each):
// medium packing, the volumetric source CDF, tally finalisation (fixed point -> normalised
// channel-major FP32), H and eps (Sec. 2, Eq. 2), the adjoint source (Sec. 6) and the
// functional gradients (Sec. 5, Eqs. 22 and 28).
#include <math_constants.h>

#include "mcr_internal.h"

namespace mcr {
namespace {

constexpr int kThreads = 256;

// (mu_a, mu_s, 1/mu_a, 1/mu_s) per pixel, one 16-byte load per segment; 1/0 = +inf
__global__ void k_pack_medium(const float *__restrict__ mua, const float *__restrict__ mus, float4 *__restrict__ mu,
                              int64_t npix, unsigned *flags) {
  bool bad = false;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x) {
    const float a = mua[i], s = mus[i];
    bad |= !(a >= 0.f && a < CUDART_INF_F) || !(s >= 0.f && s < CUDART_INF_F);
    mu[i] = make_float4(a, s, 1.f / a, 1.f / s);
  }
  if (__any_sync(0xFFFFFFFFu, bad) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagMedium);
}

// max |q| as the bit pattern of a non-negative float (monotone as an unsigned integer)
__global__ void k_abs_max(const float *__restrict__ q, int64_t npix, unsigned *qmax_bits) {
  unsigned m = 0;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < npix; i += (int64_t)gridDim.x * blockDim.x)
    m = max(m, __float_as_uint(fabsf(q[i])));
  m = __reduce_max_sync(0xFFFFFFFFu, m);
  if ((threadIdx.x & 31) == 0 && m) atomicMax(qmax_bits, m);
}

// Block-local inclusive scan of w_i = floor(|q_i| / qmax * 2^32); writes block totals.
__global__ void k_cdf_local(const float *__restrict__ q, int64_t npix, const unsigned *qmax_bits,
                            unsigned long long *__restrict__ cdf, unsigned long long *__restrict__ block_sums) {
  __shared__ unsigned long long warp_tot[kThreads / 32];
  const double qmax = (double)__uint_as_float(*qmax_bits);
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  unsigned long long w = 0;
  if (i < npix && qmax > 0.0) w = (unsigned long long)floor(fabs((double)q[i]) / qmax * 4294967296.0);
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  unsigned long long v = w;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const unsigned long long n = __shfl_up_sync(0xFFFFFFFFu, v, o);
    if (lane >= o) v += n;
  }
  if (lane == 31) warp_tot[wid] = v;
  __syncthreads();
  if (wid == 0) {
    unsigned long long t = lane < kThreads / 32 ? warp_tot[lane] : 0ull;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long n = __shfl_up_sync(0xFFFFFFFFu, t, o);
      if (lane >= o) t += n;
    }
    if (lane < kThreads / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  if (wid > 0) v += warp_tot[wid - 1];
  if (i < npix) cdf[i] = v;
  if (threadIdx.x == kThreads - 1) block_sums[blockIdx.x] = v;
}

// Exclusive scan of the block totals (one block, sequential over chunks of 32).
__global__ void k_cdf_blocks(unsigned long long *block_sums, int nblocks) {
  const int lane = threadIdx.x;
  unsigned long long carry = 0;
  for (int base = 0; base < nblocks; base += 32) {
    const int i = base + lane;
    const unsigned long long x = i < nblocks ? block_sums[i] : 0ull;
    unsigned long long v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned long long n = __shfl_up_sync(0xFFFFFFFFu, v, o);
      if (lane >= o) v += n;
    }
    if (i < nblocks) block_sums[i] = carry + v - x;
    carry += __shfl_sync(0xFFFFFFFFu, v, 31);
  }
}

__global__ void k_cdf_add(unsigned long long *__restrict__ cdf, int64_t npix,
                          const unsigned long long *__restrict__ block_sums) {
  const int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x;
  if (i < npix) cdf[i] += block_sums[blockIdx.x];
}

// acc[c][pix] += tally[pix][c] * quantum ; the tally tile of 32 pixels is read contiguously.
__global__ void k_accumulate(const unsigned long long *__restrict__ tally, int64_t npix, int C, int Cpad,
                             double quantum, double *__restrict__ acc) {
  const int64_t p0 = (int64_t)blockIdx.x * 32;
  for (int c = threadIdx.y; c < C; c += blockDim.y) {
    const int64_t pix = p0 + threadIdx.x;
    if (pix < npix) acc[(int64_t)c * npix + pix] += (double)(long long)tally[pix * Cpad + c] * quantum;
  }
}

// Normalisation S / (N_p A) of a run's sums.  Volumetric: S = 2 pi A qmax total 2^-32 (the source
// CDF has 2^32 levels of qmax), read on the device; otherwise the host's fixed_scale.
__device__ __forceinline__ double run_scale(double fixed_scale, int volumetric, const unsigned *qmax_bits,
                                            const unsigned long long *cdf_total, double n_packets) {
  if (!volumetric) return fixed_scale;
  return 2.0 * CUDART_PI * (double)__uint_as_float(*qmax_bits) * (double)(*cdf_total) * (1.0 / 4294967296.0) /
         n_packets;
}

// Raw fixed-point sums out, pixel-major [npix][Cpad] -> channel-major [C][npix] int64 (written, or
// added with `accumulate`); the tile of 32 pixels is staged through shared memory as in k_finalize.
__global__ void k_export_raw(const unsigned long long *__restrict__ tally, int64_t npix, int C, int Cpad,
                             int accumulate, long long *__restrict__ out) {
  extern __shared__ long long tile[];  // [32][Cpad]
  const int64_t p0 = (int64_t)blockIdx.x * 32;
  const int npx = npix - p0 < 32 ? (int)(npix - p0) : 32;
  const int tid = threadIdx.y * 32 + threadIdx.x, nthr = blockDim.x * blockDim.y;
  const long long *src = reinterpret_cast<const long long *>(tally) + p0 * Cpad;
  // a row's words [C, Cpad) are not read: with a row offset (dense rows) the last pixel's would lie
  // past the tally
  for (int k = tid; k < npx * Cpad; k += nthr)
    if (k % Cpad < C) tile[k] = src[k];
  __syncthreads();
  for (int c = threadIdx.y; c < C; c += blockDim.y) {
    if (threadIdx.x < npx) {
      long long *o = out + (int64_t)c * npix + p0 + threadIdx.x;
      const long long v = tile[threadIdx.x * Cpad + c];
      *o = accumulate ? *o + v : v;
    }
  }
}

// Channel-major raw sums (e.g. summed over the packet ranges of several GPUs) -> normalised FP32:
// coeff[c][pix] (=, or += with `accumulate`) sign * raw * quantum * scale, sign (-1)^n on the
// channels of order n when `adjoint`.  Flags sums within 2 bits of overflow.
__global__ void k_finalize_raw(const long long *__restrict__ raw, int64_t npix, int C, double quantum,
                               double fixed_scale, int volumetric, const unsigned *qmax_bits,
                               const unsigned long long *cdf_total, double n_packets, int adjoint, int accumulate,
                               float *__restrict__ coeff, unsigned *flags) {
  const double scale = run_scale(fixed_scale, volumetric, qmax_bits, cdf_total, n_packets);
  bool near_overflow = false;
  const int64_t total = (int64_t)C * npix;
  for (int64_t k = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; k < total; k += (int64_t)gridDim.x * blockDim.x) {
    const int c = (int)(k / npix);
    const int n = (c + 1) >> 1;
    const double sgn = (adjoint && (n & 1)) ? -1.0 : 1.0;
    const long long v = raw[k];
    near_overflow |= (v > (1ll << 61)) || (v < -(1ll << 61));
    const float f = (float)(sgn * ((double)v * quantum * scale));
    coeff[k] = accumulate ? coeff[k] + f : f;
  }
  if (__any_sync(0xFFFFFFFFu, near_overflow) && (threadIdx.x & 31) == 0) atomicOr(flags, kFlagOverflow);
}

// Fixed point (or FP64 accumulator) -> normalised FP32, pixel-major -> channel-major.
// One block = 32 pixels: the tile [32][Cpad] is staged through shared memory so that both the
// read (contiguous rows) and the write (32 pixels per channel) are coalesced.
__global__ void k_finalize(const unsigned long long *__restrict__ tally, const double *__restrict__ acc,
                           int64_t npix, int C, int Cpad, double quantum, double fixed_scale, int volumetric,
                           const unsigned *qmax_bits, const unsigned long long *cdf_total, double n_packets,
                           int adjoint, int accumulate, float *__restrict__ coeff, unsigned *flags) {
  extern __shared__ long long tile[];  // [32][Cpad]
  const int64_t p0 = (int64_t)blockIdx.x * 32;
  const int npx = npix - p0 < 32 ? (int)(npix - p0) : 32;
  const double scale = run_scale(fixed_scale, volumetric, qmax_bits, cdf_total, n_packets);
  const int tid = threadIdx.y * 32 + threadIdx.x, nthr = blockDim.x * blockDim.y;
  bool near_overflow = false;
  if (!acc) {
    const long long *src = reinterpret_cast<const long long *>(tally) + p0 * Cpad;
    for (int k = tid; k < npx * Cpad; k += nthr) {
      if (k % Cpad >= C) continue;  // as in k_export_raw: only the row's C words are read
      const long long v = src[k];
      near_overflow |= (v > (1ll << 61)) || (v < -(1ll << 61));
      tile[k] = v;
    }
    __syncthreads();
  }
  for (int c = threadIdx.y; c < C; c += blockDim.y) {
    const int n = (c + 1) >> 1;
    const double sgn = (adjoint && (n & 1)) ? -1.0 : 1.0;
    if (threadIdx.x < npx) {
      const int64_t pix = p0 + threadIdx.x;
      double v;
      if (acc)
        v = acc[(int64_t)c * npix + pix] * scale;
      else
        v = (double)tile[threadIdx.x * Cpad + c] * quantum * scale;
      float *o = coeff + (int64_t)c * npix + pix;
      *o = accumulate ? *o + (float)(sgn * v) : (float)(sgn * v);
    }
  }
  if (__syncthreads_or(near_overflow) && tid == 0) atomicOr(flags, kFlagOverflow);
}

// H = mu_a a_0 (or H = a0 when mua is null) ; r = H^meas - H ; dL/dH = -A r ; per-block FP64
// partial sums of r^2.
__global__ void k_h_eps(const float *__restrict__ mua, const float *__restrict__ a0, const float *__restrict__ Hmeas,
                        int64_t npix, double area, float *__restrict__ H, float *__restrict__ dL_dH,
                        double *__restrict__ partials) {
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < npix; i += (int64_t)gridDim.x * kThreads) {
    const float h = mua ? mua[i] * a0[i] : a0[i];
    if (H) H[i] = h;
    if (Hmeas) {
      const double r = (double)Hmeas[i] - (double)h;  // residual and its square in FP64
      if (dL_dH) dL_dH[i] = (float)(-area * r);
      acc += r * r;
    }
  }
  if (!partials) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

// Per-block FP64 partial sums of a_i b_i (grid-stride, a fixed order for a given grid).
__global__ void k_dot(const float *__restrict__ a, const float *__restrict__ b, int64_t n,
                      double *__restrict__ partials) {
  __shared__ double red[kThreads / 32];
  double acc = 0.0;
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < n; i += (int64_t)gridDim.x * kThreads)
    acc += (double)a[i] * (double)b[i];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kThreads / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

// eps = 1/2 A sum(partials), summed by one thread in block order (deterministic).
__global__ void k_eps_final(const double *__restrict__ partials, int n, double half_area, double *eps) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += partials[i];
  *eps = half_area * s;
}

__global__ void k_adjoint_source(const float *__restrict__ mua, const float *__restrict__ dL_dH, int64_t npix,
                                 double area, float *__restrict__ q) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < npix; i += (int64_t)gridDim.x * kThreads)
    q[i] = (float)(-(double)mua[i] * (double)dL_dH[i] / area);
}

// Per pixel, FP64: G_a = a0 a0*/(2pi) + (1/pi) sum (a_n a_n* + b_n b_n*)      (Eq. 22)
//                  G_s = (1/pi) sum (a_n a_n* + b_n b_n*)(1 - g^n)            (Eq. 28)
template <typename OutT>
__global__ void k_gradient(const float *__restrict__ F, const float *__restrict__ Fs, const float *__restrict__ v,
                           int64_t npix, int K, double g, double area, OutT *__restrict__ d_mua,
                           OutT *__restrict__ d_mus) {
  for (int64_t i = blockIdx.x * (int64_t)kThreads + threadIdx.x; i < npix; i += (int64_t)gridDim.x * kThreads) {
    const double a0 = F[i];
    double Ga = a0 * (double)Fs[i] * (0.5 / CUDART_PI);
    double Gs = 0.0, gn = 1.0;
    for (int n = 1; n <= K; ++n) {
      gn *= g;
      const int64_t ca = (int64_t)(2 * n - 1) * npix + i, cb = (int64_t)(2 * n) * npix + i;
      const double pr = (double)F[ca] * (double)Fs[ca] + (double)F[cb] * (double)Fs[cb];
      Ga += pr * (1.0 / CUDART_PI);
      Gs += pr * (1.0 - gn) * (1.0 / CUDART_PI);
    }
    d_mua[i] = (OutT)((double)v[i] * a0 + area * Ga);
    if (d_mus) d_mus[i] = (OutT)(area * Gs);
  }
}

int grid_for(int64_t n, int threads) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int64_t blocks = (n + threads - 1) / threads;
  const int64_t cap = (int64_t)sms * 8;
  return (int)(blocks < 1 ? 1 : (blocks < cap ? blocks : cap));
}

}  // namespace

cudaError_t launch_pack_medium(const float *mua, const float *mus, float4 *mu, int64_t npix, unsigned *flags,
                               cudaStream_t s) {
  k_pack_medium<<<grid_for(npix, kThreads), kThreads, 0, s>>>(mua, mus, mu, npix, flags);
  return cudaGetLastError();
}

cudaError_t launch_source_cdf(const float *q, int64_t npix, unsigned long long *cdf, unsigned long long *block_sums,
                              size_t block_sums_cap, unsigned *qmax_bits, cudaStream_t s) {
  const int64_t nblocks = (npix + kThreads - 1) / kThreads;
  if ((size_t)nblocks > block_sums_cap) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(qmax_bits, 0, sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  k_abs_max<<<grid_for(npix, kThreads), kThreads, 0, s>>>(q, npix, qmax_bits);
  k_cdf_local<<<(unsigned)nblocks, kThreads, 0, s>>>(q, npix, qmax_bits, cdf, block_sums);
  k_cdf_blocks<<<1, 32, 0, s>>>(block_sums, (int)nblocks);
  k_cdf_add<<<(unsigned)nblocks, kThreads, 0, s>>>(cdf, npix, block_sums);
  return cudaGetLastError();
}

cudaError_t launch_accumulate(const unsigned long long *tally, int64_t npix, int C, int Cpad, double quantum,
                              double *acc, cudaStream_t s) {
  const dim3 block(32, 8);
  k_accumulate<<<(unsigned)((npix + 31) / 32), block, 0, s>>>(tally, npix, C, Cpad, quantum, acc);
  return cudaGetLastError();
}

cudaError_t launch_finalize(const unsigned long long *tally, const double *acc, int64_t npix, int C, int Cpad,
                            double quantum, double fixed_scale, bool volumetric, const unsigned *qmax_bits,
                            const unsigned long long *cdf_total, double n_packets, bool adjoint, bool accumulate,
                            float *coeff, unsigned *flags, cudaStream_t s) {
  const dim3 block(32, 8);
  const size_t smem = acc ? 0 : (size_t)32 * Cpad * sizeof(long long);
  k_finalize<<<(unsigned)((npix + 31) / 32), block, smem, s>>>(tally, acc, npix, C, Cpad, quantum, fixed_scale,
                                                              volumetric ? 1 : 0, qmax_bits, cdf_total, n_packets,
                                                              adjoint ? 1 : 0, accumulate ? 1 : 0, coeff, flags);
  return cudaGetLastError();
}

cudaError_t launch_export_raw(const unsigned long long *tally, int64_t npix, int C, int Cpad, bool accumulate,
                              long long *out, cudaStream_t s) {
  const dim3 block(32, 8);
  k_export_raw<<<(unsigned)((npix + 31) / 32), block, (size_t)32 * Cpad * sizeof(long long), s>>>(
      tally, npix, C, Cpad, accumulate ? 1 : 0, out);
  return cudaGetLastError();
}

cudaError_t launch_finalize_raw(const long long *raw, int64_t npix, int C, double quantum, double fixed_scale,
                                bool volumetric, const unsigned *qmax_bits, const unsigned long long *cdf_total,
                                double n_packets, bool adjoint, bool accumulate, float *coeff, unsigned *flags,
                                cudaStream_t s) {
  k_finalize_raw<<<grid_for((int64_t)C * npix, kThreads), kThreads, 0, s>>>(
      raw, npix, C, quantum, fixed_scale, volumetric ? 1 : 0, qmax_bits, cdf_total, n_packets, adjoint ? 1 : 0,
      accumulate ? 1 : 0, coeff, flags);
  return cudaGetLastError();
}

cudaError_t launch_h_eps(const float *mua, const float *a0, const float *Hmeas, int64_t npix, double area, float *H,
                         float *dL_dH, double *partials, size_t partials_cap, double *eps, cudaStream_t s) {
  int grid = grid_for(npix, kThreads);
  if ((size_t)grid > partials_cap) grid = (int)partials_cap;
  k_h_eps<<<grid, kThreads, 0, s>>>(mua, a0, Hmeas, npix, area, H, dL_dH, (Hmeas && eps) ? partials : nullptr);
  if (Hmeas && eps) k_eps_final<<<1, 1, 0, s>>>(partials, grid, 0.5 * area, eps);
  return cudaGetLastError();
}

cudaError_t launch_dot(const float *a, const float *b, int64_t n, double *partials, size_t partials_cap, double *out,
                       cudaStream_t s) {
  int grid = grid_for(n, kThreads);
  if ((size_t)grid > partials_cap) grid = (int)partials_cap;
  k_dot<<<grid, kThreads, 0, s>>>(a, b, n, partials);
  k_eps_final<<<1, 1, 0, s>>>(partials, grid, 1.0, out);
  return cudaGetLastError();
}

cudaError_t launch_adjoint_source(const float *mua, const float *dL_dH, int64_t npix, double area, float *q,
                                  cudaStream_t s) {
  k_adjoint_source<<<grid_for(npix, kThreads), kThreads, 0, s>>>(mua, dL_dH, npix, area, q);
  return cudaGetLastError();
}

cudaError_t launch_gradient(const float *coeff, const float *coeff_adj, const float *dL_dH, int64_t npix, int K,
                            double g, double area, double *d_mua, double *d_mus, cudaStream_t s) {
  k_gradient<double><<<grid_for(npix, kThreads), kThreads, 0, s>>>(coeff, coeff_adj, dL_dH, npix, K, g, area, d_mua,
                                                                   d_mus);
  return cudaGetLastError();
}

cudaError_t launch_gradient_f32(const float *coeff, const float *coeff_adj, const float *dL_dH, int64_t npix, int K,
                                double g, double area, float *d_mua, float *d_mus, cudaStream_t s) {
  k_gradient<float><<<grid_for(npix, kThreads), kThreads, 0, s>>>(coeff, coeff_adj, dL_dH, npix, K, g, area, d_mua,
                                                                  d_mus);
  return cudaGetLastError();
}

}  // namespace mcr
