// dn_ops.cu -- the memory-bound kernels of the denoiser U-Net: layout changes, pooling and
// up-sampling with their backward passes (ReLU masks and skip gradients fused), bias
// gradients, the residual MSE loss and the Adam update that also writes the BF16 weight copies.
// Tensors are NHWC bf16 slices described by (pointer, channel stride, channel offset).
#include <cuda_bf16.h>

#include "dn_internal.h"

namespace dn {
namespace {

constexpr int kT = 256;

__device__ __forceinline__ float bf(const __nv_bfloat16 v) { return __bfloat162float(v); }

int blocks_for(long long n) {
  long long b = (n + kT - 1) / kT;
  if (b < 1) b = 1;
  if (b > 152 * 32) b = 152 * 32;
  return (int)b;
}

// [B][HW][stride] slice (off, C) -> dst [C][B][HW]; with `shifted`, three copies along x
// (dst + k * C * B * HW holds x shifted by k - 1, zero outside the row).
__global__ void k_to_ct(const __nv_bfloat16 *__restrict__ src, int B, int HW, int W, int stride, int off, int C,
                        int shifted, __nv_bfloat16 *__restrict__ dst) {
  __shared__ float tile[32][33];
  const int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32, b = blockIdx.z;
  // load 32 pixels x 32 channels (rows = pixels)
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int p = p0 + r, c = c0 + threadIdx.x;
    tile[r][threadIdx.x] = (p < HW && c < C) ? bf(src[((size_t)b * HW + p) * stride + off + c]) : 0.f;
  }
  __syncthreads();
  const size_t plane = (size_t)C * B * HW;
  for (int r = threadIdx.y; r < 32; r += blockDim.y) {
    const int c = c0 + r, p = p0 + threadIdx.x;
    if (c >= C || p >= HW) continue;
    __nv_bfloat16 *d = dst + ((size_t)c * B + b) * HW + p;
    if (!shifted) {
      *d = __float2bfloat16_rn(tile[threadIdx.x][r]);
    } else {
      const int x = p % W;
      for (int k = 0; k < 3; ++k) {
        const int xs = x + k - 1;
        float v = 0.f;
        if (xs >= 0 && xs < W) {
          const int ps = p + k - 1;
          const int lr = ps - p0;
          v = (lr >= 0 && lr < 32) ? tile[lr][r] : bf(src[((size_t)b * HW + ps) * stride + off + c]);
        }
        d[k * plane] = __float2bfloat16_rn(v);
      }
    }
  }
}

// The pooling / up-sampling kernels below use one thread per (pixel, channel) with a 3D grid:
// x = blockIdx.x * 8 + threadIdx.y is the pixel column, blockIdx.y the pixel row over all images
// (row R of image b is b * rows + y, so the 2x2 neighbourhoods follow from R by shifts), and
// c = blockIdx.z * 32 + threadIdx.x the channel: a warp touches 32 consecutive channels of one
// pixel and no thread divides.

// 2x2 average pooling: dst[R][x] = mean of src[2R..2R+1][2x..2x+1] (dst Wo = W/2 columns)
__global__ void k_pool2(const __nv_bfloat16 *__restrict__ src, int W, int sstride, int soff, int C,
                        __nv_bfloat16 *__restrict__ dst, int dstride, int doff) {
  const int x = blockIdx.x * 8 + threadIdx.y, R = blockIdx.y, c = blockIdx.z * 32 + threadIdx.x;
  const int Wo = W >> 1;
  if (x >= Wo || c >= C) return;
  const size_t s00 = ((size_t)(2 * R) * W + 2 * x) * sstride + soff + c;
  const float v = 0.25f * (bf(src[s00]) + bf(src[s00 + sstride]) + bf(src[s00 + (size_t)W * sstride]) +
                           bf(src[s00 + (size_t)W * sstride + sstride]));
  dst[((size_t)R * Wo + x) * dstride + doff + c] = __float2bfloat16_rn(v);
}

// backward of pool2 plus an optional skip gradient, times the ReLU mask of the pooled tensor:
// dz[R][x] = (skip[R][x] + dp[R/2][x/2] / 4) * (act[R][x] > 0) on the full-resolution grid
__global__ void k_pool2_bwd(const __nv_bfloat16 *__restrict__ dp, int pstride, int poff,
                            const __nv_bfloat16 *__restrict__ skip, int kstride, int koff,
                            const __nv_bfloat16 *__restrict__ act, int astride, int aoff, int W, int C,
                            __nv_bfloat16 *__restrict__ dz, int zstride, int zoff) {
  const int x = blockIdx.x * 8 + threadIdx.y, R = blockIdx.y, c = blockIdx.z * 32 + threadIdx.x;
  if (x >= W || c >= C) return;
  const size_t pix = (size_t)R * W + x;
  float g = 0.25f * bf(dp[((size_t)(R >> 1) * (W >> 1) + (x >> 1)) * pstride + poff + c]);
  if (skip) g += bf(skip[pix * kstride + koff + c]);
  if (!(bf(act[pix * astride + aoff + c]) > 0.f)) g = 0.f;
  dz[pix * zstride + zoff + c] = __float2bfloat16_rn(g);
}

// nearest 2x up-sampling: dst[R][x] = src[R/2][x/2]   (src W columns, dst 2W)
__global__ void k_up2(const __nv_bfloat16 *__restrict__ src, int W, int sstride, int soff, int C,
                      __nv_bfloat16 *__restrict__ dst, int dstride, int doff) {
  const int x = blockIdx.x * 8 + threadIdx.y, R = blockIdx.y, c = blockIdx.z * 32 + threadIdx.x;
  if (x >= 2 * W || c >= C) return;
  dst[((size_t)R * 2 * W + x) * dstride + doff + c] = src[((size_t)(R >> 1) * W + (x >> 1)) * sstride + soff + c];
}

// backward of up2 times the ReLU mask of its input: dz[R][x] = sum_2x2 du * (act > 0)  (dz W columns)
__global__ void k_up2_bwd(const __nv_bfloat16 *__restrict__ du, int ustride, int uoff,
                          const __nv_bfloat16 *__restrict__ act, int astride, int aoff, int W, int C,
                          __nv_bfloat16 *__restrict__ dz, int zstride, int zoff) {
  const int x = blockIdx.x * 8 + threadIdx.y, R = blockIdx.y, c = blockIdx.z * 32 + threadIdx.x;
  if (x >= W || c >= C) return;
  const size_t u00 = ((size_t)(2 * R) * 2 * W + 2 * x) * ustride + uoff + c;
  float g = bf(du[u00]) + bf(du[u00 + ustride]) + bf(du[u00 + (size_t)2 * W * ustride]) +
            bf(du[u00 + (size_t)2 * W * ustride + ustride]);
  const size_t pix = (size_t)R * W + x;
  if (!(bf(act[pix * astride + aoff + c]) > 0.f)) g = 0.f;
  dz[pix * zstride + zoff + c] = __float2bfloat16_rn(g);
}

// 16-byte variants of the four kernels above (8 channels per thread, threadIdx.x over the C/8
// channel groups of a pixel, threadIdx.y over pixels of the row), used when every channel count,
// stride and offset is a multiple of 8; a warp then moves whole 128-byte pixel rows.
union BF8 {
  uint4 u;
  __nv_bfloat162 h[4];
};
__device__ __forceinline__ uint4 ld8(const __nv_bfloat16 *p) { return *reinterpret_cast<const uint4 *>(p); }
__device__ __forceinline__ void st8(__nv_bfloat16 *p, uint4 v) { *reinterpret_cast<uint4 *>(p) = v; }

__global__ void k_up2_v8(const __nv_bfloat16 *__restrict__ src, int W, int sstride, int soff, int G,
                         __nv_bfloat16 *__restrict__ dst, int dstride, int doff) {
  const int g = threadIdx.x, x = blockIdx.x * blockDim.y + threadIdx.y, R = blockIdx.y;
  if (g >= G || x >= 2 * W) return;
  st8(dst + ((size_t)R * 2 * W + x) * dstride + doff + 8 * g,
      ld8(src + ((size_t)(R >> 1) * W + (x >> 1)) * sstride + soff + 8 * g));
}

__global__ void k_pool2_v8(const __nv_bfloat16 *__restrict__ src, int W, int sstride, int soff, int G,
                           __nv_bfloat16 *__restrict__ dst, int dstride, int doff) {
  const int g = threadIdx.x, x = blockIdx.x * blockDim.y + threadIdx.y, R = blockIdx.y;
  const int Wo = W >> 1;
  if (g >= G || x >= Wo) return;
  const size_t s00 = ((size_t)(2 * R) * W + 2 * x) * sstride + soff + 8 * g;
  BF8 a, b, c, d, o;
  a.u = ld8(src + s00);
  b.u = ld8(src + s00 + sstride);
  c.u = ld8(src + s00 + (size_t)W * sstride);
  d.u = ld8(src + s00 + (size_t)W * sstride + sstride);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 fa = __bfloat1622float2(a.h[k]), fb = __bfloat1622float2(b.h[k]), fc = __bfloat1622float2(c.h[k]),
                 fd = __bfloat1622float2(d.h[k]);
    o.h[k] = __floats2bfloat162_rn(0.25f * (fa.x + fb.x + fc.x + fd.x), 0.25f * (fa.y + fb.y + fc.y + fd.y));
  }
  st8(dst + ((size_t)R * Wo + x) * dstride + doff + 8 * g, o.u);
}

__global__ void k_pool2_bwd_v8(const __nv_bfloat16 *__restrict__ dp, int pstride, int poff,
                               const __nv_bfloat16 *__restrict__ skip, int kstride, int koff,
                               const __nv_bfloat16 *__restrict__ act, int astride, int aoff, int W, int G,
                               __nv_bfloat16 *__restrict__ dz, int zstride, int zoff) {
  const int g = threadIdx.x, x = blockIdx.x * blockDim.y + threadIdx.y, R = blockIdx.y;
  if (g >= G || x >= W) return;
  const size_t pix = (size_t)R * W + x;
  BF8 p, k, a, o;
  p.u = ld8(dp + ((size_t)(R >> 1) * (W >> 1) + (x >> 1)) * pstride + poff + 8 * g);
  a.u = ld8(act + pix * astride + aoff + 8 * g);
  if (skip) k.u = ld8(skip + pix * kstride + koff + 8 * g);
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    float2 v = __bfloat1622float2(p.h[j]);
    v.x *= 0.25f;
    v.y *= 0.25f;
    if (skip) {
      const float2 w = __bfloat1622float2(k.h[j]);
      v.x += w.x;
      v.y += w.y;
    }
    const float2 m = __bfloat1622float2(a.h[j]);
    o.h[j] = __floats2bfloat162_rn(m.x > 0.f ? v.x : 0.f, m.y > 0.f ? v.y : 0.f);
  }
  st8(dz + pix * zstride + zoff + 8 * g, o.u);
}

__global__ void k_up2_bwd_v8(const __nv_bfloat16 *__restrict__ du, int ustride, int uoff,
                             const __nv_bfloat16 *__restrict__ act, int astride, int aoff, int W, int G,
                             __nv_bfloat16 *__restrict__ dz, int zstride, int zoff) {
  const int g = threadIdx.x, x = blockIdx.x * blockDim.y + threadIdx.y, R = blockIdx.y;
  if (g >= G || x >= W) return;
  const size_t u00 = ((size_t)(2 * R) * 2 * W + 2 * x) * ustride + uoff + 8 * g;
  BF8 a, b, c, d, m, o;
  a.u = ld8(du + u00);
  b.u = ld8(du + u00 + ustride);
  c.u = ld8(du + u00 + (size_t)2 * W * ustride);
  d.u = ld8(du + u00 + (size_t)2 * W * ustride + ustride);
  const size_t pix = (size_t)R * W + x;
  m.u = ld8(act + pix * astride + aoff + 8 * g);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const float2 fa = __bfloat1622float2(a.h[k]), fb = __bfloat1622float2(b.h[k]), fc = __bfloat1622float2(c.h[k]),
                 fd = __bfloat1622float2(d.h[k]), fm = __bfloat1622float2(m.h[k]);
    o.h[k] = __floats2bfloat162_rn(fm.x > 0.f ? fa.x + fb.x + fc.x + fd.x : 0.f,
                                   fm.y > 0.f ? fa.y + fb.y + fc.y + fd.y : 0.f);
  }
  st8(dz + pix * zstride + zoff + 8 * g, o.u);
}

// db[c] += sum over pixels of dz[p][c]
__global__ void k_bias_grad(const __nv_bfloat16 *__restrict__ dz, long long P, int stride, int off, int C,
                            float *__restrict__ db) {
  const int c = blockIdx.y * 32 + threadIdx.x;
  float acc = 0.f;
  if (c < C)
    for (long long p = blockIdx.x * (long long)blockDim.y + threadIdx.y; p < P; p += (long long)gridDim.x * blockDim.y)
      acc += bf(dz[p * stride + off + c]);
  __shared__ float red[8][32];
  red[threadIdx.y][threadIdx.x] = acc;
  __syncthreads();
  if (threadIdx.y == 0 && c < C) {
    float s = 0.f;
    for (int k = 0; k < (int)blockDim.y; ++k) s += red[k][threadIdx.x];
    atomicAdd(db + c, s);
  }
}

// db[c] += sum over pixels of dz[p][off + c] (c < C) with 16-byte loads: G = ceil(C / 8) threads
// cover one pixel row (8 channels each; the row holds at least 8 G channels from off, those past
// C are read and dropped), 256 / G rows per pass of the block; per-thread FP32 sums, a
// fixed-order sum over the block's rows in shared memory, one atomic add per channel and block.
__global__ void __launch_bounds__(256) k_bias_grad_v8(const __nv_bfloat16 *__restrict__ dz, long long P, int stride,
                                                      int off, int G, int C, float *__restrict__ db) {
  __shared__ float red[256 * 8];
  const int R = 256 / G, t = threadIdx.x, g = t % G, r = t / G, CG = 8 * G;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  if (r < R) {
#pragma unroll 4
    for (long long p = (long long)blockIdx.x * R + r; p < P; p += (long long)gridDim.x * R) {
      const uint4 u = __ldg(reinterpret_cast<const uint4 *>(dz + p * stride + off) + g);
      const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float2 f = __bfloat1622float2(h[j]);
        acc[2 * j] += f.x;
        acc[2 * j + 1] += f.y;
      }
    }
#pragma unroll
    for (int j = 0; j < 8; ++j) red[r * CG + 8 * g + j] = acc[j];
  }
  __syncthreads();
  for (int c = t; c < C; c += 256) {
    float sum = 0.f;
    for (int k = 0; k < R; ++k) sum += red[k * CG + c];
    atomicAdd(db + c, sum);
  }
}

// residual MSE: y = x + out over C channels; loss partials (FP64) and dout = 2 (y - t) / count
// written as bf16 NHWC (stride dstride) for the next convolution's input gradient.
// One thread per (pixel, channel): threadIdx.x over channels, the rest over pixels (grid-stride),
// the difference in FP32, each thread's sum of squares in FP64 (fixed order).
__global__ void k_mse(const float *__restrict__ out, int ostride, const __nv_bfloat16 *__restrict__ x, int xstride,
                      const float *__restrict__ t, long long P, int C, float two_over_count,
                      __nv_bfloat16 *__restrict__ dout, int dstride, double *__restrict__ partials) {
  __shared__ double red[kT / 32];
  double acc = 0.0;
  const int c = threadIdx.x + 32 * blockIdx.y;
  if (c < C)
    for (long long p = blockIdx.x * 8ll + threadIdx.y; p < P; p += gridDim.x * 8ll) {
      const float d = bf(x[p * xstride + c]) + out[p * ostride + c] - t[p * C + c];
      acc += (double)(d * d);
      dout[p * dstride + c] = __float2bfloat16_rn(d * two_over_count);
    }
  const int tid = threadIdx.y * 32 + threadIdx.x;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kT / 32; ++w) s += red[w];
    partials[blockIdx.y * gridDim.x + blockIdx.x] = s;
  }
}

// One block: strided per-thread sums, then a fixed-order tree (deterministic).
__global__ void k_sum_partials(const double *__restrict__ partials, int n, double scale, double *out) {
  __shared__ double red[kT];
  double s = 0.0;
  for (int i = threadIdx.x; i < n; i += kT) s += partials[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int h = kT / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h) red[threadIdx.x] += red[threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = red[0] * scale;
}

// prediction y = x + out (fp32 [P][C] from [P][ostride]); used at inference
__global__ void k_residual(const float *__restrict__ out, int ostride, const __nv_bfloat16 *__restrict__ x,
                           int xstride, long long P, int C, float *__restrict__ y) {
  const int c = threadIdx.x + 32 * blockIdx.y;
  if (c >= C) return;
  for (long long p = blockIdx.x * 8ll + threadIdx.y; p < P; p += gridDim.x * 8ll)
    y[p * C + c] = bf(x[p * xstride + c]) + out[p * ostride + c];
}

// Adam on the FP32 master weights [cout][taps][cin] and bias; writes the forward BF16 copy
// wf [n_pad][taps][cin_pad] and the input-gradient copy wd [cin_npad][taps][cout_pad] with the
// taps flipped (wd[c][8 - t][n] = w[n][t][c] for 3x3).
// One Adam step with bias-corrected moments (ic1 = 1 / (1 - b1^t), ic2 = 1 / (1 - b2^t)) on
// registers.  Explicit roundings, so that every kernel that inlines this computes the same bits;
// the final quotient is the fast division (2 ulp: far below what an optimizer step needs).
__device__ __forceinline__ void adam_math(float &w, float &m, float &v, float g, float lr, float b1, float b2, float eps,
                                          float ic1, float ic2) {
  m = __fmaf_rn(b1, m, __fmul_rn(1.f - b1, g));
  v = __fmaf_rn(b2, v, __fmul_rn(__fmul_rn(1.f - b2, g), g));
  const float step = __fdividef(__fmul_rn(lr, __fmul_rn(m, ic1)), __fadd_rn(__fsqrt_rn(__fmul_rn(v, ic2)), eps));
  w = __fsub_rn(w, step);
}

// The same on element i of the arrays; the gradient is consumed (set to zero: the next backward
// pass accumulates from zero).  Returns the new weight.
__device__ __forceinline__ float adam_elem(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                                           float *__restrict__ g, size_t i, float lr, float b1, float b2, float eps,
                                           float ic1, float ic2) {
  float wi = w[i], mi = m[i], vi = v[i];
  const float gi = g[i];
  adam_math(wi, mi, vi, gi, lr, b1, b2, eps, ic1, ic2);
  g[i] = 0.f;
  m[i] = mi;
  v[i] = vi;
  w[i] = wi;
  return wi;
}

__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       float *__restrict__ g, int cout, int taps, int cin, float lr, float b1, float b2,
                       float eps, float ic1, float ic2, __nv_bfloat16 *__restrict__ wf, int cin_pad,
                       __nv_bfloat16 *__restrict__ wd, int cout_pad, int step) {
  const long long n = (long long)cout * taps * cin;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const float wi = step > 0 ? adam_elem(w, m, v, g, (size_t)i, lr, b1, b2, eps, ic1, ic2) : w[i];
    const int c = (int)(i % cin);
    const int t = (int)((i / cin) % taps);
    const int o = (int)(i / ((long long)cin * taps));
    const __nv_bfloat16 h = __float2bfloat16_rn(wi);
    wf[((size_t)o * taps + t) * cin_pad + c] = h;
    if (wd) wd[((size_t)c * taps + (taps - 1 - t)) * cout_pad + o] = h;
  }
}

// The same update when the transposed copy wd is wanted, through a 32 x 32 (cout x cin) tile of
// one tap: the update and wf are written along cin, wd along cout (both coalesced).
__global__ void k_adam_t(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                         float *__restrict__ g, int cout, int taps, int cin, float lr, float b1, float b2,
                         float eps, float ic1, float ic2, __nv_bfloat16 *__restrict__ wf, int cin_pad,
                         __nv_bfloat16 *__restrict__ wd, int cout_pad, int step) {
  __shared__ __nv_bfloat16 tile[32][34];
  const int c0 = blockIdx.x * 32, o0 = blockIdx.y * 32, t = blockIdx.z;
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int o = o0 + r, c = c0 + threadIdx.x;
    if (o < cout && c < cin) {
      const size_t i = ((size_t)o * taps + t) * cin + c;
      const float wi = step > 0 ? adam_elem(w, m, v, g, i, lr, b1, b2, eps, ic1, ic2) : w[i];
      const __nv_bfloat16 h = __float2bfloat16_rn(wi);
      wf[((size_t)o * taps + t) * cin_pad + c] = h;
      tile[r][threadIdx.x] = h;
    }
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r, o = o0 + threadIdx.x;
    if (o < cout && c < cin) wd[((size_t)c * taps + (taps - 1 - t)) * cout_pad + o] = tile[threadIdx.x][r];
  }
}

__global__ void k_adam_bias(float *__restrict__ b, float *__restrict__ m, float *__restrict__ v,
                            float *__restrict__ g, int n, float lr, float b1, float b2, float eps, float ic1,
                            float ic2) {
  const int i = blockIdx.x * kT + threadIdx.x;
  if (i < n) adam_elem(b, m, v, g, (size_t)i, lr, b1, b2, eps, ic1, ic2);
}

// All layers' Adam steps in one launch: block -> (layer, 32 x 32 (cout x cin) tile of one tap) by
// the table's first-block indices; the tile body is k_adam_t's (wd optional) and block 0 of a
// layer also steps its bias.  Same arithmetic as the per-layer kernels.
__global__ void k_adam_multi(const __grid_constant__ AdamTable T, float lr, float b1, float b2, float eps, float ic1,
                             float ic2, int step) {
  __shared__ __nv_bfloat16 tile[32][34];
  int l = 0;
  while (l + 1 < T.n && (int)blockIdx.x >= T.L[l + 1].tile0) ++l;
  const AdamLayer L = T.L[l];  // a register copy: the stores below cannot be assumed to miss the table
  const int local = (int)blockIdx.x - L.tile0;
  const int ct = (L.cin + 31) / 32, ot = (L.cout + 31) / 32;
  const int c0 = (local % ct) * 32, o0 = ((local / ct) % ot) * 32, t = local / (ct * ot);
  const int tid = threadIdx.y * 32 + threadIdx.x;
  // the tile's four rows of this thread: all loads first (memory-level parallelism), then the updates
  float wv[4], mv[4], vv[4], gv[4];
  size_t ix[4];
  bool in[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int o = o0 + threadIdx.y + 8 * k, c = c0 + threadIdx.x;
    in[k] = o < L.cout && c < L.cin;
    ix[k] = ((size_t)o * L.taps + t) * L.cin + c;
    wv[k] = in[k] ? L.w[ix[k]] : 0.f;
    if (step > 0 && in[k]) {
      mv[k] = L.m[ix[k]];
      vv[k] = L.v[ix[k]];
      gv[k] = L.g[ix[k]];
    }
  }
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    if (!in[k]) continue;
    const int r = threadIdx.y + 8 * k, o = o0 + r, c = c0 + threadIdx.x;
    if (step > 0) {
      adam_math(wv[k], mv[k], vv[k], gv[k], lr, b1, b2, eps, ic1, ic2);
      L.g[ix[k]] = 0.f;
      L.m[ix[k]] = mv[k];
      L.v[ix[k]] = vv[k];
      L.w[ix[k]] = wv[k];
    }
    const __nv_bfloat16 h = __float2bfloat16_rn(wv[k]);
    L.wf[((size_t)o * L.taps + t) * L.cin_pad + c] = h;
    tile[r][threadIdx.x] = h;
  }
  if (local == 0 && L.b && step > 0)
    for (int i = tid; i < L.cout; i += 256) adam_elem(L.b, L.mb, L.vb, L.gb, (size_t)i, lr, b1, b2, eps, ic1, ic2);
  if (!L.wd) return;  // uniform over the block
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r, o = o0 + threadIdx.x;
    if (o < L.cout && c < L.cin) L.wd[((size_t)c * L.taps + (L.taps - 1 - t)) * L.cout_pad + o] = tile[threadIdx.x][r];
  }
}

// Layout changes between channel-major [B][C][HW] maps (the MC's output) and pixel-major NHWC
// rows go through a 32 x 32 shared-memory tile (grid: pixel blocks x channel blocks x images),
// so both the reads and the writes are coalesced.

// channel-major fp32 coefficient maps [B][C][HW] * scale[b] -> NHWC bf16 [B][HW][stride]
__global__ void k_pack_input(const float *__restrict__ src, const float *__restrict__ scale, int HW, int C,
                             __nv_bfloat16 *__restrict__ dst, int stride) {
  __shared__ float tile[32][33];
  const int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32, b = blockIdx.z;
  const float sc = scale[b];
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r, p = p0 + threadIdx.x;
    tile[r][threadIdx.x] = (c < C && p < HW) ? src[((size_t)b * C + c) * HW + p] * sc : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int p = p0 + r, c = c0 + threadIdx.x;
    if (p < HW && c < C) dst[((size_t)b * HW + p) * stride + c] = __float2bfloat16_rn(tile[threadIdx.x][r]);
  }
}

// The same with 64 pixels x 64 channels per block and 16-byte stores (8 channels per thread, 8
// threads per 128-byte row segment); channels >= C are not written.  Requires HW % 64 == 0 and a
// 16-byte aligned dst with stride % 8 == 0.
__global__ void __launch_bounds__(256) k_pack_input_v8(const float *__restrict__ src, const float *__restrict__ scale,
                                                       int HW, int C, __nv_bfloat16 *__restrict__ dst, int stride) {
  __shared__ float tile[64][65];
  const int p0 = blockIdx.x * 64, c0 = blockIdx.y * 64, b = blockIdx.z, t = threadIdx.x;
  const float sc = scale[b];
  {
    const int pp = 2 * (t & 31);
    for (int r = t >> 5; r < 64; r += 8) {
      const int c = c0 + r;
      float2 v = make_float2(0.f, 0.f);
      if (c < C) v = __ldg(reinterpret_cast<const float2 *>(src + ((size_t)b * C + c) * HW + p0 + pp));
      tile[r][pp] = v.x * sc;
      tile[r][pp + 1] = v.y * sc;
    }
  }
  __syncthreads();
  for (int k = t; k < 64 * 8; k += 256) {
    const int px = k >> 3, g = k & 7, cg = c0 + 8 * g;
    if (cg >= C) continue;
    __nv_bfloat16 *o = dst + ((size_t)b * HW + p0 + px) * stride + cg;
    if (cg + 8 <= C) {
      __align__(16) __nv_bfloat162 h[4];
#pragma unroll
      for (int j = 0; j < 4; ++j) h[j] = __floats2bfloat162_rn(tile[8 * g + 2 * j][px], tile[8 * g + 2 * j + 1][px]);
      *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(h);
    } else {
      for (int j = 0; cg + j < C; ++j) o[j] = __float2bfloat16_rn(tile[8 * g + j][px]);
    }
  }
}

// per-sample input scale 1 / mean(channel 0) of channel-major fp32 maps [B][C][HW] (the fluence
// a_0 of a harmonic map), one block per sample, FP64 sum in a fixed order
__global__ void k_sample_scale(const float *__restrict__ src, int C, long long HW, float *__restrict__ scale) {
  __shared__ double red[kT / 32];
  const float *x = src + (size_t)blockIdx.x * C * HW;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < HW; i += kT) acc += fabsf(x[i]);  // signed (adjoint) maps: mean |a_0|
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int k = 0; k < kT / 32; ++k) s += red[k];
    const double m = s / (double)HW;
    scale[blockIdx.x] = (float)(1.0 / (m > 1e-30 ? m : 1e-30));
  }
}

// channel-major fp32 [B][C][HW] * scale[b] -> NHWC fp32 [B][HW][C]   (training targets)
__global__ void k_pack_target(const float *__restrict__ src, const float *__restrict__ scale, int HW, int C,
                              float *__restrict__ dst) {
  __shared__ float tile[32][33];
  const int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32, b = blockIdx.z;
  const float sc = scale[b];
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r, p = p0 + threadIdx.x;
    tile[r][threadIdx.x] = (c < C && p < HW) ? src[((size_t)b * C + c) * HW + p] * sc : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int p = p0 + r, c = c0 + threadIdx.x;
    if (p < HW && c < C) dst[((size_t)b * HW + p) * C + c] = tile[threadIdx.x][r];
  }
}

// prediction straight to channel-major maps: dst[b][c][p] = (x[b,p][c] + out[b,p][c]) / scale[b]
// (the residual output and the un-scaling in one pass through a 32 x 32 tile)
__global__ void k_predict_output(const float *__restrict__ out, int ostride, const __nv_bfloat16 *__restrict__ x,
                                 int xstride, const float *__restrict__ scale, int HW, int C, float *__restrict__ dst) {
  __shared__ float tile[32][33];
  const int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32, b = blockIdx.z;
  const float inv = 1.f / scale[b];
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int p = p0 + r, c = c0 + threadIdx.x;
    float v = 0.f;
    if (p < HW && c < C) {
      const size_t q = (size_t)b * HW + p;
      v = (bf(x[q * xstride + c]) + out[q * ostride + c]) * inv;
    }
    tile[r][threadIdx.x] = v;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r, p = p0 + threadIdx.x;
    if (c < C && p < HW) dst[((size_t)b * C + c) * HW + p] = tile[threadIdx.x][r];
  }
}

// NHWC fp32 [B][HW][C] / scale[b] -> channel-major fp32 [B][C][HW]
__global__ void k_unpack_output(const float *__restrict__ src, const float *__restrict__ scale, int HW, int C,
                                float *__restrict__ dst) {
  __shared__ float tile[32][33];
  const int p0 = blockIdx.x * 32, c0 = blockIdx.y * 32, b = blockIdx.z;
  const float sc = scale[b];
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int p = p0 + r, c = c0 + threadIdx.x;
    tile[r][threadIdx.x] = (p < HW && c < C) ? src[((size_t)b * HW + p) * C + c] / sc : 0.f;
  }
  __syncthreads();
  for (int r = threadIdx.y; r < 32; r += 8) {
    const int c = c0 + r, p = p0 + threadIdx.x;
    if (c < C && p < HW) dst[((size_t)b * C + c) * HW + p] = tile[threadIdx.x][r];
  }
}

}  // namespace

cudaError_t to_ct(const __nv_bfloat16 *src, int B, int HW, int W, int stride, int off, int C, int shifted,
                  __nv_bfloat16 *dst, cudaStream_t s) {
  const dim3 grid((HW + 31) / 32, (C + 31) / 32, B), block(32, 8);
  k_to_ct<<<grid, block, 0, s>>>(src, B, HW, W, stride, off, C, shifted, dst);
  return cudaGetLastError();
}
static dim3 pix_grid(int cols, int rows, int C) { return dim3((cols + 7) / 8, rows, (C + 31) / 32); }
static bool pix_grid_ok(int rows, int C) { return rows >= 1 && rows <= 65535 && (C + 31) / 32 <= 65535; }
static bool al8(int a, int b, int c, int d) { return a % 8 == 0 && b % 8 == 0 && c % 8 == 0 && d % 8 == 0; }
// block and grid of the 16-byte kernels: C/8 channel groups x enough pixels for ~256 threads
static dim3 v8_block(int G) {
  int py = 256 / G;
  return dim3(G, py < 1 ? 1 : (py > 64 ? 64 : py));
}
static dim3 v8_grid(int cols, int rows, dim3 blk) { return dim3((cols + blk.y - 1) / blk.y, rows); }

cudaError_t pool2(const __nv_bfloat16 *src, int B, int H, int W, int sstride, int soff, int C, __nv_bfloat16 *dst,
                  int dstride, int doff, cudaStream_t s) {
  if (!pix_grid_ok(B * (H / 2), C)) return cudaErrorInvalidConfiguration;
  if (al8(C, sstride, soff, dstride) && doff % 8 == 0 && C / 8 <= 256) {
    const dim3 blk = v8_block(C / 8);
    k_pool2_v8<<<v8_grid(W / 2, B * (H / 2), blk), blk, 0, s>>>(src, W, sstride, soff, C / 8, dst, dstride, doff);
    return cudaGetLastError();
  }
  k_pool2<<<pix_grid(W / 2, B * (H / 2), C), dim3(32, 8), 0, s>>>(src, W, sstride, soff, C, dst, dstride, doff);
  return cudaGetLastError();
}
cudaError_t pool2_bwd(const __nv_bfloat16 *dp, int pstride, int poff, const __nv_bfloat16 *skip, int kstride, int koff,
                      const __nv_bfloat16 *act, int astride, int aoff, int B, int H, int W, int C, __nv_bfloat16 *dz,
                      int zstride, int zoff, cudaStream_t s) {
  if (!pix_grid_ok(B * H, C)) return cudaErrorInvalidConfiguration;
  if (al8(C, pstride, poff, astride) && al8(aoff, zstride, zoff, 0) && (!skip || al8(kstride, koff, 0, 0)) &&
      C / 8 <= 256) {
    const dim3 blk = v8_block(C / 8);
    k_pool2_bwd_v8<<<v8_grid(W, B * H, blk), blk, 0, s>>>(dp, pstride, poff, skip, kstride, koff, act, astride, aoff,
                                                          W, C / 8, dz, zstride, zoff);
    return cudaGetLastError();
  }
  k_pool2_bwd<<<pix_grid(W, B * H, C), dim3(32, 8), 0, s>>>(dp, pstride, poff, skip, kstride, koff, act, astride, aoff,
                                                             W, C, dz, zstride, zoff);
  return cudaGetLastError();
}
cudaError_t up2(const __nv_bfloat16 *src, int B, int H, int W, int sstride, int soff, int C, __nv_bfloat16 *dst,
                int dstride, int doff, cudaStream_t s) {
  if (!pix_grid_ok(B * 2 * H, C)) return cudaErrorInvalidConfiguration;
  if (al8(C, sstride, soff, dstride) && doff % 8 == 0 && C / 8 <= 256) {
    const dim3 blk = v8_block(C / 8);
    k_up2_v8<<<v8_grid(2 * W, B * 2 * H, blk), blk, 0, s>>>(src, W, sstride, soff, C / 8, dst, dstride, doff);
    return cudaGetLastError();
  }
  k_up2<<<pix_grid(2 * W, B * 2 * H, C), dim3(32, 8), 0, s>>>(src, W, sstride, soff, C, dst, dstride, doff);
  return cudaGetLastError();
}
cudaError_t up2_bwd(const __nv_bfloat16 *du, int ustride, int uoff, const __nv_bfloat16 *act, int astride, int aoff,
                    int B, int H, int W, int C, __nv_bfloat16 *dz, int zstride, int zoff, cudaStream_t s) {
  if (!pix_grid_ok(B * H, C)) return cudaErrorInvalidConfiguration;
  if (al8(C, ustride, uoff, astride) && al8(aoff, zstride, zoff, 0) && C / 8 <= 256) {
    const dim3 blk = v8_block(C / 8);
    k_up2_bwd_v8<<<v8_grid(W, B * H, blk), blk, 0, s>>>(du, ustride, uoff, act, astride, aoff, W, C / 8, dz, zstride,
                                                        zoff);
    return cudaGetLastError();
  }
  k_up2_bwd<<<pix_grid(W, B * H, C), dim3(32, 8), 0, s>>>(du, ustride, uoff, act, astride, aoff, W, C, dz, zstride,
                                                           zoff);
  return cudaGetLastError();
}
cudaError_t bias_grad(const __nv_bfloat16 *dz, long long P, int stride, int off, int C, float *db, cudaStream_t s) {
  const int G = (C + 7) / 8;
  if (al8(stride, off, 0, 0) && G <= 256 && off + 8 * G <= stride && (reinterpret_cast<uintptr_t>(dz) & 15) == 0) {
    const int R = 256 / G;
    long long gx = (P + 4LL * R - 1) / (4LL * R);  // at least ~4 rows per thread
    if (gx > 152 * 8) gx = 152 * 8;
    k_bias_grad_v8<<<(unsigned)gx, 256, 0, s>>>(dz, P, stride, off, G, C, db);
    return cudaGetLastError();
  }
  long long gx = (P + 8 * 64 - 1) / (8 * 64);
  if (gx > 256) gx = 256;
  const dim3 grid((unsigned)gx, (C + 31) / 32), block(32, 8);
  k_bias_grad<<<grid, block, 0, s>>>(dz, P, stride, off, C, db);
  return cudaGetLastError();
}
cudaError_t mse(const float *out, int ostride, const __nv_bfloat16 *x, int xstride, const float *t, long long P, int C,
                __nv_bfloat16 *dout, int dstride, double *partials, int partials_cap, double *loss, cudaStream_t s) {
  const int cy = (C + 31) / 32;
  if (cy > partials_cap) return cudaErrorInvalidValue;
  long long gx = (P + 8 * 16 - 1) / (8 * 16);  // ~16 pixels per thread
  if (gx > partials_cap / cy) gx = partials_cap / cy;
  const double inv = 1.0 / ((double)P * C);
  k_mse<<<dim3((unsigned)gx, cy), dim3(32, 8), 0, s>>>(out, ostride, x, xstride, t, P, C, (float)(2.0 * inv), dout,
                                                        dstride, partials);
  k_sum_partials<<<1, kT, 0, s>>>(partials, (int)gx * cy, inv, loss);
  return cudaGetLastError();
}
cudaError_t sum_partials(const double *partials, int n, double scale, double *loss, cudaStream_t s) {
  k_sum_partials<<<1, kT, 0, s>>>(partials, n, scale, loss);
  return cudaGetLastError();
}
cudaError_t residual(const float *out, int ostride, const __nv_bfloat16 *x, int xstride, long long P, int C, float *y,
                     cudaStream_t s) {
  long long gx = (P + 8 * 16 - 1) / (8 * 16);
  if (gx > 65535) gx = 65535;
  k_residual<<<dim3((unsigned)gx, (C + 31) / 32), dim3(32, 8), 0, s>>>(out, ostride, x, xstride, P, C, y);
  return cudaGetLastError();
}
cudaError_t adam(float *w, float *m, float *v, float *g, int cout, int taps, int cin, float lr, float b1,
                 float b2, float eps, int step, __nv_bfloat16 *wf, int cin_pad, __nv_bfloat16 *wd, int cout_pad,
                 cudaStream_t s) {
  const float ic1 = step > 0 ? 1.f / (1.f - powf(b1, (float)step)) : 1.f, ic2 = step > 0 ? 1.f / (1.f - powf(b2, (float)step)) : 1.f;
  if (wd) {
    k_adam_t<<<dim3((cin + 31) / 32, (cout + 31) / 32, taps), dim3(32, 8), 0, s>>>(w, m, v, g, cout, taps, cin, lr, b1,
                                                                                  b2, eps, ic1, ic2, wf, cin_pad, wd,
                                                                                  cout_pad, step);
    return cudaGetLastError();
  }
  k_adam<<<blocks_for((long long)cout * taps * cin), kT, 0, s>>>(w, m, v, g, cout, taps, cin, lr, b1, b2, eps, ic1, ic2,
                                                                  wf, cin_pad, wd, cout_pad, step);
  return cudaGetLastError();
}
cudaError_t adam_multi(const AdamTable &T, float lr, float b1, float b2, float eps, int step, int blocks,
                       cudaStream_t s) {
  const float ic1 = step > 0 ? 1.f / (1.f - powf(b1, (float)step)) : 1.f, ic2 = step > 0 ? 1.f / (1.f - powf(b2, (float)step)) : 1.f;
  k_adam_multi<<<blocks, dim3(32, 8), 0, s>>>(T, lr, b1, b2, eps, ic1, ic2, step);
  return cudaGetLastError();
}
cudaError_t adam_bias(float *b, float *m, float *v, float *g, int n, float lr, float b1, float b2, float eps,
                      int step, cudaStream_t s) {
  if (step <= 0) return cudaSuccess;
  const float ic1 = 1.f / (1.f - powf(b1, (float)step)), ic2 = 1.f / (1.f - powf(b2, (float)step));
  k_adam_bias<<<(n + kT - 1) / kT, kT, 0, s>>>(b, m, v, g, n, lr, b1, b2, eps, ic1, ic2);
  return cudaGetLastError();
}
cudaError_t pack_input(const float *src, const float *scale, int B, long long HW, int C, __nv_bfloat16 *dst, int stride,
                       cudaStream_t s) {
  if (HW > 0x7fffffffll - 31 || B > 65535) return cudaErrorInvalidValue;
  if (HW % 64 == 0 && stride % 8 == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 &&
      (reinterpret_cast<uintptr_t>(src) & 7) == 0) {
    k_pack_input_v8<<<dim3((unsigned)(HW / 64), (C + 63) / 64, B), 256, 0, s>>>(src, scale, (int)HW, C, dst, stride);
    return cudaGetLastError();
  }
  k_pack_input<<<dim3((unsigned)((HW + 31) / 32), (C + 31) / 32, B), dim3(32, 8), 0, s>>>(src, scale, (int)HW, C, dst,
                                                                                         stride);
  return cudaGetLastError();
}
cudaError_t sample_scale(const float *src, int B, long long HW, int C, float *scale, cudaStream_t s) {
  k_sample_scale<<<B, kT, 0, s>>>(src, C, HW, scale);
  return cudaGetLastError();
}
cudaError_t pack_target(const float *src, const float *scale, int B, long long HW, int C, float *dst, cudaStream_t s) {
  if (HW > 0x7fffffffll - 31 || B > 65535) return cudaErrorInvalidValue;
  k_pack_target<<<dim3((unsigned)((HW + 31) / 32), (C + 31) / 32, B), dim3(32, 8), 0, s>>>(src, scale, (int)HW, C, dst);
  return cudaGetLastError();
}
cudaError_t predict_output(const float *out, int ostride, const __nv_bfloat16 *x, int xstride, const float *scale,
                           int B, long long HW, int C, float *dst, cudaStream_t s) {
  if (HW > 0x7fffffffll - 31 || B > 65535) return cudaErrorInvalidValue;
  k_predict_output<<<dim3((unsigned)((HW + 31) / 32), (C + 31) / 32, B), dim3(32, 8), 0, s>>>(out, ostride, x, xstride,
                                                                                             scale, (int)HW, C, dst);
  return cudaGetLastError();
}
cudaError_t unpack_output(const float *src, const float *scale, int B, long long HW, int C, float *dst,
                          cudaStream_t s) {
  if (HW > 0x7fffffffll - 31 || B > 65535) return cudaErrorInvalidValue;
  k_unpack_output<<<dim3((unsigned)((HW + 31) / 32), (C + 31) / 32, B), dim3(32, 8), 0, s>>>(src, scale, (int)HW, C,
                                                                                            dst);
  return cudaGetLastError();
}

}  // namespace dn
