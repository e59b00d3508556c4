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

// 2x2 average pooling: dst[b][y][x] = mean of src[b][2y..2y+1][2x..2x+1]
__global__ void k_pool2(const __nv_bfloat16 *__restrict__ src, int B, int H, int W, int sstride, int soff, int C,
                        __nv_bfloat16 *__restrict__ dst, int dstride, int doff) {
  const int Ho = H / 2, Wo = W / 2;
  const long long n = (long long)B * Ho * Wo * C;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const int c = (int)(i % C);
    long long q = i / C;
    const int x = (int)(q % Wo);
    q /= Wo;
    const int y = (int)(q % Ho);
    const int b = (int)(q / Ho);
    const size_t s00 = (((size_t)b * H + 2 * y) * W + 2 * x) * sstride + soff + c;
    const float v = 0.25f * (bf(src[s00]) + bf(src[s00 + sstride]) + bf(src[s00 + (size_t)W * sstride]) +
                             bf(src[s00 + (size_t)W * sstride + sstride]));
    dst[(((size_t)b * Ho + y) * Wo + x) * dstride + doff + c] = __float2bfloat16_rn(v);
  }
}

// backward of pool2 plus an optional skip gradient, times the ReLU mask of the pooled tensor:
// dz[b][y][x] = (skip[b][y][x] + dp[b][y/2][x/2] / 4) * (y_act[b][y][x] > 0)
__global__ void k_pool2_bwd(const __nv_bfloat16 *__restrict__ dp, int pstride, int poff,
                            const __nv_bfloat16 *__restrict__ skip, int kstride, int koff,
                            const __nv_bfloat16 *__restrict__ act, int astride, int aoff, int B, int H, int W, int C,
                            __nv_bfloat16 *__restrict__ dz, int zstride, int zoff) {
  const long long n = (long long)B * H * W * C;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const int c = (int)(i % C);
    long long q = i / C;
    const int x = (int)(q % W);
    q /= W;
    const int y = (int)(q % H);
    const int b = (int)(q / H);
    const size_t pix = ((size_t)b * H + y) * W + x;
    float g = 0.25f * bf(dp[(((size_t)b * (H / 2) + y / 2) * (W / 2) + x / 2) * pstride + poff + c]);
    if (skip) g += bf(skip[pix * kstride + koff + c]);
    if (!(bf(act[pix * astride + aoff + c]) > 0.f)) g = 0.f;
    dz[pix * zstride + zoff + c] = __float2bfloat16_rn(g);
  }
}

// nearest 2x up-sampling: dst[b][y][x] = src[b][y/2][x/2]   (src is H x W, dst 2H x 2W)
__global__ void k_up2(const __nv_bfloat16 *__restrict__ src, int B, int H, int W, int sstride, int soff, int C,
                      __nv_bfloat16 *__restrict__ dst, int dstride, int doff) {
  const long long n = (long long)B * 4 * H * W * C;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const int c = (int)(i % C);
    long long q = i / C;
    const int x = (int)(q % (2 * W));
    q /= 2 * W;
    const int y = (int)(q % (2 * H));
    const int b = (int)(q / (2 * H));
    dst[(((size_t)b * 2 * H + y) * 2 * W + x) * dstride + doff + c] =
        src[(((size_t)b * H + y / 2) * W + x / 2) * sstride + soff + c];
  }
}

// backward of up2 times the ReLU mask of its input: dz[b][y][x] = sum_2x2 du * (act > 0)
__global__ void k_up2_bwd(const __nv_bfloat16 *__restrict__ du, int ustride, int uoff,
                          const __nv_bfloat16 *__restrict__ act, int astride, int aoff, int B, int H, int W, int C,
                          __nv_bfloat16 *__restrict__ dz, int zstride, int zoff) {
  const long long n = (long long)B * H * W * C;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const int c = (int)(i % C);
    long long q = i / C;
    const int x = (int)(q % W);
    q /= W;
    const int y = (int)(q % H);
    const int b = (int)(q / H);
    const size_t u00 = (((size_t)b * 2 * H + 2 * y) * 2 * W + 2 * x) * ustride + uoff + c;
    float g = bf(du[u00]) + bf(du[u00 + ustride]) + bf(du[u00 + (size_t)2 * W * ustride]) +
              bf(du[u00 + (size_t)2 * W * ustride + ustride]);
    const size_t pix = ((size_t)b * H + y) * W + x;
    if (!(bf(act[pix * astride + aoff + c]) > 0.f)) g = 0.f;
    dz[pix * zstride + zoff + c] = __float2bfloat16_rn(g);
  }
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

// residual MSE: y = x + out over C channels; loss partials (FP64) and dout = 2 (y - t) / count
// written as bf16 NHWC (stride dstride) for the next convolution's input gradient.
__global__ void k_mse(const float *__restrict__ out, int ostride, const __nv_bfloat16 *__restrict__ x, int xstride,
                      const float *__restrict__ t, long long P, int C, double inv_count,
                      __nv_bfloat16 *__restrict__ dout, int dstride, double *__restrict__ partials) {
  __shared__ double red[kT / 32];
  double acc = 0.0;
  const long long n = P * C;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const long long p = i / C;
    const int c = (int)(i % C);
    const float y = bf(x[p * xstride + c]) + out[p * ostride + c];
    const double d = (double)y - (double)t[i];
    acc += d * d;
    dout[p * dstride + c] = __float2bfloat16_rn((float)(2.0 * d * inv_count));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xFFFFFFFFu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < kT / 32; ++w) s += red[w];
    partials[blockIdx.x] = s;
  }
}

__global__ void k_sum_partials(const double *__restrict__ partials, int n, double scale, double *out) {
  double s = 0.0;
  for (int i = 0; i < n; ++i) s += partials[i];
  *out = s * scale;
}

// prediction y = x + out (fp32 [P][C] from [P][ostride]); used at inference
__global__ void k_residual(const float *__restrict__ out, int ostride, const __nv_bfloat16 *__restrict__ x,
                           int xstride, long long P, int C, float *__restrict__ y) {
  const long long n = P * C;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const long long p = i / C;
    const int c = (int)(i % C);
    y[i] = bf(x[p * xstride + c]) + out[p * ostride + c];
  }
}

// Adam on the FP32 master weights [cout][taps][cin] and bias; writes the forward BF16 copy
// wf [n_pad][taps][cin_pad] and the input-gradient copy wd [cin_npad][taps][cout_pad] with the
// taps flipped (wd[c][8 - t][n] = w[n][t][c] for 3x3).
__global__ void k_adam(float *__restrict__ w, float *__restrict__ m, float *__restrict__ v,
                       float *__restrict__ g, int cout, int taps, int cin, float lr, float b1, float b2,
                       float eps, float c1, float c2, __nv_bfloat16 *__restrict__ wf, int cin_pad,
                       __nv_bfloat16 *__restrict__ wd, int cout_pad, int step) {
  const long long n = (long long)cout * taps * cin;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    float wi = w[i];
    if (step > 0) {
      const float gi = g[i];
      g[i] = 0.f;  // the gradient is consumed: the next backward pass accumulates from zero
      const float mi = b1 * m[i] + (1.f - b1) * gi;
      const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
      m[i] = mi;
      v[i] = vi;
      wi -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
      w[i] = wi;
    }
    const int c = (int)(i % cin);
    const int t = (int)((i / cin) % taps);
    const int o = (int)(i / ((long long)cin * taps));
    const __nv_bfloat16 h = __float2bfloat16_rn(wi);
    wf[((size_t)o * taps + t) * cin_pad + c] = h;
    if (wd) wd[((size_t)c * taps + (taps - 1 - t)) * cout_pad + o] = h;
  }
}

__global__ void k_adam_bias(float *__restrict__ b, float *__restrict__ m, float *__restrict__ v,
                            float *__restrict__ g, int n, float lr, float b1, float b2, float eps, float c1,
                            float c2) {
  const int i = blockIdx.x * kT + threadIdx.x;
  if (i >= n) return;
  const float gi = g[i];
  g[i] = 0.f;
  const float mi = b1 * m[i] + (1.f - b1) * gi;
  const float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  b[i] -= lr * (mi / c1) / (sqrtf(vi / c2) + eps);
}

// channel-major fp32 coefficient maps [B][C][HW] * scale[b] -> NHWC bf16 [B][HW][stride]
__global__ void k_pack_input(const float *__restrict__ src, const float *__restrict__ scale, int B, long long HW,
                             int C, __nv_bfloat16 *__restrict__ dst, int stride) {
  const long long n = (long long)B * HW * C;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const long long p = q % HW;
    const int b = (int)(q / HW);
    dst[((size_t)b * HW + p) * stride + c] = __float2bfloat16_rn(src[((size_t)b * C + c) * HW + p] * scale[b]);
  }
}

// per-sample input scale 1 / mean(channel 0) of channel-major fp32 maps [B][C][HW] (the fluence
// a_0 of a harmonic map), one block per sample, FP64 sum in a fixed order
__global__ void k_sample_scale(const float *__restrict__ src, int C, long long HW, float *__restrict__ scale) {
  __shared__ double red[kT / 32];
  const float *x = src + (size_t)blockIdx.x * C * HW;
  double acc = 0.0;
  for (long long i = threadIdx.x; i < HW; i += kT) acc += x[i];
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
__global__ void k_pack_target(const float *__restrict__ src, const float *__restrict__ scale, int B, long long HW,
                              int C, float *__restrict__ dst) {
  const long long n = (long long)B * HW * C;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const long long p = q % HW;
    const int b = (int)(q / HW);
    dst[i] = src[((size_t)b * C + c) * HW + p] * scale[b];
  }
}

// NHWC fp32 [B][HW][C] / scale[b] -> channel-major fp32 [B][C][HW]
__global__ void k_unpack_output(const float *__restrict__ src, const float *__restrict__ scale, int B, long long HW,
                                int C, float *__restrict__ dst) {
  const long long n = (long long)B * HW * C;
  for (long long i = blockIdx.x * (long long)kT + threadIdx.x; i < n; i += (long long)gridDim.x * kT) {
    const int c = (int)(i % C);
    const long long q = i / C;
    const long long p = q % HW;
    const int b = (int)(q / HW);
    dst[((size_t)b * C + c) * HW + p] = src[i] / scale[b];
  }
}

}  // namespace

cudaError_t to_ct(const __nv_bfloat16 *src, int B, int HW, int W, int stride, int off, int C, int shifted,
                  __nv_bfloat16 *dst, cudaStream_t s) {
  const dim3 grid((HW + 31) / 32, (C + 31) / 32, B), block(32, 8);
  k_to_ct<<<grid, block, 0, s>>>(src, B, HW, W, stride, off, C, shifted, dst);
  return cudaGetLastError();
}
cudaError_t pool2(const __nv_bfloat16 *src, int B, int H, int W, int sstride, int soff, int C, __nv_bfloat16 *dst,
                  int dstride, int doff, cudaStream_t s) {
  k_pool2<<<blocks_for((long long)B * H * W * C / 4), kT, 0, s>>>(src, B, H, W, sstride, soff, C, dst, dstride, doff);
  return cudaGetLastError();
}
cudaError_t pool2_bwd(const __nv_bfloat16 *dp, int pstride, int poff, const __nv_bfloat16 *skip, int kstride, int koff,
                      const __nv_bfloat16 *act, int astride, int aoff, int B, int H, int W, int C, __nv_bfloat16 *dz,
                      int zstride, int zoff, cudaStream_t s) {
  k_pool2_bwd<<<blocks_for((long long)B * H * W * C), kT, 0, s>>>(dp, pstride, poff, skip, kstride, koff, act, astride,
                                                                   aoff, B, H, W, C, dz, zstride, zoff);
  return cudaGetLastError();
}
cudaError_t up2(const __nv_bfloat16 *src, int B, int H, int W, int sstride, int soff, int C, __nv_bfloat16 *dst,
                int dstride, int doff, cudaStream_t s) {
  k_up2<<<blocks_for((long long)B * 4 * H * W * C), kT, 0, s>>>(src, B, H, W, sstride, soff, C, dst, dstride, doff);
  return cudaGetLastError();
}
cudaError_t up2_bwd(const __nv_bfloat16 *du, int ustride, int uoff, const __nv_bfloat16 *act, int astride, int aoff,
                    int B, int H, int W, int C, __nv_bfloat16 *dz, int zstride, int zoff, cudaStream_t s) {
  k_up2_bwd<<<blocks_for((long long)B * H * W * C), kT, 0, s>>>(du, ustride, uoff, act, astride, aoff, B, H, W, C, dz,
                                                                 zstride, zoff);
  return cudaGetLastError();
}
cudaError_t bias_grad(const __nv_bfloat16 *dz, long long P, int stride, int off, int C, float *db, cudaStream_t s) {
  long long gx = (P + 8 * 64 - 1) / (8 * 64);
  if (gx > 256) gx = 256;
  const dim3 grid((unsigned)gx, (C + 31) / 32), block(32, 8);
  k_bias_grad<<<grid, block, 0, s>>>(dz, P, stride, off, C, db);
  return cudaGetLastError();
}
cudaError_t mse(const float *out, int ostride, const __nv_bfloat16 *x, int xstride, const float *t, long long P, int C,
                __nv_bfloat16 *dout, int dstride, double *partials, int partials_cap, double *loss, cudaStream_t s) {
  int grid = blocks_for(P * C);
  if (grid > partials_cap) grid = partials_cap;
  const double inv = 1.0 / ((double)P * C);
  k_mse<<<grid, kT, 0, s>>>(out, ostride, x, xstride, t, P, C, inv, dout, dstride, partials);
  k_sum_partials<<<1, 1, 0, s>>>(partials, grid, inv, loss);
  return cudaGetLastError();
}
cudaError_t residual(const float *out, int ostride, const __nv_bfloat16 *x, int xstride, long long P, int C, float *y,
                     cudaStream_t s) {
  k_residual<<<blocks_for(P * C), kT, 0, s>>>(out, ostride, x, xstride, P, C, y);
  return cudaGetLastError();
}
cudaError_t adam(float *w, float *m, float *v, float *g, int cout, int taps, int cin, float lr, float b1,
                 float b2, float eps, int step, __nv_bfloat16 *wf, int cin_pad, __nv_bfloat16 *wd, int cout_pad,
                 cudaStream_t s) {
  const float c1 = step > 0 ? 1.f - powf(b1, (float)step) : 1.f, c2 = step > 0 ? 1.f - powf(b2, (float)step) : 1.f;
  k_adam<<<blocks_for((long long)cout * taps * cin), kT, 0, s>>>(w, m, v, g, cout, taps, cin, lr, b1, b2, eps, c1, c2,
                                                                  wf, cin_pad, wd, cout_pad, step);
  return cudaGetLastError();
}
cudaError_t adam_bias(float *b, float *m, float *v, float *g, int n, float lr, float b1, float b2, float eps,
                      int step, cudaStream_t s) {
  if (step <= 0) return cudaSuccess;
  const float c1 = 1.f - powf(b1, (float)step), c2 = 1.f - powf(b2, (float)step);
  k_adam_bias<<<(n + kT - 1) / kT, kT, 0, s>>>(b, m, v, g, n, lr, b1, b2, eps, c1, c2);
  return cudaGetLastError();
}
cudaError_t pack_input(const float *src, const float *scale, int B, long long HW, int C, __nv_bfloat16 *dst, int stride,
                       cudaStream_t s) {
  k_pack_input<<<blocks_for((long long)B * HW * C), kT, 0, s>>>(src, scale, B, HW, C, dst, stride);
  return cudaGetLastError();
}
cudaError_t sample_scale(const float *src, int B, long long HW, int C, float *scale, cudaStream_t s) {
  k_sample_scale<<<B, kT, 0, s>>>(src, C, HW, scale);
  return cudaGetLastError();
}
cudaError_t pack_target(const float *src, const float *scale, int B, long long HW, int C, float *dst, cudaStream_t s) {
  k_pack_target<<<blocks_for((long long)B * HW * C), kT, 0, s>>>(src, scale, B, HW, C, dst);
  return cudaGetLastError();
}
cudaError_t unpack_output(const float *src, const float *scale, int B, long long HW, int C, float *dst,
                          cudaStream_t s) {
  k_unpack_output<<<blocks_for((long long)B * HW * C), kT, 0, s>>>(src, scale, B, HW, C, dst);
  return cudaGetLastError();
}

}  // namespace dn
