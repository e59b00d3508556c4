// dn_conv.cu -- BF16 tensor-core convolutions of the harmonic-map denoiser on sm_103a.
//
// k_conv_ws: 3x3 (pad 1) or 1x1 convolution as an implicit GEMM, D[pixels x Cout] =
// sum over taps and 64-channel blocks of X_tap[pixels x 64] * W_tap[Cout x 64]^T, with
//   * activations NHWC bf16 with the channel stride padded to a multiple of 64; a 128-pixel tile
//     (one row segment, or several short rows) of one tap is one 4D TMA box {64 ch, w, rows, 1};
//     the shifted boxes of the taps start at x-1 / y-1 and the hardware fills the padding with
//     zeros;
//   * weights [Cout_pad][taps][Cin_pad] bf16, one 2D TMA box {64, N} per K block;
//   * operands in shared memory with the 128-byte swizzle, a TMA -> MMA mbarrier ring,
//     tcgen05.mma (M = 128, N = Cout_pad, K = 16 per instruction) issued by one thread with the
//     FP32 accumulator in TMEM (two accumulators, so a tile's epilogue overlaps the next tile's
//     MMAs in the persistent kernel);
//   * an epilogue that reads TMEM with tcgen05.ld and applies bias, ReLU, or the ReLU mask of the
//     next layer's input (for the backward pass), writing bf16 or fp32 NHWC slices (channel
//     offset/stride, so concatenations are free).
#include <cuda_bf16.h>

#include "dn_internal.h"
#include "dn_sm100.cuh"

namespace dn {
namespace {

constexpr int kStages = 4;
constexpr int kBlockM = 128;
constexpr int kBlockK = 64;
constexpr uint32_t kATileBytes = kBlockM * kBlockK * 2;  // 16 KB

// 16 floats of one row as bf16: two 16-byte stores when all 16 lie below `valid` (16-byte
// aligned rows), else element stores of the first `valid`.
__device__ __forceinline__ void store_bf16x16(__nv_bfloat16 *o, int valid, const float *f) {
  if (valid >= 16) {
    __align__(16) __nv_bfloat162 h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
    *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(&h[0]);
    *reinterpret_cast<uint4 *>(o + 8) = *reinterpret_cast<const uint4 *>(&h[4]);
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < valid) o[j] = __float2bfloat16_rn(f[j]);
  }
}

// 16 bf16 values of one row as floats: two 16-byte loads when the row is 16-byte aligned and all
// 16 lie below `valid`, else element loads of the first `valid` (the rest read as 0).
__device__ __forceinline__ void load_bf16x16(const __nv_bfloat16 *p, bool vec, int valid, float *f) {
  if (vec && valid >= 16) {
    const uint4 u0 = __ldg(reinterpret_cast<const uint4 *>(p));
    const uint4 u1 = __ldg(reinterpret_cast<const uint4 *>(p + 8));
    const __nv_bfloat162 *h0 = reinterpret_cast<const __nv_bfloat162 *>(&u0);
    const __nv_bfloat162 *h1 = reinterpret_cast<const __nv_bfloat162 *>(&u1);
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const float2 a = __bfloat1622float2(h0[j]), b = __bfloat1622float2(h1[j]);
      f[2 * j] = a.x;
      f[2 * j + 1] = a.y;
      f[8 + 2 * j] = b.x;
      f[8 + 2 * j + 1] = b.y;
    }
  } else {
#pragma unroll
    for (int j = 0; j < 16; ++j) f[j] = j < valid ? __bfloat162float(p[j]) : 0.f;
  }
}

// Fused output head on 16 output channels c0.. of pixel p (image bi, pixel pi of it), f = the
// layer's output (accumulator + bias).  Prediction: pred[bi][c][pi] = (x0 + f) / scale; loss:
// r = x0 + f - scale * target[bi][c][pi], dout = bf16(2 r / count), returns the sum of r^2.  The
// channel-major reads and writes are coalesced: the lanes of a warp hold consecutive pixels.
__device__ __forceinline__ double head_chunk(const ConvArgs &a, long long p, long long bi, long long pi, float hs,
                                             int c0, int valid, const float *f) {
  float xv[16];
  load_bf16x16(a.res + p * a.res_stride + c0, true, valid, xv);
  if (a.head == 1) {
    float *o = a.pred + (bi * a.cout + c0) * a.HW + pi;
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < valid) o[(long long)j * a.HW] = (xv[j] + f[j]) * hs;
    return 0.0;
  }
  const float *t = a.target + (bi * a.cout + c0) * a.HW + pi;
  float g[16], sq = 0.f;
#pragma unroll
  for (int j = 0; j < 16; ++j) {
    g[j] = 0.f;
    if (j < valid) {
      // the scaled target rounded on its own, as a stored scaled copy would be
      const float r = xv[j] + f[j] - __fmul_rn(t[(long long)j * a.HW], hs);
      sq = __fmaf_rn(r, r, sq);
      g[j] = r * a.two_over_count;
    }
  }
  const double ss = (double)sq;  // FP32 within 16 channels, FP64 across them
  __nv_bfloat16 *o = a.dout + p * a.dout_stride + c0;
  if (valid >= 16) {
    __align__(16) __nv_bfloat162 h[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(g[2 * j], g[2 * j + 1]);
    *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(&h[0]);
    *reinterpret_cast<uint4 *>(o + 8) = *reinterpret_cast<const uint4 *>(&h[4]);
  } else {
    for (int j = 0; j < valid; ++j) o[j] = __float2bfloat16_rn(g[j]);
  }
  return ss;
}

// 16 bf16 of one row as raw 16-byte words (two loads when 16-byte aligned and all 16 lie below
// `valid`, else element loads of the first `valid`, the rest 0), converted after the TMEM wait so
// that the global loads of a row are all in flight while its accumulator is read.
union Raw16 {
  uint4 u[2];
  __nv_bfloat16 h[16];
};
__device__ __forceinline__ void load_raw16(const __nv_bfloat16 *p, bool vec, int valid, Raw16 &r) {
  if (vec && valid >= 16) {
    r.u[0] = __ldg(reinterpret_cast<const uint4 *>(p));
    r.u[1] = __ldg(reinterpret_cast<const uint4 *>(p + 8));
  } else {
    r.u[0] = make_uint4(0u, 0u, 0u, 0u);
    r.u[1] = r.u[0];
#pragma unroll
    for (int j = 0; j < 16; ++j)
      if (j < valid) r.h[j] = p[j];
  }
}
__device__ __forceinline__ void unpack16(const Raw16 &r, float *f) {
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(r.u);
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const float2 v = __bfloat1622float2(h[j]);
    f[2 * j] = v.x;
    f[2 * j + 1] = v.y;
  }
}

// Epilogue of 16 NCH columns c0b.. of one row: every global load (the ReLU mask, or the head's
// residual input and target) is issued first, then the TMEM loads and one wait, then the
// arithmetic and stores -- one memory latency per 16 NCH columns instead of one per 16.  HEAD:
// the fused output head (a.head != 0), else the plain epilogue.
template <int NCH, bool HEAD>
__device__ __forceinline__ double drain_row_t(const ConvArgs &a, long long p, uint32_t trow, int c0b) {
  long long bi = 0, pi = 0;
  float hs = 0.f;
  if (HEAD) {
    bi = p / a.HW;
    pi = p - bi * a.HW;
    hs = a.head == 1 ? 1.f / __ldg(a.scale + bi) : __ldg(a.scale + bi);
  }
  Raw16 raw[NCH];  // mask rows, or the head's residual input rows
  float tv[HEAD ? NCH : 1][16];
#pragma unroll
  for (int k = 0; k < NCH; ++k) {
    const int c0 = c0b + 16 * k, valid = a.cout - c0;
    if (HEAD) {
      load_raw16(a.res + p * a.res_stride + c0, true, valid, raw[k]);
      if (a.head == 2) {
        const float *t = a.target + (bi * a.cout + c0) * a.HW + pi;
#pragma unroll
        for (int j = 0; j < 16; ++j) tv[HEAD ? k : 0][j] = j < valid ? __ldg(t + (long long)j * a.HW) : 0.f;
      }
    } else if (a.mask) {
      load_raw16(a.mask + p * a.mask_stride + a.mask_off + c0, a.mask_vec != 0, valid, raw[k]);
    }
  }
  uint32_t v[NCH][16];
#pragma unroll
  for (int k = 0; k < NCH; ++k) {
    // only the accumulator's own N columns (N is a multiple of 16; warp-uniform test)
    if (c0b + 16 * k < a.N) tmem_ld16(trow + (uint32_t)(c0b + 16 * k), v[k]);
    else
#pragma unroll
      for (int j = 0; j < 16; ++j) v[k][j] = 0u;
  }
  tmem_ld_wait();
  double ss = 0.0;
#pragma unroll
  for (int k = 0; k < NCH; ++k) {
    const int c0 = c0b + 16 * k, valid = a.cout - c0;
    if (valid <= 0) break;
    float f[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      float x = __uint_as_float(v[k][j]);
      if (a.bias && j < valid) x += __ldg(a.bias + c0 + j);
      if (a.relu) x = fmaxf(x, 0.f);
      f[j] = x;
    }
    if (HEAD) {
      float xv[16];
      unpack16(raw[k], xv);
      if (a.head == 1) {
        float *o = a.pred + (bi * a.cout + c0) * a.HW + pi;
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (j < valid) o[(long long)j * a.HW] = (xv[j] + f[j]) * hs;
      } else {
        float g[16], sq = 0.f;
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          g[j] = 0.f;
          if (j < valid) {
            // the scaled target rounded on its own, as a stored scaled copy would be
            const float r = xv[j] + f[j] - __fmul_rn(tv[HEAD ? k : 0][j], hs);
            sq = __fmaf_rn(r, r, sq);
            g[j] = r * a.two_over_count;
          }
        }
        ss += (double)sq;  // FP32 within 16 channels, FP64 across them (FP64 is a slow pipe here)
        store_bf16x16(a.dout + p * a.dout_stride + c0, valid, g);
      }
      continue;
    }
    if (a.mask) {
      float mk[16];
      unpack16(raw[k], mk);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (j < valid) f[j] = mk[j] > 0.f ? f[j] : 0.f;
    }
    if (a.out_f32) {
      float *o = a.out_f32 + p * a.out_stride + a.out_off + c0;
      if (valid >= 16) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4 *>(o + j) = make_float4(f[j], f[j + 1], f[j + 2], f[j + 3]);
      } else {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (j < valid) o[j] = f[j];
      }
    } else {
      store_bf16x16(a.out_bf16 + p * a.out_stride + a.out_off + c0, valid, f);
    }
  }
  return ss;
}

// Epilogue of one output pixel p (this thread's TMEM lane, row address trow): N accumulator
// columns through bias / ReLU / the next layer's ReLU mask into the bf16 or fp32 output slice,
// or through the fused output head.  Returns the head's sum of squared residuals (else 0).
__device__ __forceinline__ double drain_row_any(const ConvArgs &a, long long p, uint32_t trow) {
  double ss = 0.0;
  long long bi = 0, pi = 0;
  float hs = 0.f;
  if (a.head) {
    bi = p / a.HW;
    pi = p - bi * a.HW;
    hs = a.head == 1 ? 1.f / a.scale[bi] : a.scale[bi];
  }
  for (int c0 = 0; c0 < a.N; c0 += 16) {
    uint32_t v[16];
    tmem_ld16(trow + (uint32_t)c0, v);
    tmem_ld_wait();
    const int valid = a.cout - c0;
    float mk[16];
    if (a.mask) load_bf16x16(a.mask + p * a.mask_stride + a.mask_off + c0, a.mask_vec != 0, valid, mk);
    float f[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
      const int n = c0 + j;
      float x = __uint_as_float(v[j]);
      if (a.bias && n < a.cout) x += a.bias[n];
      if (a.relu) x = fmaxf(x, 0.f);
      if (a.mask && n < a.cout) x = mk[j] > 0.f ? x : 0.f;
      f[j] = x;
    }
    if (a.head) {
      if (valid > 0) ss += head_chunk(a, p, bi, pi, hs, c0, valid, f);
      continue;
    }
    if (a.out_f32) {
      float *o = a.out_f32 + p * a.out_stride + a.out_off + c0;
      if (c0 + 16 <= a.cout) {
#pragma unroll
        for (int j = 0; j < 16; j += 4)
          *reinterpret_cast<float4 *>(o + j) = make_float4(f[j], f[j + 1], f[j + 2], f[j + 3]);
      } else {
        for (int j = 0; j < 16 && c0 + j < a.cout; ++j) o[j] = f[j];
      }
    } else {
      __nv_bfloat16 *o = a.out_bf16 + p * a.out_stride + a.out_off + c0;
      if (c0 + 16 <= a.cout) {
        __align__(16) __nv_bfloat162 h[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) h[j] = __floats2bfloat162_rn(f[2 * j], f[2 * j + 1]);
        *reinterpret_cast<uint4 *>(o) = *reinterpret_cast<const uint4 *>(&h[0]);
        *reinterpret_cast<uint4 *>(o + 8) = *reinterpret_cast<const uint4 *>(&h[4]);
      } else {
        for (int j = 0; j < 16 && c0 + j < a.cout; ++j) o[j] = __float2bfloat16_rn(f[j]);
      }
    }
  }
  return ss;
}

template <bool HEAD>
__device__ __forceinline__ double drain_row(const ConvArgs &a, long long p, uint32_t trow) {
  if (HEAD) return a.N == 48 ? drain_row_t<3, true>(a, p, trow, 0) : drain_row_any(a, p, trow);
  for (int c0 = 0; c0 < a.N; c0 += 32) drain_row_t<2, false>(a, p, trow, c0);
  return 0.0;
}

// one sum of squared residuals per epilogue warp (fused loss head), in a fixed order
__device__ __forceinline__ void head_partial(const ConvArgs &a, double ss, int e, int epi_warps, int lane) {
  if (a.head != 2) return;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) ss += __shfl_xor_sync(0xffffffffu, ss, o);
  if (lane == 0) a.partials[blockIdx.x * epi_warps + e] = ss;
}

// k_conv_ws: persistent, warp-specialised.  One CTA per SM
// walks the output tiles (tile = blockIdx.x + i gridDim.x); warp 0 streams the K blocks of all
// its tiles through a ring of `stages` shared-memory buffers with TMA, warp 1 issues the MMAs
// into one of two TMEM accumulators (2 x acc_cols columns), and warps 2..5 drain the other
// accumulator (TMEM lanes 32 (w % 4) ... + 31) while the next tile is being multiplied.
// SUB = 2 (N <= 128): a tile is 2 x 128 pixels whose two A tiles share one weight tile per
// stage (two MMAs per K step into the two halves of the accumulator, acc_cols / 2 >= N columns
// apart), which halves the weight bytes each output pixel pulls through L2; warps 2..9 drain
// it, warps 2..5 the first half and 6..9 the second (each warp its TMEM lane quarter w % 4).
constexpr int kWsThreads = 192;
template <int SUB>
constexpr int ws_threads() { return 64 + 128 * SUB; }

template <int SUB, bool HEAD>
__global__ void __launch_bounds__(ws_threads<SUB>(), 1)
    k_conv_ws(const __grid_constant__ CUtensorMap tmX, const __grid_constant__ CUtensorMap tmW, const ConvArgs a,
              int stages, int num_tiles) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t bTileBytes = (uint32_t)a.N * kBlockK * 2;
  const uint32_t stageBytes = SUB * kATileBytes + bTileBytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(smem + (size_t)stages * stageBytes);
  uint64_t *empty = full + stages;
  uint64_t *tfull = empty + stages;   // [2] accumulator b is ready for the epilogue
  uint64_t *tempty = tfull + 2;       // [2] accumulator b has been drained
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(tempty + 2);
  const uint32_t acc_cols = a.tmem_cols;  // columns of one accumulator

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&tfull[b], 1);
      mbar_init(&tempty[b], 128 * SUB);
    }
    fence_barrier_init();
    prefetch_tensormap(&tmX);
    prefetch_tensormap(&tmW);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 2 * acc_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int hw = a.H * a.W;
  const int cblocks = a.cin_pad / kBlockK;
  const int nk = a.taps * cblocks;

  if (warp == 0 && lane == 0) {
    // ---- TMA producer over all tiles of this CTA
    uint32_t kc = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      int b0[SUB], y0[SUB], x0[SUB];
#pragma unroll
      for (int u = 0; u < SUB; ++u) {
        const long long p0 = ((long long)tile * SUB + u) * kBlockM;
        b0[u] = (int)(p0 / hw);
        const int rem = (int)(p0 % hw);
        y0[u] = rem / a.W;
        x0[u] = rem % a.W;
      }
      for (int i = 0; i < nk; ++i, ++kc) {
        const int s = kc % stages;
        const uint32_t r = kc / stages;
        if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1)) {
          atomicOr(a.err, 64u);
          ok = false;
          break;
        }
        const int tap = i / cblocks, cb = i % cblocks;
        const int ky = a.taps == 9 ? tap / 3 : 1, kx = a.taps == 9 ? tap % 3 : 1;
        uint8_t *st = smem + (size_t)s * stageBytes;
        mbar_arrive_expect_tx(&full[s], stageBytes);
#pragma unroll
        for (int u = 0; u < SUB; ++u)
          tma_load_4d(st + u * kATileBytes, &tmX, &full[s], cb * kBlockK, x0[u] + kx - 1, y0[u] + ky - 1, b0[u]);
        tma_load_2d(st + SUB * kATileBytes, &tmW, &full[s], tap * a.cin_pad + cb * kBlockK, 0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    // ---- MMA issuer
    const uint32_t idesc = idesc_bf16_f32(kBlockM, (uint32_t)a.N);
    uint32_t kc = 0;
    int it = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x, ++it) {
      const int b = it & 1;
      const uint32_t use = it >> 1;
      if (use > 0 && !mbar_wait(&tempty[b], (use - 1) & 1)) {
        atomicOr(a.err, 128u);
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + b * acc_cols;
      for (int i = 0; i < nk; ++i, ++kc) {
        const int s = kc % stages;
        if (!mbar_wait(&full[s], (kc / stages) & 1)) {
          atomicOr(a.err, 256u);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t aBase = smem_u32(smem + (size_t)s * stageBytes), bBase = aBase + SUB * kATileBytes;
#pragma unroll
        for (int kk = 0; kk < kBlockK / 16; ++kk) {
          const uint64_t bdesc = sdesc_k128(bBase + kk * 32);
#pragma unroll
          for (int u = 0; u < SUB; ++u)
            mma_bf16(d + u * (acc_cols / 2), sdesc_k128(aBase + u * kATileBytes + kk * 32), bdesc, idesc,
                     (i > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&empty[s]);
      }
      mma_commit(&tfull[b]);
    }
  } else if (warp >= 2) {
    // ---- epilogue warps: TMEM lanes 32 (warp % 4) .. + 31 of sub-tile (warp - 2) / 4
    const int e = warp - 2, q = warp & 3, u = e >> 2;
    const int row = q * 32 + lane;
    int it = 0;
    double ss = 0.0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++it) {
      const int b = it & 1;
      const uint32_t use = it >> 1;
      // warp-uniform decision: the TMEM loads below are warp-collective
      const bool have = __all_sync(0xffffffffu, mbar_wait(&tfull[b], use & 1));
      if (!have) {
        if (lane == 0) atomicOr(a.err, 512u);
        break;
      }
      tc_fence_after();
      ss += drain_row<HEAD>(a, ((long long)tile * SUB + u) * kBlockM + row,
                      tmem + ((uint32_t)(q * 32) << 16) + b * acc_cols + u * (acc_cols / 2));
      tc_fence_before();
      mbar_arrive(&tempty[b]);
    }
    head_partial(a, ss, e, 4 * SUB, lane);
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * acc_cols);
}

// k_conv_halo: 3x3 convolution with few output channels (N <= 32) whose 128-pixel tiles lie in
// one image row (W a multiple of 128).  The weights of all taps and channel blocks (9 x cblocks
// tiles of N x 64, <= 74 KB) are loaded once per CTA and stay resident; a ring stage holds, for
// one 64-channel block, the haloed input -- rows y-1..y+1 x columns x0-1..x0+128, one 4D TMA box
// {64, 130, 3, 1} with zero fill -- and the nine taps read it at row offsets ky 130 + kx (the
// descriptor starts at that row, base-offset field 0: the 128-byte swizzle follows the address
// bits of the 1024-byte-aligned tile).  Per stage that is 36 MMAs for one barrier round trip and
// 50 KB through L2 per 128 pixels and channel block (a box per tap plus its weights would be
// 9 x (16 + N/8) KB), which is what bounds these convolutions.  Same warp roles and double TMEM
// accumulator as k_conv_ws.
// KB = 32: layers whose input has at most 32 real channels (in a 64-channel row) read only those
// 32: 64-byte rows with the 64-byte swizzle, half the MMAs and operand bytes of KB = 64.
template <int KB>
__host__ __device__ constexpr uint32_t halo_bytes() { return 3u * 130u * KB * 2u; }  // written by the input box
template <int KB>
__host__ __device__ constexpr uint32_t halo_stride() { return (halo_bytes<KB>() + 1023u) & ~1023u; }
template <int KB>
__device__ __forceinline__ uint64_t sdesc_kb(uint32_t addr) { return KB == 64 ? sdesc_k128(addr) : sdesc_k64(addr); }

template <int KB>
__global__ void __launch_bounds__(kWsThreads, 1)
    k_conv_halo(const __grid_constant__ CUtensorMap tmH, const __grid_constant__ CUtensorMap tmW, const ConvArgs a,
                int stages, int num_tiles) {
  static_assert(KB == 64 || KB == 32, "channel block of 64 (128-byte rows) or 32 (64-byte rows)");
  constexpr uint32_t kHaloBytes = halo_bytes<KB>(), kHaloStride = halo_stride<KB>();
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int cblocks = KB == 64 ? a.cin_pad / 64 : 1;
  const uint32_t bTileBytes = (uint32_t)a.N * KB * 2;      // one tap's weights, one channel block
  const uint32_t wBytes = (uint32_t)cblocks * 9u * bTileBytes;  // resident weights [cb][tap]
  uint8_t *ring = smem + wBytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(ring + (size_t)stages * kHaloStride);
  uint64_t *empty = full + stages;
  uint64_t *tfull = empty + stages;
  uint64_t *tempty = tfull + 2;
  uint64_t *wfull = tempty + 2;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(wfull + 1);
  const uint32_t acc_cols = a.tmem_cols;

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (tid == 0) {
    for (int i = 0; i < stages; ++i) {
      mbar_init(&full[i], 1);
      mbar_init(&empty[i], 1);
    }
    for (int i = 0; i < 2; ++i) {
      mbar_init(&tfull[i], 1);
      mbar_init(&tempty[i], 128);
    }
    mbar_init(wfull, 1);
    fence_barrier_init();
    prefetch_tensormap(&tmH);
    prefetch_tensormap(&tmW);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 2 * acc_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;
  const int hw = a.H * a.W;

  if (warp == 0 && lane == 0) {
    // the weights once, then the haloed input boxes of all tiles of this CTA
    mbar_arrive_expect_tx(wfull, wBytes);
    for (int cb = 0; cb < cblocks; ++cb)
      for (int tap = 0; tap < 9; ++tap)
        tma_load_2d(smem + (cb * 9 + tap) * bTileBytes, &tmW, wfull, tap * a.cin_pad + cb * KB, 0);
    uint32_t kc = 0;
    bool ok = true;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x) {
      const long long p0 = (long long)tile * kBlockM;
      const int b0 = (int)(p0 / hw), rem = (int)(p0 % hw);
      const int y0 = rem / a.W, x0 = rem % a.W;
      for (int cb = 0; cb < cblocks; ++cb, ++kc) {
        const int st = kc % stages;
        const uint32_t r = kc / stages;
        if (r > 0 && !mbar_wait(&empty[st], (r - 1) & 1)) {
          atomicOr(a.err, 1024u);
          ok = false;
          break;
        }
        mbar_arrive_expect_tx(&full[st], kHaloBytes);
        tma_load_4d(ring + (size_t)st * kHaloStride, &tmH, &full[st], cb * KB, x0 - 1, y0 - 1, b0);
      }
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16_f32(kBlockM, (uint32_t)a.N);
    const uint32_t wBase = smem_u32(smem);
    bool ok = mbar_wait(wfull, 0);
    if (!ok) atomicOr(a.err, 2048u);
    uint32_t kc = 0;
    int it = 0;
    for (int tile = blockIdx.x; tile < num_tiles && ok; tile += gridDim.x, ++it) {
      const int b = it & 1;
      const uint32_t use = it >> 1;
      if (use > 0 && !mbar_wait(&tempty[b], (use - 1) & 1)) {
        atomicOr(a.err, 2048u);
        break;
      }
      tc_fence_after();
      const uint32_t d = tmem + b * acc_cols;
      for (int cb = 0; cb < cblocks; ++cb, ++kc) {
        const int st = kc % stages;
        if (!mbar_wait(&full[st], (kc / stages) & 1)) {
          atomicOr(a.err, 2048u);
          ok = false;
          break;
        }
        tc_fence_after();
        const uint32_t aBase = smem_u32(ring + (size_t)st * kHaloStride);
        const uint32_t bBase = wBase + (uint32_t)cb * 9u * bTileBytes;
        for (int tap = 0; tap < 9; ++tap) {
          const uint32_t arow = aBase + (uint32_t)((tap / 3) * 130 + tap % 3) * (KB * 2u);
#pragma unroll
          for (int kk = 0; kk < KB / 16; ++kk)
            mma_bf16(d, sdesc_kb<KB>(arow + kk * 32), sdesc_kb<KB>(bBase + tap * bTileBytes + kk * 32), idesc,
                     (cb > 0 || tap > 0 || kk > 0) ? 1u : 0u);
        }
        mma_commit(&empty[st]);
      }
      mma_commit(&tfull[b]);
    }
  } else if (warp >= 2) {
    const int q = warp & 3;
    const int row = q * 32 + lane;
    int it = 0;
    for (int tile = blockIdx.x; tile < num_tiles; tile += gridDim.x, ++it) {
      const int b = it & 1;
      const uint32_t use = it >> 1;
      const bool have = __all_sync(0xffffffffu, mbar_wait(&tfull[b], use & 1));
      if (!have) {
        if (lane == 0) atomicOr(a.err, 4096u);
        break;
      }
      tc_fence_after();
      drain_row<false>(a, (long long)tile * kBlockM + row, tmem + ((uint32_t)(q * 32) << 16) + b * acc_cols);
      tc_fence_before();
      mbar_arrive(&tempty[b]);
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 2 * acc_cols);
}

// k_wgrad_tc: weight gradient dW[n][tap][c] += sum_p dZ[p][n] X[p + tap][c] as a GEMM over pixels
// with M = 128 output channels, N = `N` input channels, K = 64-pixel blocks.  Operands are
// K-major (pixels contiguous): dZ^T [cout][B][HW] and three x-shifted copies
// X^T_kx [cin][B][HW] (X^T_kx[c][b][y W + x] = X[b][y][x + kx - 1][c], zero outside the row).
// The y shift of a tap is a TMA coordinate offset of (ky - 1) W pixels inside one image (zero
// filled outside it), which keeps every box start 16-byte aligned.  Each CTA sums a contiguous
// range of K blocks for one tap and one (M, N) tile and adds its partial tile to dW (FP32).
__global__ void __launch_bounds__(128, 1)
    k_wgrad_tc(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB0,
               const __grid_constant__ CUtensorMap tmB1, const __grid_constant__ CUtensorMap tmB2, const WgradArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const uint32_t bTileBytes = (uint32_t)a.N * kBlockK * 2;
  uint8_t *tileA = smem;
  uint8_t *tileB = smem + kStages * kATileBytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(tileB + kStages * bTileBytes);
  uint64_t *empty = full + kStages;
  uint64_t *done = empty + kStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x, tap = blockIdx.y;
  const int m_tile = blockIdx.z % a.m_tiles, n_tile = blockIdx.z / a.m_tiles;
  const int ky = a.taps == 9 ? tap / 3 : 1, kx = a.taps == 9 ? tap % 3 : 1;
  const CUtensorMap *tmB = kx == 0 ? &tmB0 : (kx == 1 ? &tmB1 : &tmB2);
  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
    prefetch_tensormap(&tmA);
    prefetch_tensormap(tmB);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  // this CTA's K blocks: [k_begin, k_end) of B * HW / 64 blocks (image-major)
  const int blocks_per_image = a.HW / kBlockK;
  const int total = a.B * blocks_per_image;
  const int k_begin = (int)((long long)total * split / a.splits);
  const int k_end = (int)((long long)total * (split + 1) / a.splits);
  const int nk = k_end - k_begin;
  const int dy = (ky - 1) * a.W;

  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nk; ++i) {
      const int s = i % kStages, r = i / kStages;
      if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1)) {
        atomicOr(a.err, 8u);
        break;
      }
      const int kb = k_begin + i;
      const int b = kb / blocks_per_image, pix = (kb % blocks_per_image) * kBlockK;
      mbar_arrive_expect_tx(&full[s], kATileBytes + bTileBytes);
      tma_load_3d(tileA + s * kATileBytes, &tmA, &full[s], pix, b, m_tile * kBlockM);
      tma_load_3d(tileB + s * bTileBytes, tmB, &full[s], pix + dy, b, n_tile * a.N);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16_f32(kBlockM, (uint32_t)a.N);
    for (int i = 0; i < nk; ++i) {
      const int s = i % kStages, r = i / kStages;
      if (!mbar_wait(&full[s], r & 1)) {
        atomicOr(a.err, 16u);
        break;
      }
      tc_fence_after();
      const uint32_t aBase = smem_u32(tileA + s * kATileBytes), bBase = smem_u32(tileB + s * bTileBytes);
#pragma unroll
      for (int kk = 0; kk < kBlockK / 16; ++kk)
        mma_bf16(tmem, sdesc_k128(aBase + kk * 32), sdesc_k128(bBase + kk * 32), idesc, (i > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();

  const bool have = nk > 0 && mbar_wait(done, 0);
  if (nk > 0 && !have && tid == 0) atomicOr(a.err, 32u);
  tc_fence_after();
  const int m = m_tile * kBlockM + warp * 32 + lane;  // output channel of this thread's row
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  for (int c0 = 0; c0 < a.N; c0 += 16) {
    uint32_t v[16];
    tmem_ld16(trow + (uint32_t)c0, v);
    tmem_ld_wait();
    if (!have || m >= a.cout) continue;
    float *o = a.dw + ((size_t)m * a.taps + tap) * a.cin_pad + n_tile * a.N + c0;
    const int cb = n_tile * a.N + c0;
    if (a.cin_pad % 4 == 0 && cb + 16 <= a.cin) {  // 16-byte aligned: four 4-wide reductions
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        red_add_v4(o + j, __uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                   __uint_as_float(v[j + 3]));
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (cb + j < a.cin) atomicAdd(o + j, __uint_as_float(v[j]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

// k_wgrad_mn: the same weight gradient read straight from the NHWC activations, with both
// operands MN-major (channels contiguous, pixels = K rows): A = dZ [pixels][cout] in 2D boxes of
// 64 channels x 64 pixels, B = X [b][y][x][cin] in 4D boxes of 64 channels x a 64-pixel block,
// the tap's shift applied as TMA coordinates (x + kx - 1, y + ky - 1) with hardware zero fill at
// the image border -- no transposed or shifted copies.  A 128-byte-swizzled MN-major operand of
// M (or N) = 64 j channels is j boxes 8 KB apart (leading byte offset 8 KB), 8-pixel groups
// 1 KB apart (stride byte offset), and each K = 16 step advances 16 pixel rows (2 KB).
// Ring depth: 4 stages of 24 KB (N <= 64) or 3 of 32 KB, so that two blocks fit on an SM (an
// 8-deep ring at one block per SM was 20 % slower on 32 -> 32 channels at 8 x 256^2); the host
// sizes the split count for one wave of two blocks per SM.
static int wgrad_mn_stages(int N) { return N <= 64 ? 4 : 3; }

__global__ void __launch_bounds__(128, 1)
    k_wgrad_mn(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, const WgradArgs a,
               int stages) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  const int nb = (a.N + 63) / 64;  // 64-channel B boxes per stage (the MMA uses the first N)
  const uint32_t bTileBytes = (uint32_t)nb * 8192u;
  uint8_t *tileA = smem;
  uint8_t *tileB = smem + stages * kATileBytes;
  uint64_t *full = reinterpret_cast<uint64_t *>(tileB + stages * bTileBytes);
  uint64_t *empty = full + stages;
  uint64_t *done = empty + stages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x, tap = blockIdx.y;
  const int m_tile = blockIdx.z % a.m_tiles, n_tile = blockIdx.z / a.m_tiles;
  const int ky = a.taps == 9 ? tap / 3 : 1, kx = a.taps == 9 ? tap % 3 : 1;
  if (tid == 0) {
    for (int s = 0; s < stages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
    prefetch_tensormap(&tmA);
    prefetch_tensormap(&tmB);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, a.tmem_cols);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int blocks_per_image = a.HW / kBlockK;
  const int total = a.B * blocks_per_image;
  const int k_begin = (int)((long long)total * split / a.splits);
  const int k_end = (int)((long long)total * (split + 1) / a.splits);
  const int nk = k_end - k_begin;

  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nk; ++i) {
      const int s = i % stages, r = i / stages;
      if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1)) {
        atomicOr(a.err, 8u);
        break;
      }
      const int kb = k_begin + i;
      const int b = kb / blocks_per_image, p = (kb % blocks_per_image) * kBlockK;  // first pixel in image b
      const int y0 = p / a.W, x0 = p % a.W;
      mbar_arrive_expect_tx(&full[s], kATileBytes + bTileBytes);
      uint8_t *sa = tileA + s * kATileBytes, *sb = tileB + s * bTileBytes;
      const int pg = b * a.HW + p;  // pixel index in the flattened dZ
      tma_load_2d(sa, &tmA, &full[s], m_tile * kBlockM, pg);
      tma_load_2d(sa + 8192, &tmA, &full[s], m_tile * kBlockM + 64, pg);
      for (int j = 0; j < nb; ++j)
        tma_load_4d(sb + j * 8192, &tmB, &full[s], n_tile * a.N + 64 * j, x0 + kx - 1, y0 + ky - 1, b);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16_f32(kBlockM, (uint32_t)a.N) | (1u << 15) | (1u << 16);  // A, B MN-major
    for (int i = 0; i < nk; ++i) {
      const int s = i % stages, r = i / stages;
      if (!mbar_wait(&full[s], r & 1)) {
        atomicOr(a.err, 16u);
        break;
      }
      tc_fence_after();
      const uint32_t aBase = smem_u32(tileA + s * kATileBytes), bBase = smem_u32(tileB + s * bTileBytes);
#pragma unroll
      for (int kk = 0; kk < kBlockK / 16; ++kk)
        mma_bf16(tmem, sdesc_mn128(aBase + kk * 2048), sdesc_mn128(bBase + kk * 2048), idesc,
                 (i > 0 || kk > 0) ? 1u : 0u);
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();

  const bool have = nk > 0 && __all_sync(0xffffffffu, mbar_wait(done, 0));
  if (nk > 0 && !have && tid == 0) atomicOr(a.err, 32u);
  tc_fence_after();
  const int m = m_tile * kBlockM + warp * 32 + lane;  // output channel of this thread's row
  const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16);
  for (int c0 = 0; c0 < a.N; c0 += 16) {
    uint32_t v[16];
    tmem_ld16(trow + (uint32_t)c0, v);
    tmem_ld_wait();
    if (!have || m >= a.cout) continue;
    float *o = a.dw + ((size_t)m * a.taps + tap) * a.cin_pad + n_tile * a.N + c0;
    const int cb = n_tile * a.N + c0;
    if (a.cin_pad % 4 == 0 && cb + 16 <= a.cin) {  // 16-byte aligned: four 4-wide reductions
#pragma unroll
      for (int j = 0; j < 16; j += 4)
        red_add_v4(o + j, __uint_as_float(v[j]), __uint_as_float(v[j + 1]), __uint_as_float(v[j + 2]),
                   __uint_as_float(v[j + 3]));
    } else {
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (cb + j < a.cin) atomicAdd(o + j, __uint_as_float(v[j]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, a.tmem_cols);
}

// k_wgrad_halo: weight gradient of a 3x3 layer with cout <= 64 on rows of whole 64-pixel
// segments, all nine taps from one haloed input box per segment:
//   D[(tap, c)][o] = sum_p X[p + d_tap][c] dZ[p][o],
// M = 128 = two taps x 64 input channels (of channel block blockIdx.y), N = 64 (cout, zero
// filled), K = 64-pixel row segments in 16-pixel steps.  A stage holds the haloed box of X
// (channels of the block, columns x0-1 .. x0+64, rows y-1 .. y+1; zero fill outside the image)
// and the dZ box {64 channels, 64 pixels}.  Tap (ky, kx)'s window starts ky 66 + kx pixel rows
// into the box; an MMA's second 64-channel M group is the next tap's window (leading byte offset =
// the distance of the two windows).  Tap 8's partner is a 16-row block of ones in shared memory,
// so those 64 accumulator rows hold sum_p dZ[p][o]: the bias gradient comes free with the
// weight gradient.  Five accumulators of 64 columns (taps 0-1, 2-3, 4-5, 6-7, 8 + ones) stay in
// TMEM for the CTA's contiguous range of segments; the epilogue adds them into dw with one atomic
// per element (consecutive lanes = consecutive input channels) and, on channel block 0, the
// ones row into db.  Per segment the CTA reads 25 KB of
// X and 8 KB of dZ instead of 9 x (8 + 8) KB for nine separate shifted GEMMs.
constexpr uint32_t kWhBytes = 3 * 66 * 128;                          // 25,344 B written by the box
constexpr uint32_t kWhStride = (kWhBytes + 1023) & ~1023u;           // 25,600 B
constexpr uint32_t kWhStage = kWhStride + 8192;                      // + dZ box
constexpr int kWhStages = 4;
constexpr uint32_t kWhOnes = 2048;  // 16 rows x 64 bf16 ones (tap 8's partner M group)

__global__ void __launch_bounds__(128, 1)
    k_wgrad_halo(const __grid_constant__ CUtensorMap tmZ, const __grid_constant__ CUtensorMap tmH, const WgradArgs a) {
  extern __shared__ __align__(1024) uint8_t smem_raw[];
  uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
  uint8_t *ones = smem + kWhStages * kWhStage;
  uint64_t *full = reinterpret_cast<uint64_t *>(ones + kWhOnes);
  uint64_t *empty = full + kWhStages;
  uint64_t *done = empty + kWhStages;
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(done + 1);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int split = blockIdx.x, cb = blockIdx.y;
  for (int i = tid; i < (int)(kWhOnes / 4); i += blockDim.x)
    reinterpret_cast<uint32_t *>(ones)[i] = 0x3F803F80u;  // bf16 1.0 pairs (any swizzle of it is the same)
  fence_proxy_async_smem();
  if (tid == 0) {
    for (int s = 0; s < kWhStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&empty[s], 1);
    }
    mbar_init(done, 1);
    fence_barrier_init();
    prefetch_tensormap(&tmZ);
    prefetch_tensormap(&tmH);
  }
  if (warp == 0) {
    tmem_alloc(tmem_slot, 512);
    tmem_relinquish();
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot;

  const int segs_per_image = a.HW / 64, segs_per_row = a.W / 64;
  const int total = a.B * segs_per_image;
  const int k_begin = (int)((long long)total * split / a.splits);
  const int k_end = (int)((long long)total * (split + 1) / a.splits);
  const int nk = k_end - k_begin;

  if (warp == 0 && lane == 0) {
    for (int i = 0; i < nk; ++i) {
      const int s = i % kWhStages, r = i / kWhStages;
      if (r > 0 && !mbar_wait(&empty[s], (r - 1) & 1)) {
        atomicOr(a.err, 8192u);
        break;
      }
      const int kb = k_begin + i;
      const int b = kb / segs_per_image, sg = kb % segs_per_image;
      const int y0 = sg / segs_per_row, x0 = (sg % segs_per_row) * 64;
      uint8_t *st = smem + (size_t)s * kWhStage;
      mbar_arrive_expect_tx(&full[s], kWhBytes + 8192u);
      tma_load_4d(st, &tmH, &full[s], cb * 64, x0 - 1, y0 - 1, b);
      tma_load_2d(st + kWhStride, &tmZ, &full[s], 0, b * a.HW + sg * 64);
    }
  } else if (warp == 1 && lane == 0) {
    const uint32_t idesc = idesc_bf16_f32(kBlockM, 64) | (1u << 15) | (1u << 16);  // A, B MN-major
    const uint32_t onesBase = smem_u32(ones);
    for (int i = 0; i < nk; ++i) {
      const int s = i % kWhStages, r = i / kWhStages;
      if (!mbar_wait(&full[s], r & 1)) {
        atomicOr(a.err, 16384u);
        break;
      }
      tc_fence_after();
      const uint32_t hBase = smem_u32(smem + (size_t)s * kWhStage), zBase = hBase + kWhStride;
#pragma unroll
      for (int ks = 0; ks < 4; ++ks) {
        const uint64_t bdesc = sdesc_mn128(zBase + ks * 2048);
#pragma unroll
        for (int mt = 0; mt < 5; ++mt) {
          const int t0 = 2 * mt;
          const uint32_t r0 = (uint32_t)((t0 / 3) * 66 + t0 % 3);
          const uint32_t a0 = hBase + (r0 + 16 * ks) * 128;
          // partner group: the next tap's window, or for tap 8 the ones block (above every stage)
          const uint32_t lbo = t0 < 8 ? (uint32_t)(((t0 + 1) / 3) * 66 + (t0 + 1) % 3 - r0) * 128 : onesBase - a0;
          mma_bf16(tmem + mt * 64, sdesc_mn128_lbo(a0, lbo), bdesc, idesc, (i > 0 || ks > 0) ? 1u : 0u);
        }
      }
      mma_commit(&empty[s]);
    }
    mma_commit(done);
  }
  __syncwarp();

  const bool have = nk > 0 && __all_sync(0xffffffffu, mbar_wait(done, 0));
  if (nk > 0 && !have && tid == 0) atomicOr(a.err, 32768u);
  tc_fence_after();
  const int mrow = warp * 32 + lane;  // M row of this thread: tap offset mrow / 64, channel mrow % 64
  const int c = cb * 64 + (mrow & 63);
  for (int mt = 0; mt < 5; ++mt) {
    const int tap = 2 * mt + (mrow >> 6);
    const uint32_t trow = tmem + ((uint32_t)(warp * 32) << 16) + mt * 64;
    for (int c0 = 0; c0 < a.cout; c0 += 16) {
      uint32_t v[16];
      tmem_ld16(trow + (uint32_t)c0, v);
      tmem_ld_wait();
      if (have && tap == 9 && mrow == 64 && cb == 0 && a.db) {  // the ones row: sum_p dZ[p][o]
#pragma unroll
        for (int j = 0; j < 16; ++j)
          if (c0 + j < a.cout) atomicAdd(a.db + c0 + j, __uint_as_float(v[j]));
      }
      if (!have || tap > 8 || c >= a.cin) continue;
      float *o = a.dw + (size_t)tap * a.cin_pad + c;
#pragma unroll
      for (int j = 0; j < 16; ++j)
        if (c0 + j < a.cout) atomicAdd(o + (size_t)(c0 + j) * 9 * a.cin_pad, __uint_as_float(v[j]));
    }
  }
  tc_fence_before();
  __syncthreads();
  if (warp == 0) tmem_dealloc(tmem, 512);
}

}  // namespace

cudaError_t launch_wgrad_tc(const CUtensorMap &tmA, const CUtensorMap tmB[3], const WgradArgs &a, cudaStream_t s) {
  const size_t smem = 1024 + kStages * (kATileBytes + (size_t)a.N * kBlockK * 2) + 256;
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  const dim3 grid((unsigned)a.splits, (unsigned)a.taps, (unsigned)(a.m_tiles * a.n_tiles));
  k_wgrad_tc<<<grid, 128, smem, s>>>(tmA, tmB[0], tmB[1], tmB[2], a);
  return cudaGetLastError();
}

// Ring depth of the persistent convolution: as many stages as fit in ~200 KB of shared memory,
// at most 8.
static int conv_stages(int N, int sub) {
  const size_t stage = sub * kATileBytes + (size_t)N * kBlockK * 2;
  int s = (int)((200u * 1024u) / stage);
  return s > 8 ? 8 : (s < 2 ? 2 : s);
}

static size_t conv_smem(int N, int sub) {
  return 1024 + conv_stages(N, sub) * (sub * kATileBytes + (size_t)N * kBlockK * 2) + 256;
}

static int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
  }
  return n;
}

template <int SUB, bool HEAD>
static cudaError_t launch_ws(const CUtensorMap &tmX, const CUtensorMap &tmW, ConvArgs a, cudaStream_t s,
                             int *partials_out) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_ws<SUB, HEAD>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  uint32_t cols = 32;  // one accumulator: SUB x N columns, a power of two
  while (cols < (uint32_t)(SUB * a.N)) cols <<= 1;
  a.tmem_cols = cols;
  const long long tiles = (long long)a.B * a.H * a.W / (kBlockM * SUB);
  const int grid = (int)(tiles < sm_count() ? tiles : sm_count());
  if (partials_out) *partials_out = grid * 4 * SUB;
  k_conv_ws<SUB, HEAD><<<grid, ws_threads<SUB>(), conv_smem(a.N, SUB), s>>>(tmX, tmW, a, conv_stages(a.N, SUB),
                                                                            (int)tiles);
  return cudaGetLastError();
}

cudaError_t launch_conv_tc(const CUtensorMap &tmX, const CUtensorMap &tmW, const ConvArgs &a, cudaStream_t s,
                           int *partials_out) {
  const long long P = (long long)a.B * a.H * a.W;
  // two 128-pixel tiles per weight stage when two accumulators of N columns, double-buffered,
  // fit in the 512 TMEM columns and the pixels split into 256-pixel tiles
  const bool pair = a.N <= 128 && P % (2 * kBlockM) == 0;
  if (a.head) return pair ? launch_ws<2, true>(tmX, tmW, a, s, partials_out) : launch_ws<1, true>(tmX, tmW, a, s, partials_out);
  return pair ? launch_ws<2, false>(tmX, tmW, a, s, partials_out) : launch_ws<1, false>(tmX, tmW, a, s, partials_out);
}

cudaError_t launch_wgrad_mn(const CUtensorMap &tmA, const CUtensorMap &tmB, const WgradArgs &a, cudaStream_t s) {
  const int st = wgrad_mn_stages(a.N);
  const size_t smem = 1024 + st * (kATileBytes + (size_t)((a.N + 63) / 64) * 8192) + 256;
  static size_t configured = 0;
  if (smem > configured) {
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_mn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = smem;
  }
  const dim3 grid((unsigned)a.splits, (unsigned)a.taps, (unsigned)(a.m_tiles * a.n_tiles));
  k_wgrad_mn<<<grid, 128, smem, s>>>(tmA, tmB, a, st);
  return cudaGetLastError();
}

// ring depth of k_conv_halo beside its resident weights (cblocks x 9 x N x KB x 2 B), at most 4
static int halo_stages(int N, int cblocks, int kb) {
  const long long stride = kb == 64 ? halo_stride<64>() : halo_stride<32>();
  const long long avail = 232448 - 1024 - 512 - (long long)cblocks * 9 * N * kb * 2;
  const long long st = avail / stride;
  return st > 4 ? 4 : (st < 0 ? 0 : (int)st);
}

bool conv_halo_applies(const ConvArgs &a) {
  return a.taps == 9 && a.W % kBlockM == 0 && a.N <= 32 && halo_stages(a.N, a.cin_pad / kBlockK, 64) >= 2;
}

template <int KB>
static cudaError_t launch_halo_kb(const CUtensorMap &tmH, const CUtensorMap &tmW, ConvArgs a, cudaStream_t s) {
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_conv_halo<KB>, cudaFuncAttributeMaxDynamicSharedMemorySize, 232448);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  uint32_t cols = 32;
  while (cols < (uint32_t)a.N) cols <<= 1;
  a.tmem_cols = cols;
  const int cblocks = KB == 64 ? a.cin_pad / kBlockK : 1;
  const int st = halo_stages(a.N, cblocks, KB);
  if (st < 2) return cudaErrorInvalidValue;
  const size_t smem = 1024 + (size_t)cblocks * 9 * a.N * KB * 2 + (size_t)st * halo_stride<KB>() + 512;
  const long long tiles = (long long)a.B * a.H * a.W / kBlockM;
  const int grid = (int)(tiles < sm_count() ? tiles : sm_count());
  k_conv_halo<KB><<<grid, kWsThreads, smem, s>>>(tmH, tmW, a, st, (int)tiles);
  return cudaGetLastError();
}

cudaError_t launch_conv_halo(const CUtensorMap &tmH, const CUtensorMap &tmW, ConvArgs a, cudaStream_t s, int kb) {
  return kb == 32 ? launch_halo_kb<32>(tmH, tmW, a, s) : launch_halo_kb<64>(tmH, tmW, a, s);
}

bool wgrad_halo_applies(int taps, int cout, int W) { return taps == 9 && cout <= 64 && W % 64 == 0; }

cudaError_t launch_wgrad_halo(const CUtensorMap &tmZ, const CUtensorMap &tmH, const WgradArgs &a, cudaStream_t s) {
  const size_t smem = 1024 + kWhStages * (size_t)kWhStage + kWhOnes + 256;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(k_wgrad_halo, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const int cblocks = (a.cin + 63) / 64;
  k_wgrad_halo<<<dim3((unsigned)a.splits, (unsigned)cblocks), 128, smem, s>>>(tmZ, tmH, a);
  return cudaGetLastError();
}

// ---------------------------------------------------------------- bounded-wait test hook
namespace {
__global__ void k_wait_probe(unsigned *err, uint32_t spins, int *timed_out) {
  __shared__ __align__(8) uint64_t bar;
  if (threadIdx.x == 0) mbar_init(&bar, 1);  // one arrival expected; none will come
  fence_barrier_init();
  __syncwarp();
  const bool done = mbar_wait(&bar, 0, spins);
  if (threadIdx.x == 0) {
    if (!done) atomicOr(err, 64u);
    *timed_out = done ? 0 : 1;
  }
}
}  // namespace

cudaError_t launch_wait_probe(unsigned *err, uint32_t spins, int *timed_out, cudaStream_t s) {
  k_wait_probe<<<1, 32, 0, s>>>(err, spins, timed_out);
  return cudaGetLastError();
}

}  // namespace dn
