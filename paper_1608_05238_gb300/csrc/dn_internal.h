// dn_internal.h -- declarations shared by the denoiser translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dn {

// Implicit-GEMM convolution launch arguments (see k_conv_ws).
struct ConvArgs {
  int B, H, W;       // images and spatial size (output = input size)
  int cin_pad;       // channel stride of the input (multiple of 64)
  int taps;          // 9 (3x3, pad 1) or 1 (1x1)
  int N;             // MMA N = padded output channels (multiple of 16, 16..256)
  int cout;          // output channels written (<= N)
  uint32_t tmem_cols;  // TMEM columns allocated (power of two >= max(32, N))
  const float *bias;   // [cout] or null
  int relu;            // apply ReLU after the bias
  const __nv_bfloat16 *mask;  // if set: zero outputs where mask[p * mask_stride + mask_off + n] <= 0
  int mask_stride, mask_off;
  __nv_bfloat16 *out_bf16;  // one of out_bf16 / out_f32
  float *out_f32;
  int out_stride, out_off;  // channel stride and offset of the output slice
  unsigned *err;            // device error word (bounded waits that gave up)
  int mask_vec;             // mask rows 16-byte aligned (stride and offset multiples of 8): vector loads
  // fused output head of a 1x1 output layer (k_conv_ws only; out_bf16 / out_f32 unused when set)
  int head;                   // 0 none, 1 prediction, 2 residual MSE loss and its gradient
  const __nv_bfloat16 *res;   // residual input x0: NHWC bf16, channel stride res_stride (multiple of 8)
  int res_stride;
  const float *scale;         // [B] per-sample input scale
  int HW;                     // pixels per image
  float *pred;                // head 1: [B][cout][HW] = (x0 + out) / scale
  const float *target;        // head 2: [B][cout][HW], unscaled
  __nv_bfloat16 *dout;        // head 2: NHWC bf16 2 (x0 + out - scale target) / count, stride dout_stride
  int dout_stride;
  float two_over_count;
  double *partials;           // head 2: one sum of squares per (block, epilogue warp)
};

// partials_out (optional): the number of partial sums the fused loss head writes (one per epilogue warp)
cudaError_t launch_conv_tc(const CUtensorMap &tmX, const CUtensorMap &tmW, const ConvArgs &a, cudaStream_t s,
                           int *partials_out = nullptr);
// 3x3 convolution with N <= 32 on rows of whole 128-pixel tiles: one haloed input box {64, 130, 3, 1}
// and all nine taps' weights per channel block
bool conv_halo_applies(const ConvArgs &a);
// kb = 64: channel blocks of 64 (box {64, 130, 3, 1}, 128-byte swizzle); kb = 32: only the first 32
// channels of each row (box {32, 130, 3, 1} and weight box {32, N}, 64-byte swizzle)
cudaError_t launch_conv_halo(const CUtensorMap &tmH, const CUtensorMap &tmW, ConvArgs a, cudaStream_t s, int kb);

// Weight-gradient GEMM launch arguments (see k_wgrad_tc).
struct WgradArgs {
  int B, HW, W;      // images, pixels per image, row length (for the y shift)
  int taps;          // 9 or 1
  int cout, cin;     // real channel counts
  int cin_pad;       // dW row length per tap
  int N;             // input channels per CTA tile (multiple of 16, <= 256)
  int m_tiles, n_tiles, splits;
  uint32_t tmem_cols;
  float *dw;         // fp32 [n_pad][taps][cin_pad], accumulated with atomics
  unsigned *err;
  float *db;         // k_wgrad_halo: if set, db[o] += sum_p dZ[p][o] (the bias gradient), else unused
};
cudaError_t launch_wgrad_tc(const CUtensorMap &tmA, const CUtensorMap tmB[3], const WgradArgs &a, cudaStream_t s);
cudaError_t launch_wgrad_mn(const CUtensorMap &tmA, const CUtensorMap &tmB, const WgradArgs &a, cudaStream_t s);
// 3x3 weight gradient with cout <= 64 on rows of 64-pixel segments: one haloed X box {64, 66, 3, 1}
// per segment serves all nine taps (grid: splits x 64-channel blocks of cin; one block per SM)
bool wgrad_halo_applies(int taps, int cout, int W);
cudaError_t launch_wgrad_halo(const CUtensorMap &tmZ, const CUtensorMap &tmH, const WgradArgs &a, cudaStream_t s);

// Test hook (dn_conv.cu): one warp waits, with the kernels' own bounded mbarrier wait limited to
// `spins` polls, on an mbarrier that nothing arrives at; on the timeout it latches the kernels'
// wait-failure bit (64) in err and writes 1 to *timed_out (else 0).  Nothing is in flight.
cudaError_t launch_wait_probe(unsigned *err, uint32_t spins, int *timed_out, cudaStream_t s);

// memory-bound kernels (dn_ops.cu)
cudaError_t to_ct(const __nv_bfloat16 *src, int B, int HW, int W, int stride, int off, int C, int shifted,
                  __nv_bfloat16 *dst, cudaStream_t s);
cudaError_t pool2(const __nv_bfloat16 *src, int B, int H, int W, int sstride, int soff, int C, __nv_bfloat16 *dst,
                  int dstride, int doff, cudaStream_t s);
cudaError_t pool2_bwd(const __nv_bfloat16 *dp, int pstride, int poff, const __nv_bfloat16 *skip, int kstride, int koff,
                      const __nv_bfloat16 *act, int astride, int aoff, int B, int H, int W, int C, __nv_bfloat16 *dz,
                      int zstride, int zoff, cudaStream_t s);
cudaError_t up2(const __nv_bfloat16 *src, int B, int H, int W, int sstride, int soff, int C, __nv_bfloat16 *dst,
                int dstride, int doff, cudaStream_t s);
cudaError_t up2_bwd(const __nv_bfloat16 *du, int ustride, int uoff, const __nv_bfloat16 *act, int astride, int aoff,
                    int B, int H, int W, int C, __nv_bfloat16 *dz, int zstride, int zoff, cudaStream_t s);
cudaError_t bias_grad(const __nv_bfloat16 *dz, long long P, int stride, int off, int C, float *db, cudaStream_t s);
// One layer of a multi-tensor Adam step (k_adam_multi): tile0 = its first block.
struct AdamLayer {
  float *w, *m, *v, *g;
  __nv_bfloat16 *wf, *wd;
  float *b, *mb, *vb, *gb;
  int cout, taps, cin, cin_pad, cout_pad;
  int tile0;
};
constexpr int kMaxAdamLayers = 32;
struct AdamTable {
  AdamLayer L[kMaxAdamLayers];
  int n;
};
cudaError_t adam_multi(const AdamTable &T, float lr, float b1, float b2, float eps, int step, int blocks,
                       cudaStream_t s);
// loss = scale * (sum of partials[0..n)) in one block, fixed order
cudaError_t sum_partials(const double *partials, int n, double scale, double *loss, cudaStream_t s);
cudaError_t mse(const float *out, int ostride, const __nv_bfloat16 *x, int xstride, const float *t, long long P, int C,
                __nv_bfloat16 *dout, int dstride, double *partials, int partials_cap, double *loss, cudaStream_t s);
cudaError_t residual(const float *out, int ostride, const __nv_bfloat16 *x, int xstride, long long P, int C, float *y,
                     cudaStream_t s);
cudaError_t adam(float *w, float *m, float *v, float *g, int cout, int taps, int cin, float lr, float b1,
                 float b2, float eps, int step, __nv_bfloat16 *wf, int cin_pad, __nv_bfloat16 *wd, int cout_pad,
                 cudaStream_t s);
cudaError_t adam_bias(float *b, float *m, float *v, float *g, int n, float lr, float b1, float b2, float eps,
                      int step, cudaStream_t s);
cudaError_t pack_input(const float *src, const float *scale, int B, long long HW, int C, __nv_bfloat16 *dst, int stride,
                       cudaStream_t s);
cudaError_t sample_scale(const float *src, int B, long long HW, int C, float *scale, cudaStream_t s);
cudaError_t pack_target(const float *src, const float *scale, int B, long long HW, int C, float *dst, cudaStream_t s);
cudaError_t predict_output(const float *out, int ostride, const __nv_bfloat16 *x, int xstride, const float *scale,
                           int B, long long HW, int C, float *dst, cudaStream_t s);
cudaError_t unpack_output(const float *src, const float *scale, int B, long long HW, int C, float *dst,
                          cudaStream_t s);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link needed).
CUresult encode_tiled(CUtensorMap *map, CUtensorMapDataType dtype, uint32_t rank, void *base, const uint64_t *dims,
                      const uint64_t *strides_bytes, const uint32_t *box, CUtensorMapSwizzle swizzle);

}  // namespace dn
