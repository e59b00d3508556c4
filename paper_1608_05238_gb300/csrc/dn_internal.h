// dn_internal.h -- declarations shared by the denoiser translation units (not part of the ABI).
#pragma once

#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace dn {

// Implicit-GEMM convolution launch arguments (see k_conv_tc).
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
};

size_t conv_smem_bytes(int N);
cudaError_t launch_conv_tc(const CUtensorMap &tmX, const CUtensorMap &tmW, const ConvArgs &a, cudaStream_t s);

// cuTensorMapEncodeTiled through the runtime's driver entry point (no libcuda link needed).
CUresult encode_tiled(CUtensorMap *map, CUtensorMapDataType dtype, uint32_t rank, void *base, const uint64_t *dims,
                      const uint64_t *strides_bytes, const uint32_t *box, CUtensorMapSwizzle swizzle);

}  // namespace dn
