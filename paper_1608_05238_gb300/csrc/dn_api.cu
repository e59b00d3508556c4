// dn_api.cu -- C ABI of the denoiser kernels (include/mcr_denoise.h): argument checks, TMA
// tensor-map encoding and launches.
#include <mutex>

#include "../../include/mcr.h"
#include "../../include/mcr_denoise.h"
#include "dn_internal.h"

namespace dn {

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

std::mutex g_mu;
EncodeTiledFn g_encode = nullptr;
unsigned *g_err[64];  // device error word per device

EncodeTiledFn encoder() {
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_encode) {
    void *fn = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) ==
            cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      g_encode = reinterpret_cast<EncodeTiledFn>(fn);
  }
  return g_encode;
}

}  // namespace

CUresult encode_tiled(CUtensorMap *map, CUtensorMapDataType dtype, uint32_t rank, void *base, const uint64_t *dims,
                      const uint64_t *strides_bytes, const uint32_t *box, CUtensorMapSwizzle swizzle) {
  EncodeTiledFn fn = encoder();
  if (!fn) return CUDA_ERROR_NOT_SUPPORTED;
  cuuint32_t estr[5] = {1, 1, 1, 1, 1};
  return fn(map, dtype, rank, base, reinterpret_cast<const cuuint64_t *>(dims),
            reinterpret_cast<const cuuint64_t *>(strides_bytes), reinterpret_cast<const cuuint32_t *>(box), estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, swizzle, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
}

unsigned *error_word() {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_err[dev]) {
    void *p = nullptr;
    if (cudaMalloc(&p, 256) != cudaSuccess) return nullptr;
    if (cudaMemset(p, 0, 256) != cudaSuccess) return nullptr;
    g_err[dev] = static_cast<unsigned *>(p);
  }
  return g_err[dev];
}

bool conv_shape_ok(int B, int H, int W) {
  if (B <= 0 || H <= 0 || W < 32 || (W & (W - 1))) return false;
  if (((long long)H * W) % 128) return false;
  return true;
}

}  // namespace dn

using namespace dn;

extern "C" {

int dn_conv(const dn_conv_desc *d, void *stream) {
  if (!d || !d->x || !d->w || !d->out) return MCR_ERR_ARG;
  if (!conv_shape_ok(d->B, d->H, d->W)) return MCR_ERR_ARG;
  if (d->cin_pad < 64 || d->cin_pad % 64) return MCR_ERR_ARG;
  if (d->taps != 9 && d->taps != 1) return MCR_ERR_ARG;
  if (d->n_pad < 16 || d->n_pad > 256 || d->n_pad % 16 || d->cout < 1 || d->cout > d->n_pad) return MCR_ERR_ARG;
  if (d->out_stride % 8 || d->out_off % 8 || d->out_off + d->cout > d->out_stride) return MCR_ERR_ARG;
  if (d->mask && (d->mask_off + d->cout > d->mask_stride)) return MCR_ERR_ARG;
  unsigned *err = error_word();
  if (!err) return MCR_ERR_CUDA;

  const int wbox = d->W < 128 ? d->W : 128;
  const int rows = 128 / wbox;
  CUtensorMap tmX, tmW;
  {
    const uint64_t dims[4] = {(uint64_t)d->cin_pad, (uint64_t)d->W, (uint64_t)d->H, (uint64_t)d->B};
    const uint64_t strides[3] = {(uint64_t)d->cin_pad * 2, (uint64_t)d->W * d->cin_pad * 2,
                                 (uint64_t)d->H * d->W * d->cin_pad * 2};
    const uint32_t box[4] = {64, (uint32_t)wbox, (uint32_t)rows, 1};
    if (encode_tiled(&tmX, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(d->x), dims, strides, box,
                     CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
      return MCR_ERR_CUDA;
  }
  {
    const uint64_t K = (uint64_t)d->taps * d->cin_pad;
    const uint64_t dims[2] = {K, (uint64_t)d->n_pad};
    const uint64_t strides[1] = {K * 2};
    const uint32_t box[2] = {64, (uint32_t)d->n_pad};
    if (encode_tiled(&tmW, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(d->w), dims, strides, box,
                     CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
      return MCR_ERR_CUDA;
  }
  ConvArgs a{};
  a.B = d->B;
  a.H = d->H;
  a.W = d->W;
  a.cin_pad = d->cin_pad;
  a.taps = d->taps;
  a.N = d->n_pad;
  a.cout = d->cout;
  uint32_t cols = 32;
  while (cols < (uint32_t)d->n_pad) cols <<= 1;
  a.tmem_cols = cols;
  a.bias = d->bias;
  a.relu = d->relu;
  a.mask = static_cast<const __nv_bfloat16 *>(d->mask);
  a.mask_stride = d->mask_stride;
  a.mask_off = d->mask_off;
  if (d->out_f32)
    a.out_f32 = static_cast<float *>(d->out);
  else
    a.out_bf16 = static_cast<__nv_bfloat16 *>(d->out);
  a.out_stride = d->out_stride;
  a.out_off = d->out_off;
  a.err = err;
  if (launch_conv_tc(tmX, tmW, a, (cudaStream_t)stream) != cudaSuccess) return MCR_ERR_CUDA;
  return MCR_OK;
}

int dn_check(void *stream) {
  unsigned *err = error_word();
  if (!err) return MCR_ERR_CUDA;
  unsigned v = 0;
  if (cudaMemcpyAsync(&v, err, sizeof(v), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess)
    return MCR_ERR_CUDA;
  if (cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess) return MCR_ERR_CUDA;
  if (v) {
    cudaMemsetAsync(err, 0, sizeof(v), (cudaStream_t)stream);
    cudaStreamSynchronize((cudaStream_t)stream);
    return MCR_ERR_CUDA;
  }
  return MCR_OK;
}

}  // extern "C"
