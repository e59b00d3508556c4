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

constexpr int kPartialsCap = 4096;  // doubles in the per-device scratch of the loss reductions

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

double *partials_buffer() {
  static double *g_partials[64];
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lock(g_mu);
  if (!g_partials[dev]) {
    void *p = nullptr;
    if (cudaMalloc(&p, kPartialsCap * sizeof(double)) != cudaSuccess) return nullptr;
    g_partials[dev] = static_cast<double *>(p);
  }
  return g_partials[dev];
}

bool conv_shape_ok(int B, int H, int W) {
  if (B <= 0 || H <= 0 || W < 16 || (W & (W - 1))) return false;
  if (((long long)H * W) % 128) return false;
  return true;
}

}  // namespace dn

using namespace dn;

extern "C" {

}  // extern "C"

// Shape checks, tensor maps and epilogue arguments shared by dn_conv and dn_conv_head.
static int conv_setup(const dn_conv_desc *d, CUtensorMap &tmX, CUtensorMap &tmW, ConvArgs &a) {
  if (!d->x || !d->w) return MCR_ERR_ARG;
  if (!conv_shape_ok(d->B, d->H, d->W)) return MCR_ERR_ARG;
  if (d->cin_pad < 64 || d->cin_pad % 64) return MCR_ERR_ARG;
  if (d->taps != 9 && d->taps != 1) return MCR_ERR_ARG;
  if (d->n_pad < 16 || d->n_pad > 256 || d->n_pad % 16 || d->cout < 1 || d->cout > d->n_pad) return MCR_ERR_ARG;
  if (d->mask && (d->mask_off + d->cout > d->mask_stride)) return MCR_ERR_ARG;
  if (d->cin < 0 || d->cin > d->cin_pad) return MCR_ERR_ARG;
  unsigned *err = error_word();
  if (!err) return MCR_ERR_CUDA;

  const int wbox = d->W < 128 ? d->W : 128;
  const int rows = 128 / wbox;
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
  a.mask_vec = d->mask && d->mask_stride % 8 == 0 && d->mask_off % 8 == 0 &&
               (reinterpret_cast<uintptr_t>(d->mask) & 15) == 0;
  a.err = err;
  return MCR_OK;
}

extern "C" {

int dn_conv(const dn_conv_desc *d, void *stream) {
  if (!d || !d->out) return MCR_ERR_ARG;
  if (d->out_stride % 8 || d->out_off % 8 || d->out_off + d->cout > d->out_stride) return MCR_ERR_ARG;
  CUtensorMap tmX, tmW;
  ConvArgs a{};
  const int rc = conv_setup(d, tmX, tmW, a);
  if (rc != MCR_OK) return rc;
  if (d->out_f32)
    a.out_f32 = static_cast<float *>(d->out);
  else
    a.out_bf16 = static_cast<__nv_bfloat16 *>(d->out);
  a.out_stride = d->out_stride;
  a.out_off = d->out_off;
  if (conv_halo_applies(a)) {  // few output channels: one haloed input box per channel block
    // an input with <= 32 channels of data: 32-channel rows (64-byte swizzle), half the MMAs
    const int kb = (d->cin > 0 && d->cin <= 32) ? 32 : 64;
    const CUtensorMapSwizzle sw = kb == 32 ? CU_TENSOR_MAP_SWIZZLE_64B : CU_TENSOR_MAP_SWIZZLE_128B;
    CUtensorMap tmH, tmWk;
    const uint64_t dims[4] = {(uint64_t)d->cin_pad, (uint64_t)d->W, (uint64_t)d->H, (uint64_t)d->B};
    const uint64_t strides[3] = {(uint64_t)d->cin_pad * 2, (uint64_t)d->W * d->cin_pad * 2,
                                 (uint64_t)d->H * d->W * d->cin_pad * 2};
    const uint32_t box[4] = {(uint32_t)kb, 130, 3, 1};
    if (encode_tiled(&tmH, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, const_cast<void *>(d->x), dims, strides, box, sw) !=
        CUDA_SUCCESS)
      return MCR_ERR_CUDA;
    if (kb == 32) {  // weight boxes of 32 channels of each tap
      const uint64_t K = (uint64_t)d->taps * d->cin_pad;
      const uint64_t wdims[2] = {K, (uint64_t)d->n_pad};
      const uint64_t wstrides[1] = {K * 2};
      const uint32_t wbox[2] = {32, (uint32_t)d->n_pad};
      if (encode_tiled(&tmWk, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void *>(d->w), wdims, wstrides, wbox,
                       CU_TENSOR_MAP_SWIZZLE_64B) != CUDA_SUCCESS)
        return MCR_ERR_CUDA;
    }
    if (launch_conv_halo(tmH, kb == 32 ? tmWk : tmW, a, (cudaStream_t)stream, kb) != cudaSuccess) return MCR_ERR_CUDA;
    return MCR_OK;
  }
  if (launch_conv_tc(tmX, tmW, a, (cudaStream_t)stream) != cudaSuccess) return MCR_ERR_CUDA;
  return MCR_OK;
}

int dn_conv_head(const dn_conv_desc *d, const dn_head_desc *h, void *stream) {
  if (!d || !h || d->taps != 1 || d->relu || d->mask) return MCR_ERR_ARG;
  if (h->mode != DN_HEAD_PREDICT && h->mode != DN_HEAD_LOSS) return MCR_ERR_ARG;
  const auto al16 = [](const void *p) { return (reinterpret_cast<uintptr_t>(p) & 15) == 0; };
  if (!h->res || !h->scale || h->res_stride < d->cout || h->res_stride % 8 || !al16(h->res)) return MCR_ERR_ARG;
  if (h->mode == DN_HEAD_PREDICT && !h->pred) return MCR_ERR_ARG;
  if (h->mode == DN_HEAD_LOSS &&
      (!h->target || !h->dout || !h->loss || h->dout_stride < d->cout || h->dout_stride % 8 || !al16(h->dout)))
    return MCR_ERR_ARG;
  CUtensorMap tmX, tmW;
  ConvArgs a{};
  const int rc = conv_setup(d, tmX, tmW, a);
  if (rc != MCR_OK) return rc;
  double *partials = partials_buffer();
  if (!partials) return MCR_ERR_CUDA;
  int dev = 0, sms = 0;  // the loss head writes <= 8 partial sums per block, at most one block per SM
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    return MCR_ERR_CUDA;
  if (8 * sms > kPartialsCap) return MCR_ERR_ARG;
  const long long P = (long long)d->B * d->H * d->W;
  const double inv = 1.0 / ((double)P * d->cout);
  a.head = h->mode;
  a.res = static_cast<const __nv_bfloat16 *>(h->res);
  a.res_stride = h->res_stride;
  a.scale = h->scale;
  a.HW = d->H * d->W;
  a.pred = h->pred;
  a.target = h->target;
  a.dout = static_cast<__nv_bfloat16 *>(h->dout);
  a.dout_stride = h->dout_stride;
  a.two_over_count = (float)(2.0 * inv);
  a.partials = partials;
  int n_partials = 0;
  if (launch_conv_tc(tmX, tmW, a, (cudaStream_t)stream, &n_partials) != cudaSuccess) return MCR_ERR_CUDA;
  if (h->mode == DN_HEAD_LOSS && sum_partials(partials, n_partials, inv, h->loss, (cudaStream_t)stream) != cudaSuccess)
    return MCR_ERR_CUDA;
  return MCR_OK;
}

int dn_wgrad(int32_t B, int32_t H, int32_t W, int32_t taps, int32_t cout, int32_t cin, const void *dzT,
             const void *xT, float *dw, void *stream) {
  if (!dzT || !xT || !dw || (taps != 9 && taps != 1)) return MCR_ERR_ARG;
  if (B <= 0 || H <= 0 || W < 16 || (W & (W - 1)) || ((long long)H * W) % 64) return MCR_ERR_ARG;
  if (cout < 1 || cin < 1 || cout > 512 || cin > 512) return MCR_ERR_ARG;
  unsigned *err = error_word();
  if (!err) return MCR_ERR_CUDA;
  const uint64_t HW = (uint64_t)H * W;
  CUtensorMap tmA, tmB[3];
  {
    const uint64_t dims[3] = {HW, (uint64_t)B, (uint64_t)cout};
    const uint64_t strides[2] = {HW * 2, (uint64_t)B * HW * 2};
    const uint32_t box[3] = {64, 1, 128};
    if (encode_tiled(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, const_cast<void *>(dzT), dims, strides, box,
                     CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
      return MCR_ERR_CUDA;
  }
  const int N = cin > 128 ? 128 : ((cin + 15) / 16) * 16;
  for (int k = 0; k < 3; ++k) {
    const uint64_t dims[3] = {HW, (uint64_t)B, (uint64_t)cin};
    const uint64_t strides[2] = {HW * 2, (uint64_t)B * HW * 2};
    const uint32_t box[3] = {64, 1, (uint32_t)N};
    void *base = static_cast<char *>(const_cast<void *>(xT)) + (size_t)k * cin * B * HW * 2;
    if (encode_tiled(&tmB[k], CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 3, base, dims, strides, box,
                     CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
      return MCR_ERR_CUDA;
  }
  WgradArgs a{};
  a.B = B;
  a.HW = (int)HW;
  a.W = W;
  a.taps = taps;
  a.cout = cout;
  a.cin = cin;
  a.cin_pad = cin;
  a.N = N;
  a.m_tiles = (cout + 127) / 128;
  a.n_tiles = (cin + N - 1) / N;
  const long long kblocks = (long long)B * HW / 64;
  long long splits = (2 * 152 + taps * a.m_tiles * a.n_tiles - 1) / (taps * a.m_tiles * a.n_tiles);
  if (splits > kblocks) splits = kblocks;
  if (splits < 1) splits = 1;
  a.splits = (int)splits;
  uint32_t cols = 32;
  while (cols < (uint32_t)N) cols <<= 1;
  a.tmem_cols = cols;
  a.dw = dw;
  a.err = err;
  if (launch_wgrad_tc(tmA, tmB, a, (cudaStream_t)stream) != cudaSuccess) return MCR_ERR_CUDA;
  return MCR_OK;
}

#define DN_TRY(expr) return (expr) == cudaSuccess ? MCR_OK : MCR_ERR_CUDA

static bool slice_ok(const dn_slice &s, int C) { return s.data && s.off >= 0 && s.off + C <= s.stride; }

int dn_wgrad_nhwc(dn_slice dz, dn_slice x, int32_t B, int32_t H, int32_t W, int32_t taps, int32_t cout, int32_t cin,
                  float *dw, void *stream) {
  return dn_wgrad_bias_nhwc(dz, x, B, H, W, taps, cout, cin, dw, nullptr, stream);
}

int dn_wgrad_bias_nhwc(dn_slice dz, dn_slice x, int32_t B, int32_t H, int32_t W, int32_t taps, int32_t cout,
                       int32_t cin, float *dw, float *db, void *stream) {
  if (!slice_ok(dz, cout) || !slice_ok(x, cin) || !dw || (taps != 9 && taps != 1)) return MCR_ERR_ARG;
  if (B <= 0 || H <= 0 || W < 16 || (W & (W - 1)) || ((long long)H * W) % 64) return MCR_ERR_ARG;
  if (cout < 1 || cin < 1 || cout > 512 || cin > 512) return MCR_ERR_ARG;
  // TMA: 16-byte aligned slice bases and row strides
  if (dz.off % 8 || dz.stride % 8 || x.off % 8 || x.stride % 8) return MCR_ERR_ARG;
  unsigned *err = error_word();
  if (!err) return MCR_ERR_CUDA;
  const uint64_t HW = (uint64_t)H * W;
  CUtensorMap tmA, tmB;
  {
    const uint64_t dims[2] = {(uint64_t)cout, (uint64_t)B * HW};
    const uint64_t strides[1] = {(uint64_t)dz.stride * 2};
    const uint32_t box[2] = {64, 64};
    void *base = static_cast<char *>(dz.data) + (size_t)dz.off * 2;
    if (encode_tiled(&tmA, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, base, dims, strides, box,
                     CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
      return MCR_ERR_CUDA;
  }
  {
    const int wbox = W < 64 ? W : 64;
    const uint64_t dims[4] = {(uint64_t)cin, (uint64_t)W, (uint64_t)H, (uint64_t)B};
    const uint64_t strides[3] = {(uint64_t)x.stride * 2, (uint64_t)W * x.stride * 2, HW * x.stride * 2};
    const uint32_t box[4] = {64, (uint32_t)wbox, (uint32_t)(64 / wbox), 1};
    void *base = static_cast<char *>(x.data) + (size_t)x.off * 2;
    if (encode_tiled(&tmB, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box,
                     CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
      return MCR_ERR_CUDA;
  }
  WgradArgs a{};
  a.B = B;
  a.HW = (int)HW;
  a.W = W;
  a.taps = taps;
  a.cout = cout;
  a.cin = cin;
  a.cin_pad = cin;
  a.dw = dw;
  a.err = err;
  if (wgrad_halo_applies(taps, cout, W)) {  // few output channels: all nine taps from one haloed box
    a.db = db;                              // its bias gradient comes with it
    CUtensorMap tmH;
    const uint64_t dims[4] = {(uint64_t)cin, (uint64_t)W, (uint64_t)H, (uint64_t)B};
    const uint64_t strides[3] = {(uint64_t)x.stride * 2, (uint64_t)W * x.stride * 2, HW * x.stride * 2};
    const uint32_t box[4] = {64, 66, 3, 1};
    void *base = static_cast<char *>(x.data) + (size_t)x.off * 2;
    if (encode_tiled(&tmH, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 4, base, dims, strides, box,
                     CU_TENSOR_MAP_SWIZZLE_128B) != CUDA_SUCCESS)
      return MCR_ERR_CUDA;
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
      return MCR_ERR_CUDA;
    const long long segs = (long long)B * HW / 64;
    long long splits = sms / ((cin + 63) / 64);  // one block per SM, one wave
    if (splits > segs) splits = segs;
    if (splits < 1) splits = 1;
    a.splits = (int)splits;
    if (launch_wgrad_halo(tmA, tmH, a, (cudaStream_t)stream) != cudaSuccess) return MCR_ERR_CUDA;
    return MCR_OK;
  }
  a.N = cin > 128 ? 128 : ((cin + 15) / 16) * 16;  // MMA N; B arrives in whole 64-channel boxes
  a.m_tiles = (cout + 127) / 128;
  a.n_tiles = (cin + a.N - 1) / a.N;
  const long long kblocks = (long long)B * HW / 64;
  long long splits = (2 * 152) / (taps * a.m_tiles * a.n_tiles);  // one wave of two blocks per SM
  if (splits > kblocks / 16) splits = kblocks / 16;  // >= 16 K blocks per CTA: its atomic epilogue stays small
  if (splits < 1) splits = 1;
  a.splits = (int)splits;
  uint32_t cols = 32;
  while (cols < (uint32_t)a.N) cols <<= 1;
  a.tmem_cols = cols;
  if (launch_wgrad_mn(tmA, tmB, a, (cudaStream_t)stream) != cudaSuccess) return MCR_ERR_CUDA;
  if (db && bias_grad(static_cast<const __nv_bfloat16 *>(dz.data), (long long)B * HW, dz.stride, dz.off, cout, db,
                      (cudaStream_t)stream) != cudaSuccess)
    return MCR_ERR_CUDA;
  return MCR_OK;
}

int dn_to_ct(dn_slice src, int32_t B, int32_t H, int32_t W, int32_t C, int32_t shifted, void *dst, void *stream) {
  if (!slice_ok(src, C) || !dst || B <= 0 || H <= 0 || W <= 0 || C <= 0) return MCR_ERR_ARG;
  DN_TRY(to_ct(static_cast<const __nv_bfloat16 *>(src.data), B, H * W, W, src.stride, src.off, C, shifted,
               static_cast<__nv_bfloat16 *>(dst), (cudaStream_t)stream));
}

int dn_pool2(dn_slice src, int32_t B, int32_t H, int32_t W, int32_t C, dn_slice dst, void *stream) {
  if (!slice_ok(src, C) || !slice_ok(dst, C) || B <= 0 || H < 2 || W < 2 || H % 2 || W % 2) return MCR_ERR_ARG;
  DN_TRY(pool2(static_cast<const __nv_bfloat16 *>(src.data), B, H, W, src.stride, src.off, C,
               static_cast<__nv_bfloat16 *>(dst.data), dst.stride, dst.off, (cudaStream_t)stream));
}

int dn_pool2_bwd(dn_slice dp, dn_slice skip, dn_slice act, int32_t B, int32_t H, int32_t W, int32_t C, dn_slice dz,
                 void *stream) {
  if (!slice_ok(dp, C) || !slice_ok(act, C) || !slice_ok(dz, C) || (skip.data && !slice_ok(skip, C))) return MCR_ERR_ARG;
  if (B <= 0 || H < 2 || W < 2 || H % 2 || W % 2) return MCR_ERR_ARG;
  DN_TRY(pool2_bwd(static_cast<const __nv_bfloat16 *>(dp.data), dp.stride, dp.off,
                   static_cast<const __nv_bfloat16 *>(skip.data), skip.stride, skip.off,
                   static_cast<const __nv_bfloat16 *>(act.data), act.stride, act.off, B, H, W, C,
                   static_cast<__nv_bfloat16 *>(dz.data), dz.stride, dz.off, (cudaStream_t)stream));
}

int dn_up2(dn_slice src, int32_t B, int32_t H, int32_t W, int32_t C, dn_slice dst, void *stream) {
  if (!slice_ok(src, C) || !slice_ok(dst, C) || B <= 0 || H <= 0 || W <= 0) return MCR_ERR_ARG;
  DN_TRY(up2(static_cast<const __nv_bfloat16 *>(src.data), B, H, W, src.stride, src.off, C,
             static_cast<__nv_bfloat16 *>(dst.data), dst.stride, dst.off, (cudaStream_t)stream));
}

int dn_up2_bwd(dn_slice du, dn_slice act, int32_t B, int32_t H, int32_t W, int32_t C, dn_slice dz, void *stream) {
  if (!slice_ok(du, C) || !slice_ok(act, C) || !slice_ok(dz, C) || B <= 0 || H <= 0 || W <= 0) return MCR_ERR_ARG;
  DN_TRY(up2_bwd(static_cast<const __nv_bfloat16 *>(du.data), du.stride, du.off,
                 static_cast<const __nv_bfloat16 *>(act.data), act.stride, act.off, B, H, W, C,
                 static_cast<__nv_bfloat16 *>(dz.data), dz.stride, dz.off, (cudaStream_t)stream));
}

int dn_bias_grad(dn_slice dz, int64_t pixels, int32_t C, float *db, void *stream) {
  if (!slice_ok(dz, C) || !db || pixels <= 0) return MCR_ERR_ARG;
  DN_TRY(bias_grad(static_cast<const __nv_bfloat16 *>(dz.data), pixels, dz.stride, dz.off, C, db,
                   (cudaStream_t)stream));
}

int dn_mse(const float *out, int32_t ostride, const void *x, int32_t xstride, const float *t, int64_t P, int32_t C,
           void *dout, int32_t dstride, double *loss, void *stream) {
  if (!out || !x || !t || !dout || !loss || P <= 0 || C <= 0 || ostride < C || xstride < C || dstride < C)
    return MCR_ERR_ARG;
  double *partials = partials_buffer();
  if (!partials) return MCR_ERR_CUDA;
  DN_TRY(mse(out, ostride, static_cast<const __nv_bfloat16 *>(x), xstride, t, P, C, static_cast<__nv_bfloat16 *>(dout),
             dstride, partials, kPartialsCap, loss, (cudaStream_t)stream));
}

int dn_residual(const float *out, int32_t ostride, const void *x, int32_t xstride, int64_t P, int32_t C, float *y,
                void *stream) {
  if (!out || !x || !y || P <= 0 || C <= 0 || ostride < C || xstride < C) return MCR_ERR_ARG;
  DN_TRY(residual(out, ostride, static_cast<const __nv_bfloat16 *>(x), xstride, P, C, y, (cudaStream_t)stream));
}

int dn_adam(float *w, float *m, float *v, float *g, int32_t cout, int32_t taps, int32_t cin, float lr,
            float beta1, float beta2, float eps, int32_t step, void *wf, int32_t cin_pad, void *wd, int32_t cout_pad,
            void *stream) {
  if (!w || !wf || cout <= 0 || cin <= 0 || cin_pad < cin || (taps != 9 && taps != 1)) return MCR_ERR_ARG;
  if (step > 0 && (!m || !v || !g)) return MCR_ERR_ARG;
  if (wd && cout_pad < cout) return MCR_ERR_ARG;
  DN_TRY(adam(w, m, v, g, cout, taps, cin, lr, beta1, beta2, eps, step, static_cast<__nv_bfloat16 *>(wf), cin_pad,
              static_cast<__nv_bfloat16 *>(wd), cout_pad, (cudaStream_t)stream));
}

int dn_adam_multi(const dn_adam_layer *layers, int32_t n, float lr, float beta1, float beta2, float eps, int32_t step,
                  void *stream) {
  if (!layers || n < 1 || n > kMaxAdamLayers) return MCR_ERR_ARG;
  AdamTable T{};
  T.n = n;
  long long blocks = 0;
  for (int l = 0; l < n; ++l) {
    const dn_adam_layer &d = layers[l];
    if (!d.w || !d.wf || d.cout <= 0 || d.cin <= 0 || d.cin_pad < d.cin || (d.taps != 9 && d.taps != 1)) return MCR_ERR_ARG;
    if (step > 0 && (!d.m || !d.v || !d.g)) return MCR_ERR_ARG;
    if (d.wd && d.cout_pad < d.cout) return MCR_ERR_ARG;
    if (d.b && step > 0 && (!d.mb || !d.vb || !d.gb)) return MCR_ERR_ARG;
    AdamLayer &L = T.L[l];
    L.w = d.w;
    L.m = d.m;
    L.v = d.v;
    L.g = d.g;
    L.wf = static_cast<__nv_bfloat16 *>(d.wf);
    L.wd = static_cast<__nv_bfloat16 *>(d.wd);
    L.b = d.b;
    L.mb = d.mb;
    L.vb = d.vb;
    L.gb = d.gb;
    L.cout = d.cout;
    L.taps = d.taps;
    L.cin = d.cin;
    L.cin_pad = d.cin_pad;
    L.cout_pad = d.cout_pad;
    L.tile0 = (int)blocks;
    blocks += (long long)d.taps * ((d.cout + 31) / 32) * ((d.cin + 31) / 32);
  }
  if (blocks > 0x7fffffffll) return MCR_ERR_ARG;
  DN_TRY(adam_multi(T, lr, beta1, beta2, eps, step, (int)blocks, (cudaStream_t)stream));
}

int dn_adam_bias(float *b, float *m, float *v, float *g, int32_t n, float lr, float beta1, float beta2,
                 float eps, int32_t step, void *stream) {
  if (!b || !m || !v || !g || n <= 0) return MCR_ERR_ARG;
  DN_TRY(adam_bias(b, m, v, g, n, lr, beta1, beta2, eps, step, (cudaStream_t)stream));
}

int dn_pack_input(const float *src, const float *scale, int32_t B, int64_t HW, int32_t C, void *dst, int32_t stride,
                  void *stream) {
  if (!src || !scale || !dst || B <= 0 || HW <= 0 || C <= 0 || stride < C) return MCR_ERR_ARG;
  DN_TRY(pack_input(src, scale, B, HW, C, static_cast<__nv_bfloat16 *>(dst), stride, (cudaStream_t)stream));
}

int dn_sample_scale(const float *src, int32_t B, int64_t HW, int32_t C, float *scale, void *stream) {
  if (!src || !scale || B <= 0 || HW <= 0 || C <= 0) return MCR_ERR_ARG;
  DN_TRY(sample_scale(src, B, HW, C, scale, (cudaStream_t)stream));
}

int dn_pack_target(const float *src, const float *scale, int32_t B, int64_t HW, int32_t C, float *dst, void *stream) {
  if (!src || !scale || !dst || B <= 0 || HW <= 0 || C <= 0) return MCR_ERR_ARG;
  DN_TRY(pack_target(src, scale, B, HW, C, dst, (cudaStream_t)stream));
}

int dn_predict_output(const float *out, int32_t ostride, const void *x, int32_t xstride, const float *scale,
                      int32_t B, int64_t HW, int32_t C, float *dst, void *stream) {
  if (!out || !x || !scale || !dst || B <= 0 || HW <= 0 || C <= 0 || ostride < C || xstride < C) return MCR_ERR_ARG;
  DN_TRY(predict_output(out, ostride, static_cast<const __nv_bfloat16 *>(x), xstride, scale, B, HW, C, dst,
                        (cudaStream_t)stream));
}

int dn_unpack_output(const float *src, const float *scale, int32_t B, int64_t HW, int32_t C, float *dst,
                     void *stream) {
  if (!src || !scale || !dst || B <= 0 || HW <= 0 || C <= 0) return MCR_ERR_ARG;
  DN_TRY(unpack_output(src, scale, B, HW, C, dst, (cudaStream_t)stream));
}

int dn_wait_probe(uint32_t spins, int32_t *timed_out, void *stream) {
  if (!timed_out || spins == 0 || spins > (1u << 24)) return MCR_ERR_ARG;
  unsigned *err = error_word();
  if (!err) return MCR_ERR_CUDA;
  int *d = nullptr;
  if (cudaMalloc(&d, sizeof(int)) != cudaSuccess) {
    cudaGetLastError();
    return MCR_ERR_NOMEM;
  }
  int rc = MCR_OK;
  if (launch_wait_probe(err, spins, d, (cudaStream_t)stream) != cudaSuccess ||
      cudaMemcpyAsync(timed_out, d, sizeof(int), cudaMemcpyDeviceToHost, (cudaStream_t)stream) != cudaSuccess ||
      cudaStreamSynchronize((cudaStream_t)stream) != cudaSuccess)
    rc = MCR_ERR_CUDA;
  cudaFree(d);
  return rc;
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
