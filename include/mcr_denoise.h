/*
 * mcr_denoise.h -- C ABI of the learned harmonic-map denoiser kernels in libmcr (sm_103a).
 *
 * The paper has no learned component; this is the denoiser that maps low-packet-count harmonic
 * coefficient maps (Sec. 3.1, Eqs. 8-11) to high-count ones.  Its network is a U-Net built from
 * the operations below, all hand-written: BF16 tensor-core (tcgen05, TMEM accumulator, TMA
 * operand tiles) convolutions for the forward pass and both backward passes, and small
 * memory-bound kernels for pooling, up-sampling, losses and the optimiser.
 *
 * Layout: activations are NHWC bf16 [B][H][W][C_pad] with the channel stride C_pad a multiple
 * of 64 (unused channels hold zeros); a tensor may be a channel slice [off, off + C) of a wider
 * buffer (skip-connection concatenation without copies).  Weights are [N_pad][taps][Cin_pad]
 * bf16 (taps = 9 for 3x3, 1 for 1x1), N_pad = output channels rounded up to 16; bias fp32 [C].
 * All pointers are device pointers; every call is asynchronous on `stream` and returns 0 or a
 * negative status (same codes as mcr.h).  Requirements of the convolutions: W a power of two,
 * 16 <= W, H*W a multiple of 128, N_pad <= 256.
 */
#ifndef MCR_DENOISE_H
#define MCR_DENOISE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* One convolution call: out[p, out_off + n] = epilogue(sum_{tap, c} x[p + tap, c] w[n, tap, c]). */
typedef struct {
  int32_t B, H, W;          /* images, rows, columns (stride 1, "same" padding) */
  int32_t cin_pad;          /* channel stride of x (multiple of 64) */
  const void *x;            /* bf16 NHWC input */
  int32_t taps;             /* 9 (3x3, zero padding 1) or 1 (1x1) */
  int32_t cout;             /* output channels written */
  int32_t n_pad;            /* weight rows (cout rounded up to 16, <= 256) */
  const void *w;            /* bf16 [n_pad][taps][cin_pad] */
  const float *bias;        /* fp32 [cout] or NULL */
  int32_t relu;             /* 1: ReLU after the bias */
  const void *mask;         /* bf16 NHWC or NULL: outputs where mask <= 0 are zeroed (ReLU backward) */
  int32_t mask_stride, mask_off;
  void *out;                /* NHWC output slice */
  int32_t out_f32;          /* 1: fp32 output, 0: bf16 output */
  int32_t out_stride, out_off;
  int32_t cin;              /* input channels in use (<= cin_pad; 0: all cin_pad): the weights of
                               channels [cin, cin_pad) must be zero.  With cin <= 32 a 3x3 layer of
                               <= 32 outputs reads only the first 32 channels (half the work) */
} dn_conv_desc;

/*
 * dn_conv -- forward convolution (and, with transposed weights and a mask, the input-gradient
 * pass of a ReLU convolution layer) on the tensor cores: implicit GEMM with M = 128 pixels,
 * N = n_pad, K = taps * cin_pad, BF16 operands, FP32 accumulation.  Returns MCR_ERR_ARG when the
 * shape requirements above are not met.
 */
int dn_conv(const dn_conv_desc *d, void *stream);

/* Fused output head of the denoiser (its residual output; Sec. 3.1 defines the maps it predicts). */
enum { DN_HEAD_PREDICT = 1, DN_HEAD_LOSS = 2 };
typedef struct {
  int32_t mode;             /* DN_HEAD_PREDICT or DN_HEAD_LOSS */
  const void *res;          /* x0: bf16 NHWC [B][H][W][res_stride], channels [0, cout); stride multiple of 8,
                               16-byte aligned */
  int32_t res_stride;
  const float *scale;       /* fp32 [B] per-sample input scale */
  float *pred;              /* DN_HEAD_PREDICT: fp32 [B][cout][H][W] */
  const float *target;      /* DN_HEAD_LOSS: fp32 [B][cout][H][W], unscaled */
  void *dout;               /* DN_HEAD_LOSS: bf16 NHWC, channel stride dout_stride (multiple of 8), 16-byte aligned */
  int32_t dout_stride;
  double *loss;             /* DN_HEAD_LOSS: device FP64 scalar */
} dn_head_desc;

/*
 * dn_conv_head -- the 1x1 output convolution d (taps 1, bias allowed; relu, mask and out are not
 * used) with the residual head in its epilogue, so that no NHWC fp32 output is written or re-read:
 *   y = x0 + conv(x, w) + bias  (per pixel, channels < cout)
 *   DN_HEAD_PREDICT: pred[b][c][p] = y / scale[b]              (channel-major maps)
 *   DN_HEAD_LOSS:    r = y - scale[b] target[b][c][p];  dout = bf16(2 r / (B H W cout));
 *                    loss = sum r^2 / (B H W cout): FP32 sums over 16 channels of a pixel, FP64 across
 *                    them and over per-warp partial sums in a fixed order (deterministic)
 * Bit-identical to dn_conv + dn_predict_output (prediction) and, for dout, to dn_conv + dn_pack_target
 * + dn_mse (whose loss sums every square in FP64: the two losses agree to ~1e-6 relative).  Uses the library's
 * reduction scratch: calls on one device must not overlap.  MCR_ERR_ARG on a bad shape or pointer.
 */
int dn_conv_head(const dn_conv_desc *d, const dn_head_desc *h, void *stream);

/*
 * dn_wgrad -- weight gradient of a convolution on the tensor cores:
 *   dw[n][tap][c] += sum_{b, pixel} dz[b, pixel][n] x[b, pixel + tap][c]     (FP32 accumulate)
 * with the operands in pixel-contiguous ("transposed") layouts made by dn_to_ct: dzT
 * [cout][B][H*W] and xT = three x-shifted copies [3][cin][B][H*W].  dw is fp32
 * [cout][taps][cin] and is ADDED to (zero it first); partial sums of split reductions are added
 * with atomics, so the last bits depend on scheduling.  Requires W >= 16 a power of two and
 * H*W a multiple of 64; cout, cin <= 512.
 */
int dn_wgrad(int32_t B, int32_t H, int32_t W, int32_t taps, int32_t cout, int32_t cin, const void *dzT,
             const void *xT, float *dw, void *stream);

/* NHWC bf16 slice (data + channel stride + channel offset). */
typedef struct {
  void *data;
  int32_t stride, off;
} dn_slice;

/*
 * dn_wgrad_nhwc -- weight gradient of a convolution on the tensor cores,
 *   dw[n][tap][c] += sum_{b, pixel} dz[b, pixel][n] x[b, pixel + tap][c]     (FP32 accumulate)
 * read directly from NHWC bf16 slices (no transposed copies): dz [B][H][W] channels
 * [off, off + cout) of rows of `stride`, x likewise with cin channels.  Both operands enter the tensor cores MN-major (channels contiguous); the tap's
 * shift is a TMA coordinate with zero fill at the image border.  Slice offsets and strides must
 * be multiples of 8 channels (16-byte aligned rows).  Same dw layout, accumulation and limits as
 * dn_wgrad.
 */
int dn_wgrad_nhwc(dn_slice dz, dn_slice x, int32_t B, int32_t H, int32_t W, int32_t taps, int32_t cout, int32_t cin,
                  float *dw, void *stream);
/* dn_wgrad_nhwc plus, if db != NULL, the bias gradient db[n] += sum_{b, pixel} dz[b, pixel][n]
 * (FP32).  For 3x3 layers with cout <= 64 and W a multiple of 64 the tensor cores produce it in
 * the same pass (a block of ones as one more MMA operand), otherwise a reduction kernel follows. */
int dn_wgrad_bias_nhwc(dn_slice dz, dn_slice x, int32_t B, int32_t H, int32_t W, int32_t taps, int32_t cout,
                       int32_t cin, float *dw, float *db, void *stream);

/* dst[c][b][p] = src[b][p][off + c] for c < C (bf16); shifted = 1 writes three copies
 * (dst + k*C*B*HW) with x shifted by k - 1 and zeros outside the row. */
int dn_to_ct(dn_slice src, int32_t B, int32_t H, int32_t W, int32_t C, int32_t shifted, void *dst, void *stream);
/* 2x2 average pooling of an H x W slice into an (H/2) x (W/2) slice. */
int dn_pool2(dn_slice src, int32_t B, int32_t H, int32_t W, int32_t C, dn_slice dst, void *stream);
/* dz = (skip + pool2-backward(dp)) * (act > 0) on the H x W grid (skip may have data NULL). */
int dn_pool2_bwd(dn_slice dp, dn_slice skip, dn_slice act, int32_t B, int32_t H, int32_t W, int32_t C, dn_slice dz,
                 void *stream);
/* nearest 2x up-sampling of an H x W slice into a 2H x 2W slice. */
int dn_up2(dn_slice src, int32_t B, int32_t H, int32_t W, int32_t C, dn_slice dst, void *stream);
/* dz (H x W) = 2x2 sums of du (2H x 2W) times (act > 0). */
int dn_up2_bwd(dn_slice du, dn_slice act, int32_t B, int32_t H, int32_t W, int32_t C, dn_slice dz, void *stream);
/* db[c] += sum over the B*H*W pixels of dz[., off + c]. */
int dn_bias_grad(dn_slice dz, int64_t pixels, int32_t C, float *db, void *stream);
/* Residual MSE over C channels of P pixels: y = x + out, loss = mean (y - t)^2 (FP64, fixed
 * order), dout = 2 (y - t) / (P C) as bf16 NHWC (stride dstride).  out fp32 [P][ostride], x bf16
 * [P][xstride], t fp32 [P][C]. */
int dn_mse(const float *out, int32_t ostride, const void *x, int32_t xstride, const float *t, int64_t P, int32_t C,
           void *dout, int32_t dstride, double *loss, void *stream);
/* y = x + out over C channels (fp32 [P][C]). */
int dn_residual(const float *out, int32_t ostride, const void *x, int32_t xstride, int64_t P, int32_t C, float *y,
                void *stream);
/* Adam step `step` (>= 1; 0 only refreshes the bf16 copies) on fp32 master weights [cout][taps][cin] with
 * gradient g, which it then sets to zero (the next backward pass accumulates into it); writes wf bf16
 * [n_pad][taps][cin_pad] and, if wd != NULL, the flipped input-gradient copy wd bf16
 * [cin_npad][taps][cout_pad] (wd[c][taps-1-t][n] = w[n][t][c]). */
int dn_adam(float *w, float *m, float *v, float *g, int32_t cout, int32_t taps, int32_t cin, float lr, float beta1,
            float beta2, float eps, int32_t step, void *wf, int32_t cin_pad, void *wd, int32_t cout_pad, void *stream);
int dn_adam_bias(float *b, float *m, float *v, float *g, int32_t n, float lr, float beta1, float beta2, float eps,
                 int32_t step, void *stream);
/* Every layer's dn_adam (and, where b != NULL, dn_adam_bias) step in one launch: the same
 * arithmetic and outputs as the per-layer calls.  layers: host array of n <= 32 descriptors (read
 * during the call only); all pointers device memory. */
typedef struct {
  float *w, *m, *v, *g;     /* fp32 [cout][taps][cin]: master weights, moments, gradient (zeroed) */
  void *wf;                 /* bf16 [>= cout][taps][cin_pad] forward copy */
  int32_t cin_pad;
  void *wd;                 /* bf16 flipped input-gradient copy [cin][taps][cout_pad], or NULL */
  int32_t cout_pad;
  int32_t cout, taps, cin;
  float *b, *mb, *vb, *gb;  /* fp32 [cout] bias, its moments and gradient (zeroed), or b = NULL */
} dn_adam_layer;
int dn_adam_multi(const dn_adam_layer *layers, int32_t n, float lr, float beta1, float beta2, float eps, int32_t step,
                  void *stream);
/* Per-sample input scale of channel-major fp32 maps [B][C][HW] (device): scale[b] = 1 / mean of
 * channel 0 (the fluence a_0) over the HW pixels of sample b, clamped below at 1e-30; FP64 sum in
 * a fixed order.  scale: device out [B] fp32. */
int dn_sample_scale(const float *src, int32_t B, int64_t HW, int32_t C, float *scale, void *stream);
/* channel-major fp32 maps [B][C][HW] times scale[b] -> NHWC bf16 [B][HW][stride] (input) or NHWC
 * fp32 [B][HW][C] (target); and back (output / scale). */
int dn_pack_input(const float *src, const float *scale, int32_t B, int64_t HW, int32_t C, void *dst, int32_t stride,
                  void *stream);
int dn_pack_target(const float *src, const float *scale, int32_t B, int64_t HW, int32_t C, float *dst, void *stream);
int dn_unpack_output(const float *src, const float *scale, int32_t B, int64_t HW, int32_t C, float *dst, void *stream);
/* The prediction in one pass: dst channel-major fp32 [B][C][HW] = (x + out) / scale[b], with out
 * fp32 NHWC [B*HW][ostride] (the network's output) and x bf16 NHWC [B*HW][xstride] (its scaled
 * input); = dn_residual followed by dn_unpack_output without the intermediate buffer. */
int dn_predict_output(const float *out, int32_t ostride, const void *x, int32_t xstride, const float *scale,
                      int32_t B, int64_t HW, int32_t C, float *dst, void *stream);

/* Device error word of the denoiser kernels (a bounded wait that gave up); read and clear.
 * Synchronises `stream`. */
int dn_check(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MCR_DENOISE_H */
