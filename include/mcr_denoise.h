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
 * 32 <= W, H*W a multiple of 128, N_pad <= 256.
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
} dn_conv_desc;

/*
 * dn_conv -- forward convolution (and, with transposed weights and a mask, the input-gradient
 * pass of a ReLU convolution layer) on the tensor cores: implicit GEMM with M = 128 pixels,
 * N = n_pad, K = taps * cin_pad, BF16 operands, FP32 accumulation.  Returns MCR_ERR_ARG when the
 * shape requirements above are not met.
 */
int dn_conv(const dn_conv_desc *d, void *stream);

/* Device error word of the denoiser kernels (a bounded wait that gave up); read and clear.
 * Synchronises `stream`. */
int dn_check(void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MCR_DENOISE_H */
