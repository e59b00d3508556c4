/*
 * mcr3.h -- C ABI of the 3D forward/adjoint radiance Monte Carlo (libmcr.so), the extension the
 * paper names in Sec. 3.1: its 2D Fourier angular basis becomes real spherical harmonics in 3D.
 *
 * Geometry: voxels [nz][ny][nx] of side dx (mm), voxel (ix, iy, iz) covers
 * [ix dx, (ix+1) dx) x [iy dx, (iy+1) dx) x [iz dx, (iz+1) dx); z is depth.  Directions
 * s = (sin th cos ph, sin th sin ph, cos th), th from +z.  Scattering: the 3D Henyey-Greenstein
 * phase function.  Tally: c_lm = sum over voxel segments of the track weight t = W (1 - e^{-mu_a l})
 * / mu_a times Y_lm(s), for orthonormal real spherical harmonics Y_lm up to l = L (index
 * l^2 + l + m, (L+1)^2 channels), normalised by S / (N_p dx^3); then phi(s) = sum c_lm Y_lm(s),
 * the fluence is sqrt(4 pi) c_00 and H = mu_a sqrt(4 pi) c_00 (Sec. 2).  Adjoint runs (Sec. 4,
 * Eq. 12, source q* per unit volume and solid angle, sampled by |q*|, W0 = sign q*) tally at -s:
 * c*_lm = (-1)^l c_lm of the run from q*.  Gradients (Sec. 5 in 3D): for a voxel loss L(H) with
 * v = dL/dH, q* = -mu_a v / dx^3 and
 *   dL/dmu_a = v sqrt(4 pi) c_00 + dx^3 sum_lm c_lm c*_lm,
 *   dL/dmu_s = dx^3 sum_lm (1 - g^l) c_lm c*_lm          (the HG kernel is sum_l g^l sum_m Y_lm Y_lm).
 * Random numbers, uniforms and roulette as in mcr.h; launch event 0: words 0, 1 pick the voxel of
 * a volumetric source, word 2 -> cos th = 2u - 1, word 3 -> ph = 2 pi u; event 1: words 0..2 -> the
 * position in that voxel; flight k >= 1 uses event k+1: word 0 free path, 1 HG cosine, 2 roulette,
 * 3 scattering azimuth.  All arrays are caller-owned device memory; statuses as in mcr.h.
 */
#ifndef MCR3_H
#define MCR3_H

#include <stdint.h>

#include "mcr.h"

#ifdef __cplusplus
extern "C" {
#endif

#define MCR3_MAX_L 8

typedef struct {
  int32_t nx, ny, nz; /* voxels, each >= 1, nx ny nz < 2^26 */
  float dx;           /* voxel side, mm, > 0 */
  float g;            /* 3D Henyey-Greenstein anisotropy, -1 < g < 1 */
  const float *mua;   /* device [nz][ny][nx], 1/mm, >= 0 */
  const float *mus;   /* device [nz][ny][nx], 1/mm, >= 0 */
} mcr3_medium;

typedef struct {
  int32_t kind;             /* MCR_PENCIL (collimated) or MCR_ISO_POINT */
  float x0, y0, z0;         /* mm */
  float dir_x, dir_y, dir_z; /* pencil direction, normalised by the library */
  float power;              /* total source power S */
} mcr3_source;

/* Forward run: coeff device out [(L+1)^2][nz][ny][nx], L = run->K <= MCR3_MAX_L, n_packets <= 2^26
 * per call (use first_packet and run->accumulate to add further ranges); run->sectors and
 * run->time_bins must be 0. */
int mc3_forward(const mcr3_medium *med, const mcr3_source *src, const mcr_run *run, float *coeff, mcr_stats *stats,
                void *stream);
/* Adjoint run from qstar (device [nz][ny][nx], signed, per unit volume and solid angle). */
int mc3_adjoint(const mcr3_medium *med, const float *qstar, const mcr_run *run, float *coeff_adj, mcr_stats *stats,
                void *stream);
/* H = mu_a sqrt(4 pi) c_00 (device out [nz][ny][nx]); if Hmeas: dL_dH = -dx^3 (Hmeas - H) and
 * eps = 1/2 dx^3 sum (Hmeas - H)^2 (device FP64 scalar); dL_dH, eps may be NULL. */
int mc3_h_eps(const mcr3_medium *med, const float *coeff, const float *Hmeas, float *H, float *dL_dH, double *eps,
              void *stream);
/* qstar = -mu_a dL_dH / dx^3. */
int mc3_adjoint_source(const mcr3_medium *med, const float *dL_dH, float *qstar, void *stream);
/* The gradients above in FP64 (device out [nz][ny][nx] each), L the coefficients' order. */
int mc3_gradient(const mcr3_medium *med, int32_t L, const float *coeff, const float *coeff_adj, const float *dL_dH,
                 double *d_mua, double *d_mus, void *stream);
/* The same FP64 sums, each result rounded once to FP32 (device out [nz][ny][nx] each). */
int mc3_gradient_f32(const mcr3_medium *med, int32_t L, const float *coeff, const float *coeff_adj,
                     const float *dL_dH, float *d_mua, float *d_mus, void *stream);

#ifdef __cplusplus
}
#endif
#endif
