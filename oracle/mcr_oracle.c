/*
 * mcr_oracle.c -- plain, slow, FP64 CPU oracle for the 2D forward and adjoint
 * harmonic radiance Monte Carlo of Hochuli, Powell, Arridge & Cox,
 * "Quantitative photoacoustic tomography using forward and adjoint Monte
 * Carlo models of radiance" (arXiv 1608.05238).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the correctness reference against
 * which the CUDA path is checked.  Only the test-suite, the smoke check and
 * the CPU-baseline leg of the benchmark may build, load or call it.  It shares
 * no code, header, table or helper with the CUDA library.
 *
 * What it computes, step by step, in the order of the paper (Section 3):
 *   launch a packet ("photon") of weight W from the source;
 *   sample a free path from mu_s only;                         (Sec. 3, text)
 *   along the path, pixel by pixel, deposit the weight lost to absorption
 *   and attenuate W <- W exp(-mu_a s);                          (Sec. 3, text)
 *   tally the deposit into the harmonic coefficients a_0, a_n, b_n of the
 *   pixel at the packet's direction theta;              (Sec. 3.1, Eq. 9-11)
 *   at the end of the path, scatter by the 2D Henyey-Greenstein angle
 *   theta_s = 2 atan((1-g)/(1+g) tan(pi U));                      (Eq. 7)
 *   repeat until the weight falls below a threshold.            (Sec. 3, text)
 * The adjoint run (Sec. 4, Sec. 6) launches isotropically from a volumetric,
 * signed source q*(x) with the position uniform over the source pixel, and
 * its tally is taken at theta + pi (the adjoint radiance looks back along
 * the path; see the readings below).
 *
 * Readings of the paper taken here (where it is silent or garbled):
 *  - Free path: the paper prints s = U/mu_s; read as s = -ln(U)/mu_s, an
 *    exponential free path with absorption applied as continuous weight
 *    loss (absorption weighting).
 *  - Tally quantity: the coefficients hold RADIANCE, so that a_0 is the
 *    fluence (Sec. 5) and H = mu_a a_0 (Sec. 2).  Each pixel segment of
 *    length l deposits its track weight t = W (1 - exp(-mu_a l)) / mu_a
 *    (= W l when mu_a = 0), i.e. the absorbed weight dW divided by mu_a,
 *    normalised by N_p and the pixel area.
 *  - Adjoint direction: with psi(x,s) = phi*(x,-s), psi solves the forward
 *    RTE (Eq. 12 vs Eq. 5, HG symmetric), so the adjoint coefficients are
 *    tallied at theta + pi: a*_n = (-1)^n a_n^psi, b*_n = (-1)^n b_n^psi.
 *  - Termination: the paper's threshold on |W| (Sec. 6) is completed by
 *    Russian roulette (survive with probability p, W <- W/p) so that the
 *    estimate stays unbiased.
 *  - Adjoint source sampling: the source pixel is drawn with probability
 *    proportional to |q*_i| (uniform pixel areas), quantised to integers
 *    relative to max|q*| with 2^32 levels, and the packet weight is
 *    sign(q*_i); the total source strength is S = 2 pi A sum|q*| (q* is per
 *    unit area and unit angle and isotropic).
 *
 * Conventions.  x = column (lateral), z = row (depth, z = 0 the top edge).
 * Pixel (ix, iz) covers [ix dx, (ix+1) dx) x [iz dx, (iz+1) dx); a source
 * point exactly on the far edge belongs to the last pixel.  The direction
 * angle theta is measured from the +z axis: s = (sin theta, cos theta) =
 * (s_x, s_z) (Sec. 3.1).  Coefficient channel c: c = 0 is a_0, c = 2n-1 is
 * a_n, c = 2n is b_n; output layout [2K+1][nz][nx].
 *
 * Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11),
 * written here from its published definition.  Key (seed_lo, seed_hi ^
 * stream_id), counter (packet_lo, packet_hi, event, 0).  Event 0 and 1 are
 * the launch; flight k >= 1 uses event k+1 (word 0 -> free path, word 1 ->
 * scattering angle, word 2 -> roulette).  A 32-bit word x maps to the
 * uniform u = ((x >> 9) + 1/2) 2^-23, which is exact in FP32 and FP64.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_PENCIL 0
#define ORC_LINE 1
#define ORC_ISO_POINT 2
#define ORC_ANGULAR_POINT 3 /* point source with an angular density (a detector's, Sec. 4.1) */
#define ORC_VOLUME 100      /* internal: volumetric isotropic source (adjoint) */
#define ORC_MAX_ANG 8

#define ORC_OK 0
#define ORC_ERR_ARG -1
#define ORC_ERR_NOMEM -3

typedef struct {
  int32_t nx, nz;
  double dx;          /* pixel side, mm */
  double g;           /* HG anisotropy */
  const double *mua;  /* [nz][nx], 1/mm */
  const double *mus;  /* [nz][nx], 1/mm */
} orc_medium;

typedef struct {
  int32_t kind;
  double x0, z0, x1, z1; /* mm */
  double dir_x, dir_z;   /* unit direction for pencil / line */
  double power;          /* total source power */
  /* angular point: p(theta) = (1 + sum_n ang_c[n-1] cos n theta + ang_s[n-1] sin n theta) / (2 pi),
   * theta from +z, n = 1 .. n_ang */
  int32_t n_ang;
  double ang_c[ORC_MAX_ANG], ang_s[ORC_MAX_ANG];
} orc_source;

typedef struct {
  int32_t K;
  int32_t n_threads;
  uint64_t n_packets;
  uint64_t first_packet;
  uint64_t seed;
  uint32_t stream_id;
  uint32_t max_scatter; /* a packet is killed at its collision number max_scatter+1 */
  uint32_t max_events;  /* flights per packet before it is ended */
  double w_threshold;   /* roulette when |W| < w_threshold |W0| */
  float roulette_p;     /* survival probability (FP32 so both paths compare alike) */
  /* discrete ordinates (Sec. 3.1's alternative to the harmonics): > 0 tallies t into
   * `sectors` equal angular sectors [m dth, (m+1) dth), dth = 2 pi / sectors, of theta in
   * [0, 2 pi) instead of the 2K+1 harmonics; 0: harmonics */
  uint32_t sectors;
  /* fixed != 0 (2D tally): every deposit term (t, t cos n theta, t sin n theta) is rounded to the nearest
   * multiple of 2^-fixed_q before it is summed, so that the sums are integers (in units of
   * 2^-fixed_q, exact in FP64 while below 2^53) and the sums of disjoint packet ranges add up
   * exactly -- the fixed-point form of the tally (the normalisation of Sec. 3.1 then applies) */
  int32_t fixed_q;
  uint32_t fixed;
  /* time_bins > 0 (2D, forward): the fluence resolved by the packet's path length since launch
   * (time of flight x c / n): bin b holds the track weight of the path-length interval
   * [b w, (b+1) w), w = time_bin_mm, the last bin everything beyond (T-1) w, so the bins sum to
   * a_0; tally [time_bins][nz][nx] instead of the harmonics */
  uint32_t time_bins;
  double time_bin_mm;
} orc_run;

typedef struct {
  uint64_t launched, flights, collisions, segments, escapes;
  uint64_t rr_kill, rr_survive, scatter_limit, event_limit;
  double launched_w, escaped_w, rr_net_w, absorbed_w, killed_w;
} orc_stats;

/* ---------------------------------------------------------------- Philox */
static void orc_philox_round(uint32_t c[4], const uint32_t k[2]) {
  const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
  const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
  const uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
  const uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
  const uint32_t n0 = hi1 ^ c[1] ^ k[0];
  const uint32_t n2 = hi0 ^ c[3] ^ k[1];
  c[0] = n0;
  c[1] = lo1;
  c[2] = n2;
  c[3] = lo0;
}

void orc_philox4x32_10(const uint32_t ctr[4], const uint32_t key[2], uint32_t out[4]) {
  uint32_t c[4] = {ctr[0], ctr[1], ctr[2], ctr[3]};
  uint32_t k[2] = {key[0], key[1]};
  for (int r = 0; r < 10; ++r) {
    orc_philox_round(c, k);
    k[0] += 0x9E3779B9u; /* Weyl key schedule */
    k[1] += 0xBB67AE85u;
  }
  memcpy(out, c, sizeof(c));
}

static double orc_u01(uint32_t x) { return ((double)(x >> 9) + 0.5) * (1.0 / 8388608.0); }

/* ------------------------------------------------------------ HG (Eq. 7) */
double orc_hg_angle(double g, double u) {
  return 2.0 * atan((1.0 - g) / (1.0 + g) * tan(M_PI * u));
}

/* 2D Henyey-Greenstein phase function of Eq. 6, P(dtheta). */
double orc_hg_phase(double g, double dtheta) {
  return (1.0 / (2.0 * M_PI)) * (1.0 - g * g) / (1.0 + g * g - 2.0 * g * cos(dtheta));
}

static double orc_wrap(double th) {
  while (th > M_PI) th -= 2.0 * M_PI;
  while (th <= -M_PI) th += 2.0 * M_PI;
  return th;
}

/* Direction angle of an angular point source: the theta in [0, 2 pi) with F(theta) = u, where
 * F(theta) = theta / (2 pi) + (1 / 2 pi) sum_n [c_n sin(n theta) + s_n (1 - cos(n theta))] / n is
 * the integral of its density from 0 (non-decreasing for a density >= 0), by bisection to the
 * last FP64 bits. */
static double orc_angle_sample(const orc_source *s, double u) {
  double lo = 0.0, hi = 2.0 * M_PI;
  for (int it = 0; it < 64; ++it) {
    const double mid = 0.5 * (lo + hi);
    double F = mid;
    for (int n = 1; n <= s->n_ang; ++n)
      F += (s->ang_c[n - 1] * sin(n * mid) + s->ang_s[n - 1] * (1.0 - cos(n * mid))) / n;
    F /= 2.0 * M_PI;
    if (F < u)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5 * (lo + hi);
}

/* --------------------------------------------- volumetric source sampling */
typedef struct {
  const float *q;     /* [nz][nx] signed source density */
  uint64_t *cdf;      /* inclusive prefix sum of quantised |q| */
  uint64_t total;
  double qmax;
} orc_volsrc;

static int orc_volsrc_build(orc_volsrc *vs, const float *q, int64_t npix) {
  vs->q = q;
  vs->cdf = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(npix > 0 ? npix : 1));
  if (!vs->cdf) return ORC_ERR_NOMEM;
  double qmax = 0.0;
  for (int64_t i = 0; i < npix; ++i) {
    double a = fabs((double)q[i]);
    if (a > qmax) qmax = a;
  }
  vs->qmax = qmax;
  uint64_t run = 0;
  for (int64_t i = 0; i < npix; ++i) {
    uint64_t w = 0;
    if (qmax > 0.0) w = (uint64_t)floor(fabs((double)q[i]) / qmax * 4294967296.0);
    run += w;
    vs->cdf[i] = run;
  }
  vs->total = run;
  return ORC_OK;
}

/* smallest i with cdf[i] > target */
static int64_t orc_volsrc_pick(const orc_volsrc *vs, int64_t npix, uint32_t w0, uint32_t w1) {
  const uint64_t r48 = ((uint64_t)w0 << 16) | (uint64_t)(w1 >> 16);
  const uint64_t target = (uint64_t)(((unsigned __int128)r48 * (unsigned __int128)vs->total) >> 48);
  int64_t lo = 0, hi = npix - 1;
  while (lo < hi) {
    int64_t mid = lo + (hi - lo) / 2;
    if (vs->cdf[mid] > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

/* ------------------------------------------------------------ one thread */
typedef struct {
  const orc_medium *med;
  const orc_source *src;
  const orc_volsrc *vol;
  const orc_run *run;
  int adjoint;
  uint64_t p_begin, p_end;
  double *tally;   /* [C][npix] sums of t cos/sin */
  double *sq;      /* [npix] sum over packets of (per-packet a_0 sum)^2, or NULL */
  double *pk;      /* [npix] current packet's a_0 sums */
  int64_t *touched;
  int64_t n_touched;
  orc_stats st;
} orc_job;

static void orc_deposit(orc_job *j, int64_t pix, double t, double theta_tally) {
  const int K = j->run->K;
  const int64_t npix = (int64_t)j->med->nx * j->med->nz;
  double *T = j->tally;
  if (j->run->sectors) { /* discrete ordinates: the sector holding theta */
    const uint32_t M = j->run->sectors;
    double th = fmod(theta_tally, 2.0 * M_PI);
    if (th < 0.0) th += 2.0 * M_PI;
    uint32_t sct = (uint32_t)(th * (M / (2.0 * M_PI)));
    if (sct >= M) sct = M - 1;
    T[(int64_t)sct * npix + pix] += t;
    if (j->sq) {
      if (j->pk[pix] == 0.0) j->touched[j->n_touched++] = pix;
      j->pk[pix] += t;
    }
    return;
  }
  if (j->run->fixed) { /* the same terms, each rounded to the quantum 2^-fixed_q */
    const int q = j->run->fixed_q;
    T[pix] += nearbyint(ldexp(t, q));
    for (int n = 1; n <= K; ++n) {
      T[(int64_t)(2 * n - 1) * npix + pix] += nearbyint(ldexp(t * cos(n * theta_tally), q));
      T[(int64_t)(2 * n) * npix + pix] += nearbyint(ldexp(t * sin(n * theta_tally), q));
    }
  } else {
    T[pix] += t; /* a_0: Eq. 9 */
    for (int n = 1; n <= K; ++n) {
      T[(int64_t)(2 * n - 1) * npix + pix] += t * cos(n * theta_tally); /* a_n: Eq. 10 */
      T[(int64_t)(2 * n) * npix + pix] += t * sin(n * theta_tally);     /* b_n: Eq. 11 */
    }
  }
  if (j->sq) {
    if (j->pk[pix] == 0.0) j->touched[j->n_touched++] = pix;
    j->pk[pix] += t;
  }
}

/* Time-resolved deposit of a segment of length l that starts at path length L0 with weight W:
 * the piece of the segment inside the path-length bin [b w, (b+1) w) (the last bin open-ended),
 * s in [s1, s2) measured along the segment, holds the track weight int W e^{-mu_a s} ds =
 * W (e^{-mu_a s1} - e^{-mu_a s2}) / mu_a (= W (s2 - s1) when mu_a = 0). */
static void orc_deposit_timed(orc_job *j, int64_t pix, double W, double mua, double L0, double l) {
  const int64_t npix = (int64_t)j->med->nx * j->med->nz;
  const uint32_t T = j->run->time_bins;
  const double w = j->run->time_bin_mm;
  double sum = 0.0;
  /* from one bin before floor(L0 / w), so that a quotient rounded up loses no sliver */
  for (uint32_t b = (uint32_t)fmax(fmin(floor(L0 / w), (double)(T - 1)) - 1.0, 0.0);; ++b) {
    const double s1 = fmax(b * w - L0, 0.0);
    const double s2 = (b + 1 == T) ? l : fmin((b + 1) * w - L0, l);
    if (s2 > s1) {
      const double tp = mua > 0.0 ? W * (exp(-mua * s1) - exp(-mua * s2)) / mua : W * (s2 - s1);
      j->tally[(int64_t)b * npix + pix] += tp;
      sum += tp;
    }
    if (s2 >= l || b + 1 == T) break;
  }
  if (j->sq && sum != 0.0) {
    if (j->pk[pix] == 0.0) j->touched[j->n_touched++] = pix;
    j->pk[pix] += sum;
  }
}

static void orc_packet(orc_job *j, uint64_t p) {
  const orc_medium *m = j->med;
  const orc_run *r = j->run;
  const int nx = m->nx, nz = m->nz;
  const double dx = m->dx;
  const int64_t npix = (int64_t)nx * nz;
  const uint32_t key[2] = {(uint32_t)r->seed, (uint32_t)(r->seed >> 32) ^ r->stream_id};
  uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0u, 0u};
  uint32_t b0[4], b1[4], b[4];
  orc_philox4x32_10(ctr, key, b0);
  ctr[2] = 1u;
  orc_philox4x32_10(ctr, key, b1);

  /* ---- launch */
  double x, z, theta, W0 = 1.0;
  int ix, iz;
  const orc_source *s = j->src;
  switch (j->vol ? ORC_VOLUME : s->kind) {
    case ORC_PENCIL:
      x = s->x0;
      z = s->z0;
      theta = atan2(s->dir_x, s->dir_z);
      break;
    case ORC_LINE: {
      const double u = orc_u01(b0[0]);
      x = s->x0 + u * (s->x1 - s->x0);
      z = s->z0 + u * (s->z1 - s->z0);
      theta = atan2(s->dir_x, s->dir_z);
      break;
    }
    case ORC_ISO_POINT:
      x = s->x0;
      z = s->z0;
      theta = orc_wrap(2.0 * M_PI * orc_u01(b0[2]));
      break;
    case ORC_ANGULAR_POINT:
      x = s->x0;
      z = s->z0;
      theta = orc_wrap(orc_angle_sample(s, orc_u01(b0[2])));
      break;
    default: { /* ORC_VOLUME */
      const int64_t pix = orc_volsrc_pick(j->vol, npix, b0[0], b0[1]);
      const int pxi = (int)(pix % nx), pzi = (int)(pix / nx);
      x = (pxi + orc_u01(b1[0])) * dx;
      z = (pzi + orc_u01(b1[1])) * dx;
      theta = orc_wrap(2.0 * M_PI * orc_u01(b0[2]));
      W0 = j->vol->q[pix] < 0.0f ? -1.0 : 1.0;
      break;
    }
  }
  double W = W0;
  j->st.launched++;
  j->st.launched_w += W0;

  const double Wmax = nx * dx, Dmax = nz * dx;
  if (!(x >= 0.0 && x <= Wmax && z >= 0.0 && z <= Dmax)) {
    j->st.escapes++;
    j->st.escaped_w += W;
    return;
  }
  ix = (int)floor(x / dx);
  iz = (int)floor(z / dx);
  if (ix >= nx) ix = nx - 1;
  if (iz >= nz) iz = nz - 1;

  uint32_t flight = 0, n_scatter = 0;
  double plen = 0.0; /* path length since launch (time-resolved tally) */
  for (;;) {
    /* ---- a new free flight: s = -ln(U)/mu_s, as optical depth tau */
    if (flight >= r->max_events) {
      j->st.event_limit++;
      j->st.killed_w += W;
      break;
    }
    ++flight;
    j->st.flights++;
    ctr[2] = flight + 1u;
    orc_philox4x32_10(ctr, key, b);
    double tau = -log(orc_u01(b[0]));
    int escaped = 0;
    for (;;) {
      const int64_t pix = (int64_t)iz * nx + ix;
      const double mua = m->mua[pix], mus = m->mus[pix];
      const double sx = sin(theta), sz = cos(theta);
      double dist_x = INFINITY, dist_z = INFINITY;
      if (sx > 0.0) dist_x = ((ix + 1) * dx - x) / sx;
      if (sx < 0.0) dist_x = (ix * dx - x) / sx;
      if (sz > 0.0) dist_z = ((iz + 1) * dx - z) / sz;
      if (sz < 0.0) dist_z = (iz * dx - z) / sz;
      if (dist_x < 0.0) dist_x = 0.0;
      if (dist_z < 0.0) dist_z = 0.0;
      const double d_edge = dist_x < dist_z ? dist_x : dist_z;
      const double d_coll = mus > 0.0 ? tau / mus : INFINITY;
      const int collide = d_coll < d_edge;
      const double l = collide ? d_coll : d_edge;
      /* deposit the track weight of this pixel segment (Sec. 3 + Eq. 9-11) */
      const double t = mua > 0.0 ? -W * expm1(-mua * l) / mua : W * l;
      if (r->time_bins) {
        orc_deposit_timed(j, pix, W, mua, plen, l);
        plen += l;
      } else if (t != 0.0) {
        orc_deposit(j, pix, t, j->adjoint ? theta + M_PI : theta);
      }
      j->st.segments++;
      const double W_next = W * exp(-mua * l); /* W <- W exp(-mu_a s) (Sec. 3) */
      j->st.absorbed_w += W - W_next;          /* weight lost, booked apart from t */
      W = W_next;
      x += l * sx;
      z += l * sz;
      if (collide) break;
      tau -= mus * l;
      if (dist_x <= dist_z) { /* ties: cross x first, z follows as a zero-length segment */
        if (sx > 0.0) {
          ++ix;
          x = ix * dx;
        } else {
          x = ix * dx;
          --ix;
        }
      } else {
        if (sz > 0.0) {
          ++iz;
          z = iz * dx;
        } else {
          z = iz * dx;
          --iz;
        }
      }
      if (ix < 0 || ix >= nx || iz < 0 || iz >= nz) {
        escaped = 1;
        break;
      }
    }
    if (escaped) {
      j->st.escapes++;
      j->st.escaped_w += W;
      break;
    }
    /* ---- collision */
    j->st.collisions++;
    if (n_scatter >= r->max_scatter) {
      j->st.scatter_limit++;
      j->st.killed_w += W;
      break;
    }
    theta = orc_wrap(theta + orc_hg_angle(m->g, orc_u01(b[1])));
    ++n_scatter;
    /* ---- threshold on |W| with Russian roulette */
    if (fabs(W) < r->w_threshold * fabs(W0)) {
      const double p = (double)r->roulette_p;
      if (orc_u01(b[2]) < p) {
        const double Wn = W / p;
        j->st.rr_survive++;
        j->st.rr_net_w += Wn - W;
        W = Wn;
      } else {
        j->st.rr_kill++;
        j->st.rr_net_w -= W;
        break;
      }
    }
  }
}

static void *orc_worker(void *arg) {
  orc_job *j = (orc_job *)arg;
  for (uint64_t p = j->p_begin; p < j->p_end; ++p) {
    orc_packet(j, p);
    if (j->sq) {
      for (int64_t k = 0; k < j->n_touched; ++k) {
        const int64_t pix = j->touched[k];
        j->sq[pix] += j->pk[pix] * j->pk[pix];
        j->pk[pix] = 0.0;
      }
      j->n_touched = 0;
    }
  }
  return NULL;
}

static int orc_check(const orc_medium *m, const orc_run *r) {
  if (!m || !r || !m->mua || !m->mus) return ORC_ERR_ARG;
  if (m->nx <= 0 || m->nz <= 0 || !(m->dx > 0.0)) return ORC_ERR_ARG;
  if (!(m->g > -1.0 && m->g < 1.0)) return ORC_ERR_ARG;
  if (r->K < 0 || r->K > 256 || r->n_threads <= 0 || r->sectors > 4096) return ORC_ERR_ARG;
  if (r->time_bins > 4096 || (r->time_bins && (r->sectors || !(r->time_bin_mm > 0.0)))) return ORC_ERR_ARG;
  if (!(r->roulette_p > 0.0f && r->roulette_p <= 1.0f)) return ORC_ERR_ARG;
  const int64_t npix = (int64_t)m->nx * m->nz;
  for (int64_t i = 0; i < npix; ++i)
    if (!(m->mua[i] >= 0.0) || !(m->mus[i] >= 0.0)) return ORC_ERR_ARG;
  return ORC_OK;
}

/*
 * Runs packets [first_packet, first_packet + n_packets) and ADDS raw sums to
 * tally ([2K+1][nz][nx], sums of t cos(n theta), t sin(n theta), no
 * normalisation; with sectors > 0, [sectors][nz][nx] sums of t per sector) and to sq ([nz][nx], sums over packets of the squared
 * per-packet a_0 sum; may be NULL).  Normalisation is done by the caller
 * (S / (N_p dx^2)).  Threads take equal contiguous packet ranges; their tallies
 * are summed in thread order.
 */
static int orc_run_packets(const orc_medium *m, const orc_source *s, const orc_volsrc *vol,
                           const orc_run *r, int adjoint, double *tally, double *sq, orc_stats *st) {
  const int64_t npix = (int64_t)m->nx * m->nz;
  const int64_t C = r->time_bins ? (int64_t)r->time_bins : r->sectors ? (int64_t)r->sectors : 2 * (int64_t)r->K + 1;
  const int nt = r->n_threads;
  orc_job *jobs = (orc_job *)calloc((size_t)nt, sizeof(orc_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return ORC_ERR_NOMEM;
  }
  int rc = ORC_OK;
  for (int k = 0; k < nt; ++k) {
    orc_job *j = &jobs[k];
    j->med = m;
    j->src = s;
    j->vol = vol;
    j->run = r;
    j->adjoint = adjoint;
    j->p_begin = r->first_packet + r->n_packets * (uint64_t)k / (uint64_t)nt;
    j->p_end = r->first_packet + r->n_packets * (uint64_t)(k + 1) / (uint64_t)nt;
    j->tally = (double *)calloc((size_t)(C * npix), sizeof(double));
    if (!j->tally) rc = ORC_ERR_NOMEM;
    if (sq) {
      j->sq = (double *)calloc((size_t)npix, sizeof(double));
      j->pk = (double *)calloc((size_t)npix, sizeof(double));
      j->touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)npix);
      if (!j->sq || !j->pk || !j->touched) rc = ORC_ERR_NOMEM;
    }
  }
  if (rc == ORC_OK) {
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, orc_worker, &jobs[k]);
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
    memset(st, 0, sizeof(*st));
    for (int k = 0; k < nt; ++k) {
      orc_job *j = &jobs[k];
      for (int64_t i = 0; i < C * npix; ++i) tally[i] += j->tally[i];
      if (sq)
        for (int64_t i = 0; i < npix; ++i) sq[i] += j->sq[i];
      st->launched += j->st.launched;
      st->flights += j->st.flights;
      st->collisions += j->st.collisions;
      st->segments += j->st.segments;
      st->escapes += j->st.escapes;
      st->rr_kill += j->st.rr_kill;
      st->rr_survive += j->st.rr_survive;
      st->scatter_limit += j->st.scatter_limit;
      st->event_limit += j->st.event_limit;
      st->launched_w += j->st.launched_w;
      st->escaped_w += j->st.escaped_w;
      st->rr_net_w += j->st.rr_net_w;
      st->absorbed_w += j->st.absorbed_w;
      st->killed_w += j->st.killed_w;
    }
  }
  for (int k = 0; k < nt; ++k) {
    free(jobs[k].tally);
    free(jobs[k].sq);
    free(jobs[k].pk);
    free(jobs[k].touched);
  }
  free(jobs);
  free(th);
  return rc;
}

/* Forward run from a boundary / point source (Sec. 3).  Adds raw sums. */
int orc_forward_raw(const orc_medium *m, const orc_source *s, const orc_run *r, double *tally,
                    double *sq, orc_stats *st) {
  int rc = orc_check(m, r);
  if (rc) return rc;
  if (!s || !tally || !st || s->kind < ORC_PENCIL || s->kind > ORC_ANGULAR_POINT) return ORC_ERR_ARG;
  if (s->kind == ORC_ANGULAR_POINT && (s->n_ang < 0 || s->n_ang > ORC_MAX_ANG)) return ORC_ERR_ARG;
  return orc_run_packets(m, s, NULL, r, 0, tally, sq, st);
}

/*
 * Adjoint run (Sec. 4, Sec. 6) from the signed volumetric source q ([nz][nx],
 * per unit area and unit angle).  Adds raw sums; *source_strength receives
 * S = 2 pi dx^2 qmax total / 2^32 (the strength that the sampled distribution
 * represents), by which the caller scales.  Set adjoint = 0 to tally at theta
 * (a plain forward run from the same volumetric source).
 */
int orc_volume_raw(const orc_medium *m, const float *q, const orc_run *r, int adjoint,
                   double *tally, double *sq, orc_stats *st, double *source_strength) {
  int rc = orc_check(m, r);
  if (rc) return rc;
  if (!q || !tally || !st || !source_strength) return ORC_ERR_ARG;
  const int64_t npix = (int64_t)m->nx * m->nz;
  orc_volsrc vs;
  rc = orc_volsrc_build(&vs, q, npix);
  if (rc) return rc;
  *source_strength = 2.0 * M_PI * m->dx * m->dx * vs.qmax * (double)vs.total / 4294967296.0;
  if (vs.total == 0) {
    memset(st, 0, sizeof(*st));
    free(vs.cdf);
    return ORC_OK;
  }
  rc = orc_run_packets(m, NULL, &vs, r, adjoint ? 1 : 0, tally, sq, st);
  free(vs.cdf);
  return rc;
}

/* Pixel drawn for packet p by the volumetric source sampler (for tests). */
int64_t orc_volume_pick(const float *q, int64_t npix, uint64_t seed, uint32_t stream_id, uint64_t p) {
  orc_volsrc vs;
  if (orc_volsrc_build(&vs, q, npix)) return -1;
  const uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32) ^ stream_id};
  const uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0u, 0u};
  uint32_t b0[4];
  orc_philox4x32_10(ctr, key, b0);
  int64_t pix = vs.total ? orc_volsrc_pick(&vs, npix, b0[0], b0[1]) : -1;
  free(vs.cdf);
  return pix;
}

/* ======================================================================
 * 3D: the extension the paper names (Sec. 3.1: "in 3D ... spherical
 * harmonics").  Voxels [nz][ny][nx] of side dx; direction
 * s = (sin th cos ph, sin th sin ph, cos th), th from +z; the 3D
 * Henyey-Greenstein phase function; the tally holds c_lm = sum t Y_lm(s)
 * over orthonormal real spherical harmonics (index l^2 + l + m, l <= L), so
 * that phi(s) = sum c_lm Y_lm(s) and the fluence is sqrt(4 pi) c_00.
 * Adjoint runs tally at -s: Y_lm(-s) = (-1)^l Y_lm(s).
 * Random numbers as in 2D; launch event 0: words 0, 1 -> the voxel of a
 * volumetric source, word 2 -> cos th = 2u - 1, word 3 -> ph = 2 pi u
 * (isotropic directions); event 1: words 0..2 -> the position in the voxel;
 * flight k >= 1, event k+1: word 0 -> free path, 1 -> HG cos, 2 ->
 * roulette, 3 -> azimuth of the scattering.
 * ====================================================================== */
#define ORC3_MAX_L 16

typedef struct {
  int32_t nx, ny, nz;
  double dx;
  double g;
  const double *mua; /* [nz][ny][nx] */
  const double *mus;
} orc3_medium;

typedef struct {
  int32_t kind;            /* ORC_PENCIL or ORC_ISO_POINT */
  double x0, y0, z0;       /* mm */
  double dir_x, dir_y, dir_z; /* unit direction (pencil) */
  double power;
} orc3_source;

/* Orthonormal real spherical harmonics Y_lm(s) for l <= L at index l^2 + l + m:
 * Y_l0 = N_l0 P_l(cos th), Y_lm = sqrt 2 N_lm P_l^m(cos th) cos(m ph) (m > 0),
 * Y_l,-m = sqrt 2 N_lm P_l^m(cos th) sin(m ph), N_lm^2 = (2l+1)/(4 pi) (l-m)!/(l+m)!,
 * with the associated Legendre functions from their standard three-term
 * recurrence in l (no Condon-Shortley sign: any fixed sign is orthonormal). */
void orc3_sh(int L, double sx, double sy, double sz, double *Y) {
  const double ct = sz, st = sqrt(fmax(0.0, 1.0 - sz * sz));
  const double ph = atan2(sy, sx);
  for (int m = 0; m <= L; ++m) {
    /* P_m^m = (2m-1)!! st^m */
    double pmm = 1.0;
    for (int k = 1; k <= m; ++k) pmm *= (2.0 * k - 1.0) * st;
    double plm2 = 0.0, plm1 = pmm;
    for (int l = m; l <= L; ++l) {
      double plm;
      if (l == m)
        plm = pmm;
      else if (l == m + 1)
        plm = ct * (2.0 * m + 1.0) * pmm;
      else
        plm = ((2.0 * l - 1.0) * ct * plm1 - (l + m - 1.0) * plm2) / (double)(l - m);
      if (l > m) {
        plm2 = plm1;
        plm1 = plm;
      }
      double ratio = 1.0; /* (l-m)!/(l+m)! */
      for (int k = l - m + 1; k <= l + m; ++k) ratio /= (double)k;
      const double N = sqrt((2.0 * l + 1.0) / (4.0 * M_PI) * ratio);
      if (m == 0) {
        Y[l * l + l] = N * plm;
      } else {
        Y[l * l + l + m] = M_SQRT2 * N * plm * cos(m * ph);
        Y[l * l + l - m] = M_SQRT2 * N * plm * sin(m * ph);
      }
    }
  }
}

/* cos of the scattering angle of the 3D Henyey-Greenstein phase function
 * p(cos) = (1 - g^2) / (4 pi (1 + g^2 - 2 g cos)^(3/2)), by inverting its
 * cumulative distribution at u. */
double orc3_hg_cos(double g, double u) {
  if (g == 0.0) return 2.0 * u - 1.0;
  const double f = (1.0 - g * g) / (1.0 - g + 2.0 * g * u);
  double c = (1.0 + g * g - f * f) / (2.0 * g);
  if (c > 1.0) c = 1.0;
  if (c < -1.0) c = -1.0;
  return c;
}

/* Turn the unit direction u by polar angle (cos ct) and azimuth psi about it,
 * in the orthonormal frame (t1, t2, u) of Duff et al., "Building an
 * orthonormal basis, revisited" (JCGT 2017). */
static void orc3_turn(double *ux, double *uy, double *uz, double ct, double psi) {
  const double sgn = *uz >= 0.0 ? 1.0 : -1.0;
  const double a = -1.0 / (sgn + *uz), b = *ux * *uy * a;
  const double t1x = 1.0 + sgn * *ux * *ux * a, t1y = sgn * b, t1z = -sgn * *ux;
  const double t2x = b, t2y = sgn + *uy * *uy * a, t2z = -*uy;
  const double st = sqrt(fmax(0.0, 1.0 - ct * ct)), cp = cos(psi), sp = sin(psi);
  double nx = ct * *ux + st * (cp * t1x + sp * t2x);
  double ny = ct * *uy + st * (cp * t1y + sp * t2y);
  double nz = ct * *uz + st * (cp * t1z + sp * t2z);
  const double n = sqrt(nx * nx + ny * ny + nz * nz);
  *ux = nx / n;
  *uy = ny / n;
  *uz = nz / n;
}

typedef struct {
  const orc3_medium *med;
  const orc3_source *src;
  const orc_volsrc *vol;
  const orc_run *run;
  int adjoint;
  uint64_t p_begin, p_end;
  double *tally; /* [C][nvox] */
  double *sq, *pk;
  int64_t *touched;
  int64_t n_touched;
  orc_stats st;
} orc3_job;

static void orc3_deposit(orc3_job *j, int64_t v, double t, double sx, double sy, double sz) {
  const int L = j->run->K;
  const int64_t nvox = (int64_t)j->med->nx * j->med->ny * j->med->nz;
  double Y[(ORC3_MAX_L + 1) * (ORC3_MAX_L + 1)];
  if (j->adjoint)
    orc3_sh(L, -sx, -sy, -sz, Y);
  else
    orc3_sh(L, sx, sy, sz, Y);
  for (int c = 0; c < (L + 1) * (L + 1); ++c) j->tally[(int64_t)c * nvox + v] += t * Y[c];
  if (j->sq) {
    if (j->pk[v] == 0.0) j->touched[j->n_touched++] = v;
    j->pk[v] += t;
  }
}

static void orc3_packet(orc3_job *j, uint64_t p) {
  const orc3_medium *m = j->med;
  const orc_run *r = j->run;
  const int nx = m->nx, ny = m->ny, nz = m->nz;
  const double dx = m->dx;
  const int64_t nvox = (int64_t)nx * ny * nz;
  const uint32_t key[2] = {(uint32_t)r->seed, (uint32_t)(r->seed >> 32) ^ r->stream_id};
  uint32_t ctr[4] = {(uint32_t)p, (uint32_t)(p >> 32), 0u, 0u};
  uint32_t b0[4], b1[4], b[4];
  orc_philox4x32_10(ctr, key, b0);
  ctr[2] = 1u;
  orc_philox4x32_10(ctr, key, b1);

  double x, y, z, ux, uy, uz, W0 = 1.0;
  if (j->vol) {
    const int64_t v = orc_volsrc_pick(j->vol, nvox, b0[0], b0[1]);
    const int vx = (int)(v % nx), vy = (int)((v / nx) % ny), vz = (int)(v / ((int64_t)nx * ny));
    x = (vx + orc_u01(b1[0])) * dx;
    y = (vy + orc_u01(b1[1])) * dx;
    z = (vz + orc_u01(b1[2])) * dx;
    W0 = j->vol->q[v] < 0.0f ? -1.0 : 1.0;
  } else {
    x = j->src->x0;
    y = j->src->y0;
    z = j->src->z0;
  }
  if (j->vol || j->src->kind == ORC_ISO_POINT) {
    const double ct = 2.0 * orc_u01(b0[2]) - 1.0, st = sqrt(fmax(0.0, 1.0 - ct * ct));
    const double ph = 2.0 * M_PI * orc_u01(b0[3]);
    ux = st * cos(ph);
    uy = st * sin(ph);
    uz = ct;
  } else {
    ux = j->src->dir_x;
    uy = j->src->dir_y;
    uz = j->src->dir_z;
  }
  double W = W0;
  j->st.launched++;
  j->st.launched_w += W0;
  if (!(x >= 0.0 && x <= nx * dx && y >= 0.0 && y <= ny * dx && z >= 0.0 && z <= nz * dx)) {
    j->st.escapes++;
    j->st.escaped_w += W;
    return;
  }
  int ix = (int)floor(x / dx), iy = (int)floor(y / dx), iz = (int)floor(z / dx);
  if (ix >= nx) ix = nx - 1;
  if (iy >= ny) iy = ny - 1;
  if (iz >= nz) iz = nz - 1;

  uint32_t flight = 0, n_scatter = 0;
  for (;;) {
    if (flight >= r->max_events) {
      j->st.event_limit++;
      j->st.killed_w += W;
      break;
    }
    ++flight;
    j->st.flights++;
    ctr[2] = flight + 1u;
    orc_philox4x32_10(ctr, key, b);
    double tau = -log(orc_u01(b[0]));
    int escaped = 0;
    for (;;) {
      const int64_t v = ((int64_t)iz * ny + iy) * nx + ix;
      const double mua = m->mua[v], mus = m->mus[v];
      double dxf = INFINITY, dyf = INFINITY, dzf = INFINITY;
      if (ux > 0.0) dxf = ((ix + 1) * dx - x) / ux;
      if (ux < 0.0) dxf = (ix * dx - x) / ux;
      if (uy > 0.0) dyf = ((iy + 1) * dx - y) / uy;
      if (uy < 0.0) dyf = (iy * dx - y) / uy;
      if (uz > 0.0) dzf = ((iz + 1) * dx - z) / uz;
      if (uz < 0.0) dzf = (iz * dx - z) / uz;
      if (dxf < 0.0) dxf = 0.0;
      if (dyf < 0.0) dyf = 0.0;
      if (dzf < 0.0) dzf = 0.0;
      double d_face = dxf;
      int axis = 0; /* ties: x first, then y, then z */
      if (dyf < d_face) {
        d_face = dyf;
        axis = 1;
      }
      if (dzf < d_face) {
        d_face = dzf;
        axis = 2;
      }
      const double d_coll = mus > 0.0 ? tau / mus : INFINITY;
      const int collide = d_coll < d_face;
      const double l = collide ? d_coll : d_face;
      const double t = mua > 0.0 ? -W * expm1(-mua * l) / mua : W * l;
      if (t != 0.0) orc3_deposit(j, v, t, ux, uy, uz);
      j->st.segments++;
      const double W_next = W * exp(-mua * l);
      j->st.absorbed_w += W - W_next;
      W = W_next;
      x += l * ux;
      y += l * uy;
      z += l * uz;
      if (collide) break;
      tau -= mus * l;
      if (axis == 0) {
        if (ux > 0.0) {
          ++ix;
          x = ix * dx;
        } else {
          x = ix * dx;
          --ix;
        }
      } else if (axis == 1) {
        if (uy > 0.0) {
          ++iy;
          y = iy * dx;
        } else {
          y = iy * dx;
          --iy;
        }
      } else {
        if (uz > 0.0) {
          ++iz;
          z = iz * dx;
        } else {
          z = iz * dx;
          --iz;
        }
      }
      if (ix < 0 || ix >= nx || iy < 0 || iy >= ny || iz < 0 || iz >= nz) {
        escaped = 1;
        break;
      }
    }
    if (escaped) {
      j->st.escapes++;
      j->st.escaped_w += W;
      break;
    }
    j->st.collisions++;
    if (n_scatter >= r->max_scatter) {
      j->st.scatter_limit++;
      j->st.killed_w += W;
      break;
    }
    orc3_turn(&ux, &uy, &uz, orc3_hg_cos(m->g, orc_u01(b[1])), 2.0 * M_PI * orc_u01(b[3]));
    ++n_scatter;
    if (fabs(W) < r->w_threshold * fabs(W0)) {
      const double pr = (double)r->roulette_p;
      if (orc_u01(b[2]) < pr) {
        const double Wn = W / pr;
        j->st.rr_survive++;
        j->st.rr_net_w += Wn - W;
        W = Wn;
      } else {
        j->st.rr_kill++;
        j->st.rr_net_w -= W;
        break;
      }
    }
  }
}

static void *orc3_worker(void *arg) {
  orc3_job *j = (orc3_job *)arg;
  for (uint64_t p = j->p_begin; p < j->p_end; ++p) {
    orc3_packet(j, p);
    if (j->sq) {
      for (int64_t k = 0; k < j->n_touched; ++k) {
        const int64_t v = j->touched[k];
        j->sq[v] += j->pk[v] * j->pk[v];
        j->pk[v] = 0.0;
      }
      j->n_touched = 0;
    }
  }
  return NULL;
}

static int orc3_check(const orc3_medium *m, const orc_run *r) {
  if (!m || !r || !m->mua || !m->mus) return ORC_ERR_ARG;
  if (m->nx <= 0 || m->ny <= 0 || m->nz <= 0 || !(m->dx > 0.0)) return ORC_ERR_ARG;
  if (!(m->g > -1.0 && m->g < 1.0)) return ORC_ERR_ARG;
  if (r->K < 0 || r->K > ORC3_MAX_L || r->n_threads <= 0 || r->sectors) return ORC_ERR_ARG;
  if (!(r->roulette_p > 0.0f && r->roulette_p <= 1.0f)) return ORC_ERR_ARG;
  const int64_t nvox = (int64_t)m->nx * m->ny * m->nz;
  for (int64_t i = 0; i < nvox; ++i)
    if (!(m->mua[i] >= 0.0) || !(m->mus[i] >= 0.0)) return ORC_ERR_ARG;
  return ORC_OK;
}

/* Packets [first, first + n) in equal contiguous ranges over threads; ADDS raw
 * sums to tally ([(L+1)^2][nz][ny][nx]) and sq ([nz][ny][nx] or NULL), thread
 * tallies summed in thread order. */
static int orc3_run_packets(const orc3_medium *m, const orc3_source *s, const orc_volsrc *vol, const orc_run *r,
                            int adjoint, double *tally, double *sq, orc_stats *st) {
  const int64_t nvox = (int64_t)m->nx * m->ny * m->nz;
  const int64_t C = (int64_t)(r->K + 1) * (r->K + 1);
  const int nt = r->n_threads;
  orc3_job *jobs = (orc3_job *)calloc((size_t)nt, sizeof(orc3_job));
  pthread_t *th = (pthread_t *)calloc((size_t)nt, sizeof(pthread_t));
  if (!jobs || !th) {
    free(jobs);
    free(th);
    return ORC_ERR_NOMEM;
  }
  int rc = ORC_OK;
  for (int k = 0; k < nt; ++k) {
    orc3_job *j = &jobs[k];
    j->med = m;
    j->src = s;
    j->vol = vol;
    j->run = r;
    j->adjoint = adjoint;
    j->p_begin = r->first_packet + r->n_packets * (uint64_t)k / (uint64_t)nt;
    j->p_end = r->first_packet + r->n_packets * (uint64_t)(k + 1) / (uint64_t)nt;
    j->tally = (double *)calloc((size_t)(C * nvox), sizeof(double));
    if (!j->tally) rc = ORC_ERR_NOMEM;
    if (sq) {
      j->sq = (double *)calloc((size_t)nvox, sizeof(double));
      j->pk = (double *)calloc((size_t)nvox, sizeof(double));
      j->touched = (int64_t *)malloc(sizeof(int64_t) * (size_t)nvox);
      if (!j->sq || !j->pk || !j->touched) rc = ORC_ERR_NOMEM;
    }
  }
  if (rc == ORC_OK) {
    for (int k = 0; k < nt; ++k) pthread_create(&th[k], NULL, orc3_worker, &jobs[k]);
    for (int k = 0; k < nt; ++k) pthread_join(th[k], NULL);
    memset(st, 0, sizeof(*st));
    for (int k = 0; k < nt; ++k) {
      orc3_job *j = &jobs[k];
      for (int64_t i = 0; i < C * nvox; ++i) tally[i] += j->tally[i];
      if (sq)
        for (int64_t i = 0; i < nvox; ++i) sq[i] += j->sq[i];
      st->launched += j->st.launched;
      st->flights += j->st.flights;
      st->collisions += j->st.collisions;
      st->segments += j->st.segments;
      st->escapes += j->st.escapes;
      st->rr_kill += j->st.rr_kill;
      st->rr_survive += j->st.rr_survive;
      st->scatter_limit += j->st.scatter_limit;
      st->event_limit += j->st.event_limit;
      st->launched_w += j->st.launched_w;
      st->escaped_w += j->st.escaped_w;
      st->rr_net_w += j->st.rr_net_w;
      st->absorbed_w += j->st.absorbed_w;
      st->killed_w += j->st.killed_w;
    }
  }
  for (int k = 0; k < nt; ++k) {
    free(jobs[k].tally);
    free(jobs[k].sq);
    free(jobs[k].pk);
    free(jobs[k].touched);
  }
  free(jobs);
  free(th);
  return rc;
}

/* 3D forward run from a pencil or isotropic point source.  Adds raw sums. */
int orc3_forward_raw(const orc3_medium *m, const orc3_source *s, const orc_run *r, double *tally, double *sq,
                     orc_stats *st) {
  int rc = orc3_check(m, r);
  if (rc) return rc;
  if (!s || !tally || !st || (s->kind != ORC_PENCIL && s->kind != ORC_ISO_POINT)) return ORC_ERR_ARG;
  return orc3_run_packets(m, s, NULL, r, 0, tally, sq, st);
}

/* 3D run from the signed volumetric isotropic source q ([nz][ny][nx], per unit
 * volume and unit solid angle); S = 4 pi dx^3 qmax total / 2^32.  adjoint = 1
 * tallies at -s. */
int orc3_volume_raw(const orc3_medium *m, const float *q, const orc_run *r, int adjoint, double *tally, double *sq,
                    orc_stats *st, double *source_strength) {
  int rc = orc3_check(m, r);
  if (rc) return rc;
  if (!q || !tally || !st || !source_strength) return ORC_ERR_ARG;
  const int64_t nvox = (int64_t)m->nx * m->ny * m->nz;
  orc_volsrc vs;
  rc = orc_volsrc_build(&vs, q, nvox);
  if (rc) return rc;
  *source_strength = 4.0 * M_PI * m->dx * m->dx * m->dx * vs.qmax * (double)vs.total / 4294967296.0;
  if (vs.total == 0) {
    memset(st, 0, sizeof(*st));
    free(vs.cdf);
    return ORC_OK;
  }
  rc = orc3_run_packets(m, NULL, &vs, r, adjoint ? 1 : 0, tally, sq, st);
  free(vs.cdf);
  return rc;
}
