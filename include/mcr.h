/*
 * mcr.h -- C ABI of libmcr: GPU (sm_103a) forward and adjoint harmonic radiance Monte Carlo,
 * after Hochuli, Powell, Arridge & Cox, "Quantitative photoacoustic tomography using forward
 * and adjoint Monte Carlo models of radiance" (arXiv 1608.05238).
 *
 * All array arguments are DEVICE pointers owned by the caller unless a comment says "host".
 * Maps are row-major [nz][nx] (x = column = lateral, z = row = depth, z = 0 the top edge;
 * pixel (ix, iz) covers [ix dx, (ix+1) dx) x [iz dx, (iz+1) dx)).  Directions are angles theta
 * from the +z axis, s = (sin theta, cos theta) = (s_x, s_z).  Coefficient arrays are
 * channel-major [2K+1][nz][nx] FP32 with channel 0 = a_0, 2n-1 = a_n, 2n = b_n (Sec. 3.1,
 * Eqs. 8-11), normalised so that phi(x, theta) = a_0/(2 pi) + (1/pi) sum (a_n cos n theta +
 * b_n sin n theta) is the radiance and a_0 the fluence.  Units: mm and 1/mm.
 *
 * Calls are asynchronous on `stream` (a cudaStream_t passed as void*; NULL = legacy default
 * stream) unless a `stats` pointer is given, in which case the call synchronises that stream
 * to fill it, or the run takes the sorted-record deposit (one problem whose fixed-point tally
 * exceeds 256 MB, see mcr_launch.deposit), which synchronises once per chunk of packets.  Every call returns MCR_OK (0) or a negative status; no C++ exception crosses the
 * ABI.  Errors found on the device (negative or NaN mu, a packet that hit its event cap, a tally
 * near overflow) are latched per device and returned by the next call that synchronises
 * (a call with stats != NULL, or mc_check).
 *
 * The library keeps one grow-only workspace per device (fixed-point tallies, packed medium,
 * source CDF, counters), allocated with cudaMalloc on first use and freed by
 * mc_release_workspace().  Calls that share a device share that workspace: calls on different
 * streams of one device must not overlap in time.
 */
#ifndef MCR_H
#define MCR_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define MCR_OK 0
#define MCR_ERR_ARG (-1)            /* bad argument (shape, pointer, range) */
#define MCR_ERR_CUDA (-2)           /* a CUDA runtime call failed */
#define MCR_ERR_NOMEM (-3)          /* workspace allocation failed */
#define MCR_ERR_EVENT_LIMIT (-4)    /* a packet reached max_events flights and was ended */
#define MCR_ERR_TALLY_OVERFLOW (-5) /* a fixed-point tally came within 2 bits of overflow */
#define MCR_ERR_MEDIUM (-6)         /* the device medium holds a negative or non-finite mu */
#define MCR_ERR_SCRATCH (-7)        /* problem too large for mc_forward_noalloc's fixed scratch */
#define MCR_ERR_CHECK (-8)          /* checked build only: an out-of-range index or a non-finite weight was
                                       found on the device (the access was skipped) */

#define MCR_PENCIL 0    /* collimated beam from (x0, z0) along (dir_x, dir_z)            */
#define MCR_LINE 1      /* collimated line source: start uniform on (x0,z0)-(x1,z1)       */
#define MCR_ISO_POINT 2 /* isotropic point source at (x0, z0)                             */
#define MCR_ANGULAR_POINT 3 /* point source at (x0, z0) with an angular density (below): a    *
                             * detector of Sec. 4.1 as the source of an adjoint computation   */
#define MCR_MAX_ANG 8   /* angular harmonics of an MCR_ANGULAR_POINT density               */

#define MCR_MAX_K 64

/* Pixelised medium (Sec. 3, Eq. 5): piecewise-constant mu_a, mu_s per pixel, scalar HG g. */
typedef struct {
  int32_t nx, nz;   /* pixels along x (columns) and z (rows), each >= 1, nx*nz < 2^26 */
  float dx;         /* pixel side, mm, > 0 */
  float g;          /* 2D Henyey-Greenstein anisotropy, -1 < g < 1 (Eq. 6) */
  const float *mua; /* device [nz][nx] absorption coefficient, 1/mm, >= 0 */
  const float *mus; /* device [nz][nx] scattering coefficient, 1/mm, >= 0 */
} mcr_medium;

/* Boundary or point source of a forward run (Sec. 3.2, Sec. 6).  Positions in mm; a point on
 * the far edge of the domain belongs to the last pixel; a point outside the domain escapes. */
typedef struct {
  int32_t kind;          /* MCR_PENCIL | MCR_LINE | MCR_ISO_POINT | MCR_ANGULAR_POINT */
  float x0, z0, x1, z1;  /* pencil / point: (x0, z0); line: segment (x0,z0)-(x1,z1) */
  float dir_x, dir_z;    /* launch direction (pencil, line); normalised by the library */
  float power;           /* total source power S (coefficients scale linearly with it) */
  /* MCR_ANGULAR_POINT: launch angles theta (from +z, theta = atan2(dir_x, dir_z)) with density
   * p(theta) = (1 + sum_{n=1..n_ang} ang_c[n-1] cos n theta + ang_s[n-1] sin n theta) / (2 pi),
   * which must be >= 0 (MCR_ERR_ARG otherwise); 0 <= n_ang <= MCR_MAX_ANG.  Ignored by the
   * other kinds. */
  int32_t n_ang;
  float ang_c[MCR_MAX_ANG], ang_s[MCR_MAX_ANG];
} mcr_source;

/* Monte Carlo run parameters.  Random numbers: Philox4x32-10 with key (seed_lo,
 * seed_hi ^ stream_id) and counter (packet_lo, packet_hi, event, 0); packet p of the run is
 * packet id first_packet + p, so a run split into packet ranges tallies bit-identically. */
typedef struct {
  int32_t K;             /* harmonic order, 0 <= K <= MCR_MAX_K (2K+1 channels) */
  uint32_t max_scatter;  /* packets end at collision max_scatter+1 (0xFFFFFFFF: unlimited) */
  uint64_t n_packets;    /* packets N_p launched by this call (normalisation divisor) */
  uint64_t first_packet; /* id of the first packet */
  uint64_t seed;
  uint32_t stream_id;
  uint32_t max_events;   /* flights per packet before it is ended (watchdog, e.g. 1e7) */
  float w_threshold;     /* Russian roulette once |W| < w_threshold |W0| (e.g. 1e-4) */
  float roulette_p;      /* roulette survival probability p, 0 < p <= 1; survivors W <- W/p */
  uint32_t accumulate;   /* 0: write coeff; 1: add this run's coefficients to coeff (the fluences of
                            several sources of one illumination sum, Eq. 5 is linear in q) */
  uint32_t sectors;      /* 0: the harmonic tally.  M in 1..1024 (mc_forward only): the discrete-
                            ordinates tally of Sec. 3.1 instead -- coeff [M][nz][nx] holds the radiance
                            integrated over the angular sectors [m 2pi/M, (m+1) 2pi/M) of theta
                            (from +z), summing to a_0; K is ignored */
  uint32_t time_bins;    /* 0: off.  T in 1..1024 (mc_forward only, not with sectors): the fluence resolved
                            by the packets' path length since launch (time of flight times c / n, the
                            radiance of a time-dependent source integrated over bins of equal time) --
                            coeff [T][nz][nx], bin b holding the track weight of the path-length interval
                            [b time_bin_mm, (b+1) time_bin_mm) and the last bin everything beyond, so the
                            bins sum to a_0; K is ignored */
  float time_bin_mm;     /* bin width in mm of path, > 0 when time_bins > 0 */
} mcr_run;

/* Run counters (host struct filled when a non-NULL pointer is passed; synchronises). */
typedef struct {
  uint64_t launched, flights, collisions, segments, escapes;
  uint64_t rr_kill, rr_survive, scatter_limit, event_limit;
  double launched_w;  /* sum of initial weights W0 (+-1) */
  double escaped_w;   /* weight carried out of the domain */
  double rr_net_w;    /* net weight added by roulette (survivor gain minus killed weight) */
  double killed_w;    /* weight of packets ended by max_scatter or max_events */
  double absorbed_w;  /* launched_w + rr_net_w - escaped_w - killed_w (bookkeeping) */
} mcr_stats;

/*
 * mc_forward -- forward harmonic radiance MC (Sec. 3 and 3.1, Eqs. 7, 9-11).
 * Launches run->n_packets packets from `src`, transports them with exponential free paths in
 * mu_s, absorption weighting W <- W exp(-mu_a l) per pixel segment, 2D HG scattering (Eq. 7)
 * and roulette below the weight threshold, and tallies each segment's track weight
 * t = W (1 - exp(-mu_a l)) / mu_a into a_0, a_n = t cos(n theta), b_n = t sin(n theta) of its
 * pixel.  coeff (device, [2K+1][nz][nx] FP32, overwritten) = power * sums / (N_p dx^2).
 * stats (host, may be NULL).  Tallies are 64-bit fixed-point sums of deposits rounded to a
 * quantum 2^-q mm, q chosen per run from dx, w_threshold and roulette_p so that one deposit
 * spans at most 2^30 quanta: the result does not depend on scheduling and is bit-reproducible
 * for a given run.  A medium with a negative or non-finite mu is detected on the device: the run
 * adds nothing to coeff (all-zero, or unchanged with accumulate = 1) and the next synchronising
 * call returns MCR_ERR_MEDIUM.
 */
int mc_forward(const mcr_medium *med, const mcr_source *src, const mcr_run *run, float *coeff,
               mcr_stats *stats, void *stream);

/*
 * mc_forward_noalloc -- mc_forward without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that cannot call cudaMalloc where they run the forward
 * model -- programs whose device memory is owned by another allocator or pool, loops that cannot
 * afford the device synchronisation that cudaMalloc/cudaFree imply, or hosts that forbid
 * allocation after start-up.  The caller passes the medium, the source and the output buffer
 * as for mc_forward; the scratch the kernels need (packed medium, fixed-point tally, counters)
 * lives in one 16 MiB array inside the library, which every GPU that loads libmcr holds until
 * the process exits.
 *   Limits: 512 + nx*nz*16 (rounded up to 256) + nx*nz*Cpad*8 bytes <= 16 MiB, with Cpad = 2K+1
 *   rounded up to a multiple of 16 when 2K+1 > 32, else to a multiple of 4 (e.g. 128x128 at
 *   K = 32, 256x256 at K = 8), and at most 2^26
 *   packets per call (use first_packet to split larger runs); larger problems return
 *   MCR_ERR_SCRATCH and launch nothing.
 *   The first call on each device looks up the array's device address (cudaGetSymbolAddress,
 *   with that device current) and caches it: make that first call before any stream capture.
 *   All calls share the one array and each call clears what it needs; calls whose work overlaps
 *   on the GPU (different streams, or different host threads) race on it and must be ordered
 *   by the caller.  No run counters are returned.  Errors found on the device (a negative or
 *   non-finite mu, a packet ended by max_events, a tally near overflow) are latched in the
 *   array and returned, like mc_forward's, by the next mc_check on this device (which reads and
 *   clears them without allocating); a run on a bad medium adds nothing to coeff (all-zero,
 *   or unchanged with accumulate = 1).
 * Same arguments (checked by the same rules), layout and results as mc_forward with
 * stats = NULL: for the same inputs the two outputs are bit-identical.
 */
int mc_forward_noalloc(const mcr_medium *med, const mcr_source *src, const mcr_run *run, float *coeff,
                       void *stream);

/*
 * mc_adjoint -- adjoint harmonic radiance MC (Sec. 4, Eq. 12; source of Sec. 6).
 * qstar (device [nz][nx] FP32, signed) is the isotropic adjoint source per unit area and unit
 * angle.  Packets start in pixel i with probability |q*_i| / sum|q*| (|q*| quantised to 2^32
 * levels of max|q*|), uniformly over the pixel, isotropically, with weight sign(q*_i); the run
 * represents the source strength S = 2 pi dx^2 sum|q*|.  The tally is the adjoint radiance
 * phi*(x, theta) = psi(x, theta + pi), psi being the forward radiance of the same source:
 * coeff_adj channels a*_n, b*_n carry the factor (-1)^n.  All-zero q* gives all-zero output.
 */
int mc_adjoint(const mcr_medium *med, const float *qstar, const mcr_run *run, float *coeff_adj,
               mcr_stats *stats, void *stream);

/*
 * mc_forward_raw / mc_adjoint_raw -- the transport of mc_forward / mc_adjoint (same arguments,
 * same packets, same random numbers) without the normalisation: `tally` (device, int64
 * [2K+1][nz][nx], channel-major, caller-owned) receives the run's 64-bit fixed-point sums of
 * Eqs. 9-11, in quanta of 2^-q weight x mm (q fixed by dx, w_threshold and roulette_p, so equal for
 * every range of one run), overwritten or, with run->accumulate = 1, added.  The adjoint's odd
 * orders are NOT yet turned by (-1)^n.  Integer sums are exact and order-free: the sums of
 * disjoint packet ranges [first_packet, first_packet + n_packets) added together (on one GPU with
 * accumulate, or across GPUs with an int64 all-reduce) equal the sums of the whole range bit for
 * bit -- the packet sharding of one problem over several GPUs (the method's packets are
 * independent, Sec. 3).  At most 2^26 packets per call (MCR_ERR_ARG; split larger ranges);
 * sectors must be 0.
 */
int mc_forward_raw(const mcr_medium *med, const mcr_source *src, const mcr_run *run, int64_t *tally,
                   mcr_stats *stats, void *stream);
int mc_adjoint_raw(const mcr_medium *med, const float *qstar, const mcr_run *run, int64_t *tally,
                   mcr_stats *stats, void *stream);

/*
 * mc_finalize -- coefficients from raw sums (Sec. 3.1 normalisation; Sec. 4's turn by pi):
 * coeff (device [2K+1][nz][nx] FP32, written or, with run->accumulate = 1, added to) =
 * sign * tally * 2^-q * S / (N_p dx^2), with N_p = run->n_packets (the TOTAL of all ranges
 * summed into `tally`), q as for the raw calls (run->w_threshold, run->roulette_p, med->dx).
 * Exactly one of `src` (forward: S = src->power, sign +1) and `qstar` (adjoint: S = 2 pi dx^2
 * sum|q*| as mc_adjoint quantises it, sign (-1)^n on order n) is non-NULL.  Bit-identical to
 * what mc_forward / mc_adjoint return for the whole range when N_p <= 2^26 (above, those sum
 * their 2^26-packet chunks in FP64 and the two agree to FP64 rounding).  A sum within 2 bits of
 * overflow is latched (MCR_ERR_TALLY_OVERFLOW at the next mc_check).
 */
int mc_finalize(const mcr_medium *med, const mcr_source *src, const float *qstar, const mcr_run *run,
                const int64_t *tally, float *coeff, void *stream);

#define MCR_MAX_BATCH 64

/* One problem of a batched launch: its own medium, source (forward) or q* (adjoint), packets,
 * seed and output. */
typedef struct {
  mcr_medium medium;
  mcr_source source;     /* forward source; ignored when qstar != NULL */
  const float *qstar;    /* device [nz][nx] adjoint source (as mc_adjoint), or NULL (forward) */
  uint64_t n_packets;    /* at most 2^26 per problem in a batch */
  uint64_t first_packet;
  uint64_t seed;
  uint32_t stream_id;
  float *coeff;          /* device out [2K+1][nz][nx], normalised as mc_forward / mc_adjoint */
} mcr_problem;

/* Launch shape of the persistent transport kernel; 0 fields take the defaults (128 threads per
 * block, as many blocks per SM as fit; collision merge where the second harmonic row per lane
 * costs no resident warps, or, with 96-thread blocks, where the tallies exceed 256 MB and their
 * reductions go to HBM).  A shape whose shared memory does not fit fails with MCR_ERR_CUDA.
 * The collision merge deposits a segment that ends in a surviving collision together with the
 * packet's next segment (same pixel) in one row reduction; the tally is bit-identical either way,
 * only the speed and the shared memory per block (one or two harmonic rows per lane) differ. */
typedef struct {
  int32_t threads_per_block; /* multiple of 32, <= 256 */
  int32_t blocks_per_sm;     /* cap on resident blocks per SM */
  int32_t merge_collisions;  /* 0 default, 1 off, 2 on */
  int32_t shared_tally;      /* 0 default (global), 1 global, 2 each block deposits into its own
                                shared-memory copy of the tally and adds it to the global one at
                                the end -- applies to a batch of one problem with 2K+1 <= 36
                                whose tally (pixels x Cpad x 8 B) fits beside the harmonic rows
                                (e.g. 32x32 at K = 8); otherwise the global tally is used */
  int32_t launch_order;      /* 0 default, 1 off, 2 on: process the packets in the order of their launch
                                position (line sources: 1/4096 of the line; volumetric sources: 32 x 32-
                                pixel tiles; other kinds keep their order), so that the packets in flight
                                start close together and their tally rows stay in L2.  The tally does not
                                depend on the order (bit-identical).  Default: on once the tallies of the
                                launch exceed 96 MB (mc_forward and mc_adjoint always use the default) */
  int32_t deposit;           /* 0 default, 1 direct, 2 sorted records (a batch of one harmonic problem):
                                the transport writes one 16-byte record per pixel segment instead of its
                                deposit, the records are sorted by pixel and each pixel's run is summed in
                                registers before one reduction -- the same rounded products, so the tally is
                                bit-identical, with far less HBM traffic when the tally does not fit in L2.
                                Default: on for one problem whose tally exceeds 256 MB (mc_forward and
                                mc_adjoint included).  It reads the record count back once per chunk of
                                packets (a stream synchronisation), so it is never used while the stream is
                                being captured into a graph. */
  int64_t record_capacity;   /* records per chunk of the sorted-record deposit (0: 2^30, two 16 GB buffers;
                                if they cannot be allocated the run deposits directly); chunks are sized
                                from the records per packet seen so far, and a chunk that overflows the
                                buffer is run again with the direct deposit */
} mcr_launch;

/*
 * mc_run_batch -- many forward and/or adjoint problems (uneven grids, different media, sources
 * and packet counts; one harmonic order) in ONE persistent transport launch: warps draw packets
 * from the concatenated packet ranges of all problems, so the launch stays full until the last
 * problem is done (the batching pattern of the method's data-parallel structure, Sec. 3 and 4).
 * `common` supplies K, max_scatter, max_events, w_threshold and roulette_p (its n_packets, seed,
 * first_packet and stream_id are ignored).  Each problem's coefficients equal what mc_forward /
 * mc_adjoint returns for it alone (same packets, bit-identical tallies).  No host
 * synchronisation and, once the workspace has grown to the batch's size (make one call outside
 * capture first), no allocation: the call can be captured in a CUDA graph.  `launch` may be
 * NULL.  stats (host, may be NULL) sums the counters of all problems and synchronises.
 */
int mc_run_batch(const mcr_problem *problems, int32_t n_problems, const mcr_run *common, const mcr_launch *launch,
                 mcr_stats *stats, void *stream);

/*
 * mc_h_eps -- absorbed energy and error functional (Sec. 2, Eq. 2).
 * H = mu_a a_0 (device out [nz][nx] FP32, Grueneisen parameter 1); if Hmeas != NULL also
 * dL_dH = -dx^2 (H^meas - H) (device out [nz][nx] FP32, may be NULL) and
 * eps = 1/2 dx^2 sum (H^meas - H)^2 (device out, one double, may be NULL), the sum reduced in
 * FP64 in a fixed order (deterministic).
 */
int mc_h_eps(const mcr_medium *med, const float *coeff, const float *Hmeas, float *H, float *dL_dH,
             double *eps, void *stream);

/*
 * mc_eps -- the error functional of Eq. 2 from a given absorbed-energy map: for npix pixels of
 * area pixel_area, eps = 1/2 pixel_area sum (H^meas - H)^2 (device out, one double, FP64
 * residuals, fixed-order reduction) and dL_dH = -pixel_area (H^meas - H) (device out FP32, may be
 * NULL).  H, Hmeas: device FP32 [npix].
 */
int mc_eps(int64_t npix, double pixel_area, const float *H, const float *Hmeas, float *dL_dH, double *eps,
           void *stream);

/*
 * mc_dot -- the inner products of the reconstruction's line searches and quasi-Newton updates
 * (Sec. 6: the directional derivative g.d of the sufficient-decrease test, Eq. 30):
 * out (device, one double) = sum_i a_i b_i over n FP32 elements (device), FP64 products and sums
 * in a fixed order (deterministic).
 */
int mc_dot(int64_t n, const float *a, const float *b, double *out, void *stream);

/*
 * mc_adjoint_source -- q*_i = -mu_a,i dL_dH_i / dx^2 (device out [nz][nx] FP32).  For the
 * paper's eps (dL_dH = -dx^2 (H^meas - H)) this is q* = mu_a (H^meas - H) of Sec. 6.
 */
int mc_adjoint_source(const mcr_medium *med, const float *dL_dH, float *qstar, void *stream);

/*
 * mc_gradient -- functional gradients from forward and adjoint coefficients (Sec. 5).
 * Per pixel, in FP64 with the sums over n in increasing n:
 *   G_a = a_0 a_0^* / (2 pi) + (1/pi) sum_{n=1..K} (a_n a_n^* + b_n b_n^*)             (Eq. 22)
 *   G_s = (1/pi) sum_{n=1..K} (a_n a_n^* + b_n b_n^*) (1 - g^n)                    (Eq. 28)
 *   d_mua = dL_dH a_0 + dx^2 G_a,   d_mus = dx^2 G_s     (device out [nz][nx] FP64)
 * i.e. the gradient of the pixel loss L with respect to each pixel's mu_a and mu_s.  With
 * dL_dH = -dx^2 (H^meas - H) this is dx^2 times Eqs. 22 and 28.  d_mus may be NULL.
 */
int mc_gradient(const mcr_medium *med, int32_t K, const float *coeff, const float *coeff_adj,
                const float *dL_dH, double *d_mua, double *d_mus, void *stream);

/* mc_gradient_f32 -- mc_gradient with the same FP64 accumulation and FP32 outputs (rounded once),
 * for callers whose parameters are FP32 (e.g. autograd leaves). */
int mc_gradient_f32(const mcr_medium *med, int32_t K, const float *coeff, const float *coeff_adj,
                    const float *dL_dH, float *d_mua, float *d_mus, void *stream);

/* Synchronises `stream` and returns (and clears) the device's latched error status. */
int mc_check(void *stream);

/*
 * mc_last_run_info -- profiling query (the paper has no counterpart).  which = 0: the last
 * mc_forward call on the current device; which = 1: the last mc_adjoint call; which = 2: the
 * last mc_run_batch call that was not being captured into a graph.  Fills `stats`
 * (host, may be NULL) with that call's counters and `transport_ms` (host, may be NULL) with the
 * device time of its transport kernel launch(es), measured by CUDA events recorded on the
 * call's stream around them.  Waits for that call to finish.  MCR_ERR_ARG if no such call ran.
 */
int mc_last_run_info(int32_t which, mcr_stats *stats, float *transport_ms);

/* Frees the calling device's workspace, the 3D calls' included (synchronises the device). */
int mc_release_workspace(void);

/* Static text for a status code. */
const char *mc_status_string(int status);

/* Library version string, e.g. "mcr 1.0 sm_103a". */
const char *mc_version(void);

#ifdef __cplusplus
}
#endif

#endif /* MCR_H */
