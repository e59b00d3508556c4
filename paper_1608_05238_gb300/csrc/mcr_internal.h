// mcr_internal.h -- declarations shared by the translation units of libmcr (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/mcr.h"

namespace mcr {

// Fixed-point tallies: each deposit t h (weight x mm) is stored as round(t h 2^q) in 64-bit sums.
// The run picks q so that |t h| 2^q < 2^31 for every possible deposit (t <= W_max dx sqrt 2),
// so one 32-bit conversion per coefficient suffices.
int tally_exponent(float dx, float w_threshold, float roulette_p);
// Packets per transport launch; longer runs are split into chunks whose fixed-point sums are
// flushed into an FP64 accumulator in chunk order (keeps |sum| far below 2^63).
constexpr uint64_t kChunkPackets = 1ull << 26;

// Source kinds seen by the transport kernel (MCR_* plus the volumetric adjoint source).
constexpr int kVolume = 100;  // not a public MCR_* source kind
static_assert(kVolume != MCR_PENCIL && kVolume != MCR_LINE && kVolume != MCR_ISO_POINT && kVolume != MCR_ANGULAR_POINT,
              "the internal volumetric kind must differ from every public source kind");

// Device counters of one run, accumulated per warp.
struct DevStats {
  unsigned long long launched, flights, collisions, segments, escapes;
  unsigned long long rr_kill, rr_survive, scatter_limit, event_limit;
  double launched_w, escaped_w, rr_net_w, killed_w;
};

// Error bits latched on the device.
constexpr unsigned kFlagEventLimit = 1u;
constexpr unsigned kFlagOverflow = 2u;
constexpr unsigned kFlagMedium = 4u;
constexpr unsigned kFlagChecked = 16u;  // checked build: an index out of range or a non-finite weight

// Checked build (-DMCR_CHECKED, libmcr_checked.so): MCR_GUARD(flags, cond) is cond, and a false
// cond latches kFlagChecked (MCR_ERR_CHECK at the next mc_check) -- the caller then skips the
// access, so a broken index never reaches memory.  In the normal build it is `true`.
#ifdef MCR_CHECKED
#define MCR_GUARD(flags, cond) ((cond) ? true : (atomicOr((flags), ::mcr::kFlagChecked), false))
#else
#define MCR_GUARD(flags, cond) true
#endif

// Problems per transport launch (the table travels in kernel parameter space).
constexpr int kMaxBatch = 64;

// One problem of a transport launch: medium, source, tally and its packet range.
struct ProblemDesc {
  const float4 *mu;               // packed (mu_a, mu_s, 1/mu_a, 1/mu_s) per pixel
  unsigned long long *tally;      // [npix][Cpad] fixed point
  const unsigned long long *cdf;  // volumetric: inclusive prefix of quantised |q|
  const float *q;                 // volumetric: signed source (for the packet sign)
  unsigned long long first_packet;  // packet id of the problem's first packet
  unsigned long long end;           // exclusive end of its packets in the launch's packet space
  int nx, nz;
  float dx;
  float hg_c;    // (1 - g) / (1 + g)
  float qscale;  // 2^q, the fixed-point scale of the deposits
  int kind;      // MCR_PENCIL | MCR_LINE | MCR_ISO_POINT | MCR_ANGULAR_POINT | kVolume
  float x0, z0, x1, z1, dir_x, dir_z;
  int n_ang;     // MCR_ANGULAR_POINT: harmonics of the launch-angle density
  float ang_c[MCR_MAX_ANG], ang_s[MCR_MAX_ANG];
  unsigned key0, key1;
  unsigned bin_base;  // launch order: the problem's first bin in the launch's bin space
};

struct TransportParams {
  int n_problems;
  int K, C, Cpad, row_stride;  // C = 2K+1 channels, Cpad = tally_row_words(C), smem row stride
  int sectors;                 // > 0: discrete-ordinates tally, C = sectors (single forward problem)
  float sector_scale;          // sectors / (2 pi)
  int time_bins;               // > 0: path-length (time-of-flight) resolved fluence, C = time_bins
  float time_bin_mm, inv_time_bin;
  unsigned max_scatter, max_events;
  float w_threshold, rr_p, rr_inv_p;
  unsigned long long total_packets;  // = prob[n_problems-1].end
  unsigned long long *work;          // packet counter
  const unsigned *order;             // launch order: the launch index taken at step g (nullptr: g)
  // sorted-record deposit (transport variant RECS): one record per segment instead of deposits
  float4 *records;                   // (pixel bits, track weight x 2^q, s_x, s_z), capacity rec_capacity
  unsigned long long *rec_count;     // records written (may pass the capacity: then rec_overflow is set)
  unsigned *rec_overflow;
  unsigned long long rec_capacity;
  unsigned *rec_hist;                // records per pixel
  DevStats *stats;
  unsigned *flags;                   // error bits: transport does nothing if kFlagMedium is set; it
                                     // latches kFlagEventLimit when a packet reached max_events
  ProblemDesc prob[kMaxBatch];
};

// Launch shape of the persistent transport kernel (0 = default: 128 threads, full occupancy).
struct TransportLaunch {
  int threads_per_block;
  int blocks_per_sm;
  int merge;         // collision merge: 0 library default, 1 off, 2 on
  int shared_tally;  // 0 default (global), 1 global, 2 per-block shared-memory copy where it applies
  int launch_order;  // 0 library default (on above kOrderTallyBytes of tallies), 1 off, 2 on
  int deposit;       // 0 library default (sorted records above kRecordTallyBytes), 1 direct, 2 sorted records
  long long record_capacity;  // records per chunk of the sorted-record deposit (0: kRecordCapacity)
};

// Sorted-record deposit (single problems whose tally lives in HBM): the transport writes one
// record per pixel segment, the records are sorted by pixel (one counting-sort pass) and a
// deposit kernel sums each pixel's run in registers before one reduction per run.  The integer
// tally is bit-identical to the direct deposit.
constexpr double kRecordTallyBytes = 256.0 * 1024 * 1024;
// Records per chunk (16 GB per buffer, two buffers): a chunk must hold several times the packets
// in flight (~1.2e5 lanes), or the transport spends it waiting for the last, longest packets.
constexpr unsigned long long kRecordCapacity = 1ull << 30;
constexpr unsigned kRecBlock = 1024;            // record slots a warp reserves at a time
constexpr unsigned kRecSentinel = 0xFFFFFFFFu;  // pixel field of an unused slot
struct RecordHeader {
  unsigned long long count;
  unsigned overflow;
  unsigned pad[13];
  DevStats stats;  // counters of the record-mode launch, added to the run's once its records are deposited
};
// dst += src (run counters)
cudaError_t launch_add_stats(DevStats *dst, const DevStats *src, cudaStream_t s);
// Launch the transport in record mode (p.records etc. set; single harmonic problem).
cudaError_t launch_transport_records(const TransportParams &p, const TransportLaunch &cfg, cudaStream_t s);
// cursor[i] = sum_{k<i} hist[k] (exclusive scan of the per-pixel counts), then the records in
// pixel order into `sorted` (cursor consumed), then the runs of each pixel deposited into the tally.
// n: the written slots to read (at most the records buffer's capacity; sentinels are skipped).
cudaError_t launch_sort_and_deposit(const float4 *records, unsigned long long n, const unsigned *hist,
                                    unsigned *cursor, unsigned *block_sums, int npix, float4 *sorted, int K, int Cpad,
                                    unsigned long long *tally, unsigned *flags, cudaStream_t s);

// Launch order: packets processed in the order of their launch position (line sources: bins of
// 1/4096 of the line; volumetric sources: 32 x 32-pixel tiles of the launch pixel; other kinds
// unordered), so that the packets in flight start close together and share the tally rows in
// L2.  The integer tally does not depend on the order.  On by default once the launch's tallies
// exceed kOrderTallyBytes (their reductions would otherwise miss L2).
constexpr double kOrderTallyBytes = 96.0 * 1024 * 1024;
// Bins of one problem's launch order (1 for unordered kinds).
unsigned order_bins(const ProblemDesc &d);
// Fills order[0, p.total_packets) with the launch indices sorted by bin (p.prob[].bin_base set,
// total_bins their sum); hist: scratch of total_bins words.
cudaError_t launch_order(const TransportParams &p, unsigned total_bins, unsigned *hist, unsigned *order,
                         cudaStream_t s);

// Workspace of one device (grow-only).
struct Workspace {
  int device = -1;
  unsigned long long *tally = nullptr;
  size_t tally_bytes = 0;
  double *acc = nullptr;  // FP64 chunk accumulator [C][npix]
  size_t acc_bytes = 0;
  float4 *mu = nullptr;
  size_t mu_bytes = 0;
  unsigned long long *cdf = nullptr;
  size_t cdf_bytes = 0;
  unsigned long long *block_sums = nullptr;
  size_t block_sums_bytes = 0;
  unsigned *order = nullptr;  // launch order of the packets of one launch
  size_t order_bytes = 0;
  unsigned *order_hist = nullptr;
  size_t order_hist_bytes = 0;
  // sorted-record deposit: records and their pixel-sorted copy, header, per-pixel counts / cursors
  float4 *records = nullptr;
  size_t records_bytes = 0;
  float4 *sorted = nullptr;
  size_t sorted_bytes = 0;
  RecordHeader *rec_hdr = nullptr;
  size_t rec_hdr_bytes = 0;
  unsigned *rec_hist = nullptr;  // [npix] counts, then [npix] cursors, then block sums
  size_t rec_hist_bytes = 0;
  double *partials = nullptr;
  size_t partials_bytes = 0;
  // small block: packet counter, run counters per call kind (0 forward, 1 adjoint, 2 batch),
  // flags, and max|q*| bits per problem of a volumetric run
  unsigned char *small = nullptr;
  unsigned long long *work() const { return reinterpret_cast<unsigned long long *>(small); }
  DevStats *stats(int slot) const { return reinterpret_cast<DevStats *>(small + 64 + 128 * slot); }
  unsigned *flags() const { return reinterpret_cast<unsigned *>(small + 448); }
  unsigned *qmax_bits(int problem = 0) const { return reinterpret_cast<unsigned *>(small + 512) + problem; }
  // events around the transport launches of the last call of each kind
  cudaEvent_t ev_start[3] = {nullptr, nullptr, nullptr};
  cudaEvent_t ev_stop[3] = {nullptr, nullptr, nullptr};
  bool ran[3] = {false, false, false};
};

constexpr size_t kSmallBytes = 512 + 4 * kMaxBatch;
static_assert(sizeof(DevStats) <= 128, "stats slot");

// ---- launchers (each enqueues on `s` and returns the launch error) ----
cudaError_t launch_pack_medium(const float *mua, const float *mus, float4 *mu, int64_t npix, unsigned *flags,
                               cudaStream_t s);
cudaError_t launch_transport(const TransportParams &p, const TransportLaunch &cfg, cudaStream_t s);
size_t transport_smem_bytes(int row_stride, int threads, bool merge);

// 8-byte words per pixel in the fixed-point tally: 2K+1 rounded up to 16 (rows of whole 128-byte
// lines, so each warp-wide 256-byte reduction touches exactly two lines: 7 % faster at K = 32)
// when 2K+1 > 32, else up to 4 (a pixel's block starts on a 32-byte sector).
// The launch-angle density of an MCR_ANGULAR_POINT source into a problem descriptor.
inline void set_angular(ProblemDesc &d, const mcr_source &src) {
  d.n_ang = src.kind == MCR_ANGULAR_POINT ? src.n_ang : 0;
  for (int n = 0; n < MCR_MAX_ANG; ++n) {
    d.ang_c[n] = n < d.n_ang ? src.ang_c[n] : 0.f;
    d.ang_s[n] = n < d.n_ang ? src.ang_s[n] : 0.f;
  }
}
// Validation of an MCR_ANGULAR_POINT density: 0 <= n_ang <= MCR_MAX_ANG, finite coefficients,
// p(theta) >= 0 on a 4096-point grid (tolerance 1e-6 / 2 pi).  Returns false when invalid.
bool angular_density_ok(const mcr_source &src);

inline int tally_row_words(int C) { return C > 32 ? (C + 15) & ~15 : (C + 3) & ~3; }

// Harmonic tallies with 2K+1 = 32 m + 1 > 32 coefficients ("dense" rows): each pixel's row starts
// 15 words into its tally_row_words(C) = 32 m + 16 word slot, so that coefficients 1..2K fill the
// slot's last 32 m words, whole 128-byte lines, and go by cooperative reductions of 32 aligned words;
// coefficient 0 -- the track weight itself -- takes the slot's word 15 and is summed per lane over a
// packet's consecutive segments in one pixel before its reduction.  The host shifts each problem's
// tally base by this offset; every kernel then indexes rows as base + pixel * Cpad + c, and the
// slot's first 15 words stay zero.  0 for every other tally (and for the sector and time tallies).
__host__ __device__ inline int tally_row_offset(int C) { return (C > 32 && (C & 31) == 1) ? 15 : 0; }

// Words per harmonic row in shared memory: channel c at word 1 + c (so the (cos, sin) pairs are
// 8-byte aligned), at least C + 1 and = 2 (mod 4), so that the lanes' 8-byte row stores fall in
// distinct banks.
inline int transport_row_stride(int C) { return (C + 1) % 4 == 0 ? C + 3 : C + 1; }
cudaError_t launch_source_cdf(const float *q, int64_t npix, unsigned long long *cdf,
                              unsigned long long *block_sums, size_t block_sums_cap, unsigned *qmax_bits,
                              cudaStream_t s);
// accumulate (chunked runs): acc[c][pix] += tally[pix][c] * quantum   (quantum = 2^-q)
cudaError_t launch_accumulate(const unsigned long long *tally, int64_t npix, int C, int Cpad, double quantum,
                              double *acc, cudaStream_t s);
// coeff[c][pix] = sums * scale, sign (-1)^n on channels 2n-1, 2n when `adjoint`; the fixed-point
// sums are multiplied by `quantum` (2^-q) first.  scale = fixed_scale (forward) or
// 2 pi qmax total 2^-32 / N_p (volumetric: read on device).
cudaError_t launch_finalize(const unsigned long long *tally, const double *acc, int64_t npix, int C, int Cpad,
                            double quantum, double fixed_scale, bool volumetric, const unsigned *qmax_bits,
                            const unsigned long long *cdf_total, double n_packets, bool adjoint, bool accumulate,
                            float *coeff, unsigned *flags, cudaStream_t s);
// raw fixed-point sums out: out[c][pix] (=, or += with accumulate) tally[pix][c] (int64 quanta)
cudaError_t launch_export_raw(const unsigned long long *tally, int64_t npix, int C, int Cpad, bool accumulate,
                              long long *out, cudaStream_t s);
// channel-major raw sums -> coeff, normalised as launch_finalize
cudaError_t launch_finalize_raw(const long long *raw, int64_t npix, int C, double quantum, double fixed_scale,
                                bool volumetric, const unsigned *qmax_bits, const unsigned long long *cdf_total,
                                double n_packets, bool adjoint, bool accumulate, float *coeff, unsigned *flags,
                                cudaStream_t s);
cudaError_t launch_h_eps(const float *mua, const float *a0, const float *Hmeas, int64_t npix, double area, float *H,
                         float *dL_dH, double *partials, size_t partials_cap, double *eps, cudaStream_t s);
cudaError_t launch_adjoint_source(const float *mua, const float *dL_dH, int64_t npix, double area, float *q,
                                  cudaStream_t s);
// *out = sum_i a_i b_i in FP64, per-block partials then one thread in block order (deterministic)
cudaError_t launch_dot(const float *a, const float *b, int64_t n, double *partials, size_t partials_cap, double *out,
                       cudaStream_t s);
cudaError_t launch_gradient(const float *coeff, const float *coeff_adj, const float *dL_dH, int64_t npix, int K,
                            double g, double area, double *d_mua, double *d_mus, cudaStream_t s);
cudaError_t launch_gradient_f32(const float *coeff, const float *coeff_adj, const float *dL_dH, int64_t npix, int K,
                                double g, double area, float *d_mua, float *d_mus, cudaStream_t s);

// Host-side argument checks shared by every entry point that takes these structs (mcr_api.cu).
int check_medium(const mcr_medium *m);
int check_run(const mcr_run *r);
// Also yields the normalised launch direction of a boundary source.
int check_source(const mcr_source *src, float *dirx, float *dirz);
// Status from the error bits of the given word (medium before overflow before event limit).
int status_from_flags(unsigned flags);
// mc_forward_noalloc's latched error bits on the current device, read and cleared on stream s
// (MCR_OK when that entry point never ran on this device); synchronises s (mcr_noalloc.cu).
int noalloc_take_flags(cudaStream_t s);

// Frees the 3D transport's workspace on device dev (mcr3.cu).
int release_workspace3(int dev);

}  // namespace mcr
