// mcr_transport.cu -- the photon-packet transport kernel of the forward and adjoint harmonic
// radiance Monte Carlo (Sec. 3, 3.1 and 4 of Hochuli et al., arXiv 1608.05238), for sm_103a.
//
// Design (one GPU, HBM/L2 resident tallies):
//  * One launch runs a table of problems (up to kMaxBatch: grids of different sizes, media,
//    sources, tallies; one harmonic order K).  The table travels in kernel parameter space, so
//    the launch needs no device-side descriptor memory and can be captured in a CUDA graph.  A
//    single mc_forward / mc_adjoint call is a table of one.
//  * Persistent warps.  Each lane carries one packet; a lane whose packet ended takes the next
//    packet index of the launch's packet space from a global counter (one atomic per warp per
//    refill) and finds its problem by binary search over the table's prefix ends, so lanes stay
//    busy until all problems' packets are used up.  One loop iteration = one pixel segment.
//  * Counter-based Philox4x32-10 per packet: the random numbers of packet p depend only on
//    (seed, stream_id, p, event), never on which warp ran it.
//  * Pixel traversal keeps integer pixel indices authoritative and the position as an offset
//    inside the pixel (exactly 0 or dx after an edge crossing), so FP32 positions do not drift.
//  * Harmonic vectors h = (1, cos theta, sin theta, ..., cos K theta, sin K theta) are built
//    once per free flight from (s_z + i s_x)^n (K complex products, no trigonometry) into a
//    per-lane shared-memory row.
//  * Deposits are warp-cooperative: for each tally row touched in this iteration, the lanes of
//    the warp take one coefficient each, sum the contributions of every lane in that row (warp
//    reduction via match_any on the row address) as 64-bit fixed-point integers, and issue one
//    coalesced red.add per coefficient into the pixel-major tally [pix][Cpad].  Integer sums are
//    exact, so the tally does not depend on scheduling.
//  * Collision merge (MERGE): a segment that ends in a collision the packet survives is not
//    deposited at once; it rides along with the next segment, which starts in the same pixel,
//    and both are added into one row reduction.  Each lane keeps two harmonic rows (the previous
//    flight's and the current one), and every term is still rounded on its own, so the integer
//    tally is identical to the unmerged one while the L2 sees one row reduction fewer per such
//    collision.  Deposits are rounded to 2^-q with q
//    chosen per problem so that one deposit fits in int32: the conversion is a 32-bit one (the
//    64-bit conversion runs on the FP64 pipe, which is narrow on this part).
//  * Dense rows (2K+1 = 32 m + 1): each tally row starts 15 words into its 128-byte aligned slot,
//    so coefficients 1..2K go by whole-line cooperative reductions, and coefficient 0 (h_0 = 1:
//    the rounded track weight itself) is summed per lane over a packet's consecutive segments in
//    one pixel and reduced when the pixel changes.
//  * Single problems keep the current pixel's medium values in registers and load the next
//    pixel's right after a crossing, off the next segment's critical path (the last packets of a
//    run advance one latency-bound segment per warp step).
#include <math_constants.h>

#include <mutex>

#include "mcr_harmonics.cuh"
#include "mcr_internal.h"
#include "mcr_rng.cuh"

namespace mcr {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kRowsPerStep = 2;  // independent single-lane rows deposited per step
constexpr double kL2SpillBytes = 256.0 * 1024 * 1024;  // tallies beyond this live in HBM

// Volumetric source: smallest i with cdf[i] > floor(r48 * total / 2^48).
__device__ __forceinline__ int pick_pixel(const unsigned long long *__restrict__ cdf, int npix,
                                          unsigned long long total, unsigned w0, unsigned w1) {
  const unsigned long long r48 = ((unsigned long long)w0 << 16) | (unsigned long long)(w1 >> 16);
  const unsigned long long target = __umul64hi(r48 << 16, total);
  int lo = 0, hi = npix - 1;
  while (lo < hi) {
    const int mid = lo + ((hi - lo) >> 1);
    if (__ldg(cdf + mid) > target)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

__device__ __forceinline__ float clamp_dx(float v, float dx) { return fminf(fmaxf(v, 0.f), dx); }

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// Launch angle (from +z) of an MCR_ANGULAR_POINT source: the theta in [0, 2 pi) at which the
// integral of its density from 0,
//   F(theta) = (theta + sum_n [c_n sin n theta + s_n (1 - cos n theta)] / n) / (2 pi),
// reaches u; 24 bisection steps resolve theta to the FP32 spacing of [0, 2 pi).  Runs once per
// packet, at launch.
__device__ __forceinline__ float launch_angle(const ProblemDesc &P, float u) {
  const float two_pi = 6.28318530717958648f;
  float lo = 0.f, hi = two_pi;
  const float target = u * two_pi;
  for (int it = 0; it < 24; ++it) {
    const float mid = 0.5f * (lo + hi);
    float F = mid;
    for (int n = 1; n <= P.n_ang; ++n) {
      float sn, cn;
      sincosf(n * mid, &sn, &cn);
      F += (P.ang_c[n - 1] * sn + P.ang_s[n - 1] * (1.f - cn)) / n;
    }
    if (F < target)
      lo = mid;
    else
      hi = mid;
  }
  return 0.5f * (lo + hi);
}

// NP = 0: the discrete-ordinates variant (Sec. 3.1's alternative to the harmonics): each segment
// adds its track weight to one of p.sectors equal angular sectors of its pixel, one per-lane
// reduction instead of 2K+1 cooperative ones (single forward problem, no merge).
// NP = -1: the time-resolved variant: each segment's track weight is split over the path-length
// bins [b w, (b+1) w) it spans (the last bin open-ended), one per-lane reduction per piece; the
// packet's path and weight updates are those of the plain run.
// RECS: the harmonic tally by sorted records -- each segment with a deposit writes one record
// (pixel, track weight x 2^q, direction) and counts it for its pixel; the deposit is done later
// by k_deposit_sorted with the same harmonic rows and products (single problem, no merge).
template <int NP, bool BATCH, bool MERGE, bool STALLY, bool RECS = false>
__global__ void __launch_bounds__(256) k_transport(const __grid_constant__ TransportParams p) {
  constexpr bool SECT = NP == 0;
  constexpr bool TIMED = NP < 0;
  constexpr bool ROWLESS = SECT || TIMED || RECS;  // no harmonic rows
  static_assert(!ROWLESS || (!BATCH && !MERGE && !STALLY), "the sector and time tallies run one plain forward problem");
  extern __shared__ float smem[];
  const int lane = threadIdx.x & 31;
  const int warp = threadIdx.x >> 5;
  // harmonic rows of this warp: row r of lane l at rows + (r * 32 + l) * row_stride (r < 2 with MERGE)
  float *const rows = smem + (size_t)warp * (MERGE ? 64 : 32) * p.row_stride;
  // STALLY (one small problem): the block deposits into its own shared-memory copy of the tally,
  // placed after all warps' rows, and adds it to the global tally once at the end
  unsigned long long *const stally =
      reinterpret_cast<unsigned long long *>(smem + (size_t)blockDim.x * (MERGE ? 2 : 1) * p.row_stride);
  if (*p.flags & kFlagMedium) return;
  if (STALLY) {
    const size_t nw = (size_t)p.prob[0].nx * p.prob[0].nz * p.Cpad;
    for (size_t i = threadIdx.x; i < nw; i += blockDim.x) stally[i] = 0ull;
    __syncthreads();
  }
  // base of the tally row of a segment key ((pixel + 1) << 6 | problem)
  auto tally_row = [&](unsigned key) -> unsigned long long * {
    return (STALLY ? stally : p.prob[BATCH ? (key & 63u) : 0].tally) + (size_t)((key >> 6) - 1u) * p.Cpad;
  };
  // checked build: the key names a pixel of its problem (and a problem of the launch)
  auto row_ok = [&](unsigned key) -> bool {
    const unsigned pi = BATCH ? (key & 63u) : 0u;
    return MCR_GUARD(p.flags, pi < (unsigned)p.n_problems && (key >> 6) >= 1u &&
                                  (key >> 6) - 1u < (unsigned)(p.prob[pi].nx * p.prob[pi].nz));
  };

  const int K = p.K, C = p.C;
  // Coefficients [c0, c0 + Cw) are deposited warp-cooperatively (32 per instruction).  Dense rows
  // (2K+1 = 32 m + 1, see tally_row_offset) take coefficients 1..2K that way, line-aligned, and
  // coefficient 0, the track weight itself, per lane: summed in a register over the packet's
  // consecutive segments in one pixel (collisions split a pixel's path) and reduced when the pixel
  // changes.  Otherwise a short remainder [Cw, C) of at most 4 is deposited by each lane into its
  // own row, all lanes in one instruction, instead of one nearly empty instruction per row.
  const bool dense = !ROWLESS && tally_row_offset(C) != 0;
  const int c0 = dense ? 1 : 0;
  const int Cw = dense ? C - 1 : ((C & 31) <= 4 ? (C & ~31) : C);
  long long acc0 = 0;     // dense: coefficient 0 of the pending pixel acc0_key
  unsigned acc0_key = 0u;
  auto flush0 = [&]() {
    if (acc0_key != 0u && row_ok(acc0_key)) atomicAdd(tally_row(acc0_key), (unsigned long long)acc0);
    acc0_key = 0u;
  };

  bool alive = false, exhausted = false;
  unsigned long long pid = 0;
  // the lane's problem, cached at launch
  const float4 *mu = nullptr;
  int prob = 0;
  int nx = 1, nz = 1;
  float dx = 1.f, hg_c = 1.f, qscale = 1.f;
  unsigned key0 = 0, key1 = 0;
  // problem fields: per-lane registers in a batch, uniform kernel parameters for a single problem
  auto NX = [&]() { return BATCH ? nx : p.prob[0].nx; };
  auto NZ = [&]() { return BATCH ? nz : p.prob[0].nz; };
  auto DX = [&]() { return BATCH ? dx : p.prob[0].dx; };
  auto HGC = [&]() { return BATCH ? hg_c : p.prob[0].hg_c; };
  auto QS = [&]() { return BATCH ? qscale : p.prob[0].qscale; };
  auto KEY0 = [&]() { return BATCH ? key0 : p.prob[0].key0; };
  auto KEY1 = [&]() { return BATCH ? key1 : p.prob[0].key1; };
  auto MU = [&]() { return BATCH ? mu : p.prob[0].mu; };
  // packet state
  float fx = 0.f, fz = 0.f, sx = 0.f, sz = 1.f, inv_ax = 0.f, inv_az = 0.f, W = 0.f, tau = 0.f;
  int ix = 0, iz = 0;
  // single problem: (mu_a, mu_s, 1/mu_a, 1/mu_s) of the packet's current pixel, loaded when the
  // packet enters a pixel -- at launch, and right after a crossing, so that the load's latency
  // overlaps the deposit and the collision instead of starting the next segment (the pixel is
  // unchanged after a collision).  Batches load it per segment (the extra registers would cost
  // their kernels resident warps).
  float4 mcur = make_float4(0.f, 0.f, CUDART_INF_F, CUDART_INF_F);
  auto load_mu = [&]() {
    float4 v = make_float4(0.f, 0.f, CUDART_INF_F, CUDART_INF_F);
    if (MCR_GUARD(p.flags, (unsigned)ix < (unsigned)NX() && (unsigned)iz < (unsigned)NZ()))
      v = __ldg(MU() + iz * NX() + ix);
    return v;
  };
  unsigned flight = 0, nscat = 0, cu1 = 0, cu2 = 0;
  // RECS: the warp's block of record slots [rec_block, rec_block + kRecBlock), filled to rec_fill;
  // slots left empty when a block is closed hold a sentinel that the sort skips
  unsigned long long rec_block = 0;
  unsigned rec_fill = kRecBlock;
  auto rec_pad = [&]() {
    if (rec_fill >= kRecBlock) return;
    for (unsigned j = rec_fill + lane; j < kRecBlock; j += 32)
      if (rec_block + j < p.rec_capacity) p.records[rec_block + j] = make_float4(__uint_as_float(kRecSentinel), 0.f, 0.f, 1.f);
  };
  int sect = 0;           // SECT: the current flight's angular sector
  float plen = 0.f;       // TIMED: path length since launch
  int rb = 0;             // row of the current flight's harmonics
  int carry_rb = 0;       // row of the deferred segment's harmonics
  float carry = 0.f;      // deferred track weight (times 2^q) of a collision segment, 0: none
  unsigned n_launch = 0, n_flight = 0, n_coll = 0, n_seg = 0, n_esc = 0, n_rrk = 0, n_rrs = 0, n_scl = 0,
           n_evl = 0;
  double w_launch = 0.0, w_esc = 0.0, w_rr = 0.0, w_kill = 0.0;

  // harmonic row of the current flight direction, h_n = (s_z + i s_x)^n, stored one slot to the
  // right (my[1 + c] holds channel c) so that each (cos n theta, sin n theta) pair is one
  // 8-byte aligned store; the row stride is 2 mod 4 words, so these stores are conflict-free.
  auto write_row = [&]() { harmonic_row(rows + (rb * 32 + lane) * p.row_stride, sx, sz, K); };
  // start free flight number `flight` (event flight+1): tau = -ln U, keep U for scatter/roulette
  auto begin_flight = [&]() {
    const uint4 r = philox4x32_10(pid, flight + 1u, KEY0(), KEY1());
    tau = -logf(u01(r.x));
    cu1 = r.y;
    cu2 = r.z;
    inv_ax = __frcp_rn(fabsf(sx));
    inv_az = __frcp_rn(fabsf(sz));
    ++n_flight;
    if (MERGE) rb ^= 1;  // keep the previous flight's row for a deferred segment
    if constexpr (SECT) {
      float th = atan2f(sx, sz);  // (-pi, pi], from +z
      if (th < 0.f) th += 6.28318530717958648f;
      sect = min((int)(th * p.sector_scale), p.sectors - 1);
    } else if constexpr (!TIMED && !RECS) {
      write_row();
    }
  };

  for (;;) {
    // ---------------------------------------------------------------- refill / launch
    const unsigned need = __ballot_sync(kFull, !alive && !exhausted);
    if (need) {
      const int leader = __ffs(need) - 1;
      unsigned long long base = 0;
      if (lane == leader) base = atomicAdd(p.work, (unsigned long long)__popc(need));
      base = __shfl_sync(kFull, base, leader);
      if (!alive && !exhausted) {
        const unsigned long long step = base + __popc(need & ((1u << lane) - 1u));
        if (step >= p.total_packets) {
          exhausted = true;
        } else {
          const unsigned long long g = p.order ? (unsigned long long)__ldg(p.order + step) : step;
          // the problem owning launch packet g: smallest pi with prob[pi].end > g
          int lo = 0;
          if (BATCH) {
            int hi = p.n_problems - 1;
            while (lo < hi) {
              const int mid = (lo + hi) >> 1;
              if (p.prob[mid].end > g)
                hi = mid;
              else
                lo = mid + 1;
            }
          }
          const ProblemDesc &P = p.prob[lo];
          const unsigned long long start = lo ? p.prob[lo - 1].end : 0ull;
          pid = P.first_packet + (g - start);
          if (BATCH) {
            mu = P.mu;
            prob = lo;
            nx = P.nx;
            nz = P.nz;
            dx = P.dx;
            hg_c = P.hg_c;
            qscale = P.qscale;
            key0 = P.key0;
            key1 = P.key1;
          }
          ++n_launch;
          float W0 = 1.f;
          bool inside = true;
          if (P.kind == kVolume) {
            const int npix = NX() * NZ();
            const unsigned long long total = __ldg(P.cdf + npix - 1);
            if (total == 0ull) {  // all-zero source: nothing to launch
              inside = false;
              W0 = 0.f;
            } else {
              const uint4 r0 = philox4x32_10(pid, 0u, KEY0(), KEY1());
              const uint4 r1 = philox4x32_10(pid, 1u, KEY0(), KEY1());
              const int pix = pick_pixel(P.cdf, npix, total, r0.x, r0.y);
              ix = pix % NX();
              iz = pix / NX();
              fx = u01(r1.x) * DX();
              fz = u01(r1.y) * DX();
              sincospif(2.f * u01(r0.z), &sx, &sz);
              W0 = __ldg(P.q + pix) < 0.f ? -1.f : 1.f;
            }
          } else {
            float x = P.x0, z = P.z0;
            sx = P.dir_x;
            sz = P.dir_z;
            if (P.kind == MCR_LINE) {
              const uint4 r0 = philox4x32_10(pid, 0u, KEY0(), KEY1());
              const float u = u01(r0.x);
              x = fmaf(u, P.x1 - P.x0, P.x0);
              z = fmaf(u, P.z1 - P.z0, P.z0);
            } else if (P.kind == MCR_ISO_POINT) {
              const uint4 r0 = philox4x32_10(pid, 0u, KEY0(), KEY1());
              sincospif(2.f * u01(r0.z), &sx, &sz);
            } else if (P.kind == MCR_ANGULAR_POINT) {
              const uint4 r0 = philox4x32_10(pid, 0u, KEY0(), KEY1());
              sincosf(launch_angle(P, u01(r0.z)), &sx, &sz);
            }
            inside = x >= 0.f && x <= NX() * DX() && z >= 0.f && z <= NZ() * DX();
            if (inside) {
              ix = min((int)floorf(x / DX()), NX() - 1);
              iz = min((int)floorf(z / DX()), NZ() - 1);
              fx = clamp_dx(x - ix * DX(), DX());
              fz = clamp_dx(z - iz * DX(), DX());
            }
          }
          W = W0;
          w_launch += W0;
          nscat = 0;
          flight = 0;
          plen = 0.f;
          if (!inside) {
            ++n_esc;
            w_esc += W;
          } else if (p.max_events == 0u) {
            ++n_evl;
            w_kill += W;
          } else {
            flight = 1;
            begin_flight();
            alive = true;
            if constexpr (!BATCH) mcur = load_mu();
          }
        }
      }
    }
    if (!__any_sync(kFull, alive)) break;
    __syncwarp();

    // ---------------------------------------------------------------- one pixel segment
    unsigned seg_key = 0u;  // (pixel + 1) << 6 | problem of this lane's segment (0: none)
    float seg_ts = 0.f;     // its track weight times 2^q
    float seg_w = 0.f, seg_l = 0.f, seg_l0 = 0.f, seg_mua = 0.f, seg_imua = 0.f;  // TIMED: the segment
    float dep_carry = 0.f;  // a deferred segment deposited with this one (same pixel)
    bool collided = false, escaped = false;
    if (alive) {
      const int pix = iz * NX() + ix;
      const float4 m = BATCH ? load_mu() : mcur;  // (mu_a, mu_s, 1/mu_a, 1/mu_s)
      float dist_x = CUDART_INF_F, dist_z = CUDART_INF_F;
      if (sx != 0.f) dist_x = fmaxf((sx > 0.f ? DX() - fx : fx) * inv_ax, 0.f);
      if (sz != 0.f) dist_z = fmaxf((sz > 0.f ? DX() - fz : fz) * inv_az, 0.f);
      const float d_edge = fminf(dist_x, dist_z);
      const float d_coll = tau * m.w;  // +inf when mu_s = 0 (tau > 0)
      collided = d_coll < d_edge;
      const float l = collided ? d_coll : d_edge;
      // track weight of the segment: W (1 - e^{-mu_a l}) / mu_a, then W <- W e^{-mu_a l}
      const float em1 = expm1f(-m.x * l);
      const float t = m.x > 0.f ? (-W * em1) * m.z : W * l;
      if constexpr (TIMED) {
        seg_w = W;
        seg_l = l;
        seg_l0 = plen;
        seg_mua = m.x;
        seg_imua = m.z;
        plen += l;
      }
      W = fmaf(W, em1, W);
      ++n_seg;
      if (MERGE) {
        dep_carry = carry;
        carry = 0.f;
      }
      if ((t != 0.f || dep_carry != 0.f) && MCR_GUARD(p.flags, isfinite(t))) {
        seg_key = ((unsigned)(pix + 1) << 6) | (unsigned)(BATCH ? prob : 0);
        seg_ts = t * QS();
      }
      if (MERGE && collided && dep_carry == 0.f && t != 0.f) {
        // defer if the packet survives this collision (the same tests as below): its next
        // segment starts in this pixel
        const bool dies = nscat >= p.max_scatter ||
                          (fabsf(W) < p.w_threshold && !(u01(cu2) < p.rr_p)) || flight >= p.max_events;
        if (!dies) {
          carry = seg_ts;
          carry_rb = rb;
          seg_key = 0u;
        }
      }
      if (collided) {
        fx = clamp_dx(fmaf(l, sx, fx), DX());
        fz = clamp_dx(fmaf(l, sz, fz), DX());
      } else {
        tau = fmaxf(fmaf(-m.y, l, tau), 0.f);
        if (dist_x <= dist_z) {  // ties: x first, z follows as a zero-length segment
          if (sx > 0.f) {
            ++ix;
            fx = 0.f;
          } else {
            --ix;
            fx = DX();
          }
          fz = clamp_dx(fmaf(l, sz, fz), DX());
        } else {
          if (sz > 0.f) {
            ++iz;
            fz = 0.f;
          } else {
            --iz;
            fz = DX();
          }
          fx = clamp_dx(fmaf(l, sx, fx), DX());
        }
        escaped = (unsigned)ix >= (unsigned)NX() || (unsigned)iz >= (unsigned)NZ();
        if (!BATCH && !escaped) mcur = __ldg(MU() + iz * NX() + ix);  // the next segment's pixel
      }
    }

    // ---------------------------------------------------------------- cooperative deposit
    if constexpr (SECT) {
      if (seg_key != 0u && row_ok(seg_key) && MCR_GUARD(p.flags, sect >= 0 && sect < p.Cpad))
        atomicAdd(tally_row(seg_key) + sect, (unsigned long long)(long long)__float2int_rn(seg_ts));
    }
    if constexpr (TIMED) {
      if (seg_key != 0u && row_ok(seg_key)) {
        // piece [s1, s2) of the segment in bin b: W e^{-mu_a s1} (1 - e^{-mu_a (s2 - s1)}) / mu_a
        unsigned long long *row = tally_row(seg_key);
        const int T = p.time_bins;
        const float w = p.time_bin_mm;
        // start one bin early: a rounded-up first index must not drop the segment's first sliver
        for (int b = max(min((int)(seg_l0 * p.inv_time_bin), T - 1) - 1, 0);; ++b) {
          const float s1 = fmaxf(fmaf((float)b, w, -seg_l0), 0.f);
          const float s2 = b + 1 == T ? seg_l : fminf(fmaf((float)(b + 1), w, -seg_l0), seg_l);
          if (s2 > s1) {
            const float d = s2 - s1;
            const float tp = seg_mua > 0.f ? seg_w * expf(-seg_mua * s1) * -expm1f(-seg_mua * d) * seg_imua
                                           : seg_w * d;
            if (MCR_GUARD(p.flags, b >= 0 && b < p.Cpad))
              atomicAdd(row + b, (unsigned long long)(long long)__float2int_rn(tp * QS()));
          }
          if (s2 >= seg_l || b + 1 == T) break;
        }
      }
    }
    if constexpr (RECS) {
      const unsigned has = __ballot_sync(kFull, seg_key != 0u);
      if (has) {  // coalesced 16-byte record stores into the warp's own block of slots
        const unsigned n = __popc(has);
        if (rec_fill + n > kRecBlock) {  // warp-uniform: close the block, reserve the next one
          rec_pad();
          unsigned long long nb = 0;
          if (lane == 0) nb = atomicAdd(p.rec_count, (unsigned long long)kRecBlock);
          rec_block = __shfl_sync(kFull, nb, 0);
          rec_fill = 0;
        }
        if (seg_key != 0u) {
          const unsigned long long slot = rec_block + rec_fill + __popc(has & ((1u << lane) - 1u));
          const unsigned pix = (seg_key >> 6) - 1u;
          if (slot < p.rec_capacity && row_ok(seg_key)) {
            p.records[slot] = make_float4(__uint_as_float(pix), seg_ts, sx, sz);
            atomicAdd(p.rec_hist + pix, 1u);
          } else {
            atomicOr(p.rec_overflow, 1u);
          }
        }
        rec_fill += n;
      }
    }
    unsigned pend = ROWLESS ? 0u : __ballot_sync(kFull, seg_key != 0u);
    if (pend) {
      // lanes with the same tally row (one pending lane -- the runs' tails -- needs no match)
      const unsigned same = (pend & (pend - 1u)) == 0u ? (1u << lane) : __match_any_sync(kFull, seg_key);
      // Rows of a single lane without a carried segment (nearly all of them away from the source)
      // go kRowsPerStep at a time: their shuffles, loads, conversions and reductions are
      // independent, so they overlap instead of running as one dependent chain per row.
      unsigned easy = pend & __ballot_sync(kFull, seg_key != 0u && same == (1u << lane) && !(MERGE && dep_carry != 0.f));
      pend &= ~easy;
      while (easy) {
        bool on[kRowsPerStep];
        float ts[kRowsPerStep];
        unsigned long long *dst[kRowsPerStep];
        const float *hr[kRowsPerStep];
#pragma unroll
        for (int r = 0; r < kRowsPerStep; ++r) {
          on[r] = easy != 0u;  // warp-uniform
          const int L = on[r] ? __ffs(easy) - 1 : 0;
          easy &= easy - 1u;
          unsigned key = on[r] ? __shfl_sync(kFull, seg_key, L) : 64u;
          if (on[r] && !row_ok(key)) {  // warp-uniform (checked build only)
            on[r] = false;
            key = 64u;
          }
          ts[r] = __shfl_sync(kFull, seg_ts, L);
          dst[r] = tally_row(key) + c0;
          hr[r] = rows + ((MERGE ? __shfl_sync(kFull, rb, L) * 32 : 0) + L) * p.row_stride + 1 + c0;
        }
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const int j = q * 32 + lane;
          if (j < Cw) {
#pragma unroll
            for (int r = 0; r < kRowsPerStep; ++r)
              if (on[r]) atomicAdd(dst[r] + j, (unsigned long long)(long long)__float2int_rn(ts[r] * hr[r][j]));
          }
        }
      }
      while (pend) {
        const int L = __ffs(pend) - 1;
        const unsigned grp = __shfl_sync(kFull, same, L) & pend;
        const unsigned key = __shfl_sync(kFull, seg_key, L);
        unsigned long long *dst = tally_row(key) + c0;
        long long acc[NP > 0 ? NP : 1];
        // |t h 2^q| < 2^31 by the choice of q, so a 32-bit conversion suffices
        const float tsL = __shfl_sync(kFull, seg_ts, L);
        const float *hrL = rows + ((MERGE ? __shfl_sync(kFull, rb, L) * 32 : 0) + L) * p.row_stride + 1 + c0;
#pragma unroll
        for (int q = 0; q < NP; ++q) {
          const int j = q * 32 + lane;
          acc[q] = j < Cw ? (long long)__float2int_rn(tsL * hrL[j]) : 0;
        }
        if (MERGE) {
          const float cL = __shfl_sync(kFull, dep_carry, L);
          if (cL != 0.f) {
            const float *hc = rows + (__shfl_sync(kFull, carry_rb, L) * 32 + L) * p.row_stride + 1 + c0;
#pragma unroll
            for (int q = 0; q < NP; ++q) {
              const int j = q * 32 + lane;
              if (j < Cw) acc[q] += (long long)__float2int_rn(cL * hc[j]);
            }
          }
        }
        unsigned g = grp & (grp - 1);  // other lanes in the same tally row (rare outside beams)
        while (g) {
          const int M = __ffs(g) - 1;
          g &= g - 1;
          const float ts = __shfl_sync(kFull, seg_ts, M);
          const float *hr = rows + ((MERGE ? __shfl_sync(kFull, rb, M) * 32 : 0) + M) * p.row_stride + 1 + c0;
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const int j = q * 32 + lane;
            if (j < Cw) acc[q] += (long long)__float2int_rn(ts * hr[j]);
          }
          if (MERGE) {
            const float cM = __shfl_sync(kFull, dep_carry, M);
            if (cM != 0.f) {
              const float *hc = rows + (__shfl_sync(kFull, carry_rb, M) * 32 + M) * p.row_stride + 1 + c0;
#pragma unroll
              for (int q = 0; q < NP; ++q) {
                const int j = q * 32 + lane;
                if (j < Cw) acc[q] += (long long)__float2int_rn(cM * hc[j]);
              }
            }
          }
        }
        if (row_ok(key)) {
#pragma unroll
          for (int q = 0; q < NP; ++q) {
            const int j = q * 32 + lane;
            if (j < Cw) atomicAdd(dst + j, (unsigned long long)acc[q]);
          }
        }
        pend &= ~grp;
      }
      if (dense) {  // coefficient 0: h_0 = 1, so each product is the rounded track weight itself
        if (seg_key != 0u) {
          long long v = (long long)__float2int_rn(seg_ts);
          if (MERGE && dep_carry != 0.f) v += (long long)__float2int_rn(dep_carry);
          if (seg_key != acc0_key) {
            flush0();
            acc0_key = seg_key;
            acc0 = v;
          } else {
            acc0 += v;
          }
        }
      } else if (!ROWLESS && Cw < C && seg_key != 0u && row_ok(seg_key)) {  // the per-lane remainder
        unsigned long long *own = tally_row(seg_key);
        const float *h = rows + ((MERGE ? rb * 32 : 0) + lane) * p.row_stride + 1;
        const float *hc = rows + ((MERGE ? carry_rb * 32 : 0) + lane) * p.row_stride + 1;
        for (int j = Cw; j < C; ++j) {
          long long v = (long long)__float2int_rn(seg_ts * h[j]);
          if (MERGE && dep_carry != 0.f) v += (long long)__float2int_rn(dep_carry * hc[j]);
          atomicAdd(own + j, (unsigned long long)v);
        }
      }
    }
    __syncwarp();

    // ---------------------------------------------------------------- escape / collision
    if (alive) {
      if (escaped) {
        ++n_esc;
        w_esc += W;
        alive = false;
      } else if (collided) {
        ++n_coll;
        if (nscat >= p.max_scatter) {
          ++n_scl;
          w_kill += W;
          alive = false;
        } else {
          // 2D HG angle theta_s = 2 atan(c tan(pi U)) (Eq. 7), applied as a rotation with
          // cos theta_s = (cp^2 - c^2 sp^2)/(cp^2 + c^2 sp^2), sin theta_s = 2 c sp cp/(...),
          // (sp, cp) = (sin pi U, cos pi U): the same angle without tan's pole at U = 1/2.
          float sp, cp;
          sincospif(u01(cu1), &sp, &cp);
          const float a = cp * cp, b = HGC() * HGC() * sp * sp;
          const float inv = 1.f / (a + b);
          const float cs = (a - b) * inv, sn = 2.f * HGC() * sp * cp * inv;
          const float nsx = fmaf(sx, cs, sz * sn), nsz = fmaf(sz, cs, -sx * sn);
          const float rn = rsqrtf(fmaf(nsx, nsx, nsz * nsz));
          sx = nsx * rn;
          sz = nsz * rn;
          ++nscat;
          if (fabsf(W) < p.w_threshold) {  // |W0| = 1
            if (u01(cu2) < p.rr_p) {
              const float Wn = W * p.rr_inv_p;
              w_rr += (double)Wn - (double)W;
              W = Wn;
              ++n_rrs;
            } else {
              w_rr -= W;
              ++n_rrk;
              alive = false;
            }
          }
          if (alive) {
            if (flight >= p.max_events) {
              ++n_evl;
              w_kill += W;
              alive = false;
            } else {
              ++flight;
              begin_flight();
            }
          }
        }
      }
    }
    __syncwarp();
  }

  if constexpr (RECS) rec_pad();  // the warp's last block
  if (dense) flush0();            // the lane's last pending coefficient 0
  // ---------------------------------------------------------------- counters
  const unsigned c_launch = __reduce_add_sync(kFull, n_launch), c_flight = __reduce_add_sync(kFull, n_flight),
                 c_coll = __reduce_add_sync(kFull, n_coll), c_seg = __reduce_add_sync(kFull, n_seg),
                 c_esc = __reduce_add_sync(kFull, n_esc), c_rrk = __reduce_add_sync(kFull, n_rrk),
                 c_rrs = __reduce_add_sync(kFull, n_rrs), c_scl = __reduce_add_sync(kFull, n_scl),
                 c_evl = __reduce_add_sync(kFull, n_evl);
  w_launch = warp_sum(w_launch);
  w_esc = warp_sum(w_esc);
  w_rr = warp_sum(w_rr);
  w_kill = warp_sum(w_kill);
  if (lane == 0 && c_evl) atomicOr(p.flags, kFlagEventLimit);
  if (lane == 0 && c_launch) {
    DevStats *s = p.stats;
    atomicAdd(&s->launched, (unsigned long long)c_launch);
    atomicAdd(&s->flights, (unsigned long long)c_flight);
    atomicAdd(&s->collisions, (unsigned long long)c_coll);
    atomicAdd(&s->segments, (unsigned long long)c_seg);
    atomicAdd(&s->escapes, (unsigned long long)c_esc);
    if (c_rrk) atomicAdd(&s->rr_kill, (unsigned long long)c_rrk);
    if (c_rrs) atomicAdd(&s->rr_survive, (unsigned long long)c_rrs);
    if (c_scl) atomicAdd(&s->scatter_limit, (unsigned long long)c_scl);
    if (c_evl) atomicAdd(&s->event_limit, (unsigned long long)c_evl);
    atomicAdd(&s->launched_w, w_launch);
    atomicAdd(&s->escaped_w, w_esc);
    atomicAdd(&s->rr_net_w, w_rr);
    atomicAdd(&s->killed_w, w_kill);
  }
  if (STALLY) {  // the block's tally into the global one: coalesced, zero words skipped (with a row
                 // offset the last slot's last words map past the tally; they are never written)
    __syncthreads();
    const size_t nw = (size_t)p.prob[0].nx * p.prob[0].nz * p.Cpad;
    unsigned long long *g = p.prob[0].tally;
    for (size_t i = threadIdx.x; i < nw; i += blockDim.x) {
      const unsigned long long v = stally[i];
      if (v) atomicAdd(g + i, v);
    }
  }
}

// ---------------------------------------------------------------- launch order
constexpr int kLineBinsLog2 = 12;  // bins along a line source
constexpr int kOrderTile = 32;     // volumetric sources: tiles of kOrderTile^2 pixels

__device__ __forceinline__ int problem_of(const TransportParams &p, unsigned long long g) {
  int lo = 0, hi = p.n_problems - 1;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (p.prob[mid].end > g)
      hi = mid;
    else
      lo = mid + 1;
  }
  return lo;
}

// The launch-order bin of launch index g: from the same random numbers the launch draws (line
// position: block 0 word 0; volumetric pixel: block 0 words 0-1), so it is where the packet starts.
__device__ unsigned launch_bin(const TransportParams &p, unsigned long long g) {
  const int pi = problem_of(p, g);
  const ProblemDesc &P = p.prob[pi];
  const unsigned long long pid = P.first_packet + (g - (pi ? p.prob[pi - 1].end : 0ull));
  unsigned bin = 0;
  if (P.kind == MCR_LINE) {
    bin = philox4x32_10(pid, 0u, P.key0, P.key1).x >> (32 - kLineBinsLog2);
  } else if (P.kind == kVolume) {
    const int npix = P.nx * P.nz;
    const unsigned long long total = __ldg(P.cdf + npix - 1);
    if (total != 0ull) {
      const uint4 r0 = philox4x32_10(pid, 0u, P.key0, P.key1);
      const int pix = pick_pixel(P.cdf, npix, total, r0.x, r0.y);
      const int ntx = (P.nx + kOrderTile - 1) / kOrderTile;
      bin = (unsigned)((pix / P.nx) / kOrderTile * ntx + (pix % P.nx) / kOrderTile);
    }
  }
  return P.bin_base + bin;
}

__global__ void k_order_count(const __grid_constant__ TransportParams p, unsigned *hist) {
  for (unsigned long long g = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; g < p.total_packets;
       g += (unsigned long long)gridDim.x * blockDim.x)
    atomicAdd(hist + launch_bin(p, g), 1u);
}

// Exclusive scan of the bin counts in place (one block of 1024 threads, chunks of 1024).
__global__ void k_order_scan(unsigned *hist, unsigned n) {
  __shared__ unsigned warp_tot[32];
  __shared__ unsigned carry;
  if (threadIdx.x == 0) carry = 0u;
  __syncthreads();
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
  for (unsigned base = 0; base < n; base += 1024) {
    const unsigned i = base + threadIdx.x;
    const unsigned x = i < n ? hist[i] : 0u;
    unsigned v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(kFull, v, o);
      if (lane >= o) v += t;
    }
    if (lane == 31) warp_tot[wid] = v;
    __syncthreads();
    if (wid == 0) {
      unsigned t = warp_tot[lane];
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const unsigned u = __shfl_up_sync(kFull, t, o);
        if (lane >= o) t += u;
      }
      warp_tot[lane] = t;
    }
    __syncthreads();
    const unsigned incl = v + (wid ? warp_tot[wid - 1] : 0u);
    if (i < n) hist[i] = carry + incl - x;
    __syncthreads();
    if (threadIdx.x == 1023) carry += incl;
    __syncthreads();
  }
}

__global__ void k_order_place(const __grid_constant__ TransportParams p, unsigned *cursor, unsigned *order) {
  for (unsigned long long g = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; g < p.total_packets;
       g += (unsigned long long)gridDim.x * blockDim.x)
    order[atomicAdd(cursor + launch_bin(p, g), 1u)] = (unsigned)g;
}

size_t shared_tally_bytes(const TransportParams &p) {
  return (size_t)p.prob[0].nx * p.prob[0].nz * p.Cpad * sizeof(unsigned long long);
}

// Opts the kernel into `smem` bytes of dynamic shared memory (once per device) and returns how
// many blocks of `threads` fit on one SM.
// Guards the per-instantiation caches of the opted-in shared-memory size: entry points that
// do not hold the workspace lock (mc_forward_noalloc) reach them from any host thread.
std::mutex g_attr_mu;

template <int NP, bool BATCH, bool MERGE, bool STALLY = false, bool RECS = false>
cudaError_t blocks_per_sm(int threads, size_t smem, int *per_sm) {
  static int configured[64];  // largest dynamic smem opted in, per device
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (smem > 232448) {  // more than a block may have: does not fit
    *per_sm = 0;
    return cudaSuccess;
  }
  {
    std::lock_guard<std::mutex> lock(g_attr_mu);
    if (dev >= 64 || configured[dev] < (int)smem) {
      e = cudaFuncSetAttribute(k_transport<NP, BATCH, MERGE, STALLY, RECS>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
      if (e != cudaSuccess) return e;
      if (dev < 64) configured[dev] = (int)smem;
    }
  }
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, k_transport<NP, BATCH, MERGE, STALLY, RECS>, threads,
                                                       smem);
}

template <int NP, bool BATCH, bool MERGE, bool STALLY = false, bool RECS = false>
cudaError_t launch_kernel(const TransportParams &p, int threads, int cap, cudaStream_t s) {
  if (threads % 32 || threads > 256 || threads <= 0) return cudaErrorInvalidValue;
  const size_t smem = RECS ? 16 : transport_smem_bytes(p.row_stride, threads, MERGE) + (STALLY ? shared_tally_bytes(p) : 0);
  int dev = 0, sms = 0, per_sm = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  e = blocks_per_sm<NP, BATCH, MERGE, STALLY, RECS>(threads, smem, &per_sm);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  if (cap > 0 && cap < per_sm) per_sm = cap;
  k_transport<NP, BATCH, MERGE, STALLY, RECS><<<sms * per_sm, threads, smem, s>>>(p);
  return cudaGetLastError();
}

// Default deposit mode: merge collisions when the second harmonic row per lane costs no resident
// warps; otherwise only when the tallies are far larger than L2 (their reductions then go to
// HBM and are the cost that matters), with 96-thread blocks.
template <int NP, bool BATCH>
cudaError_t launch_b(const TransportParams &p, const TransportLaunch &cfg, cudaStream_t s) {
  int threads = cfg.threads_per_block > 0 ? cfg.threads_per_block : 128;
  bool merge = cfg.merge == 2;
  if (cfg.merge == 0) {
    int plain = 0, merged = 0;
    cudaError_t e = blocks_per_sm<NP, BATCH, false>(threads, transport_smem_bytes(p.row_stride, threads, false), &plain);
    if (e != cudaSuccess) return e;
    e = blocks_per_sm<NP, BATCH, true>(threads, transport_smem_bytes(p.row_stride, threads, true), &merged);
    if (e != cudaSuccess) return e;
    merge = merged >= plain;
    if (!merge && cfg.threads_per_block == 0) {
      double tally = 0.0;
      for (int i = 0; i < p.n_problems; ++i) tally += (double)p.prob[i].nx * p.prob[i].nz * p.Cpad * 8.0;
      if (tally > kL2SpillBytes) {
        merge = true;
        threads = 96;
      }
    }
  }
  if constexpr (NP == 1 && !BATCH) {
    // per-block shared-memory tally when asked for and it fits beside the harmonic rows
    if (cfg.shared_tally == 2) {
      int per_sm = 0;
      const size_t smem = transport_smem_bytes(p.row_stride, threads, merge) + shared_tally_bytes(p);
      cudaError_t e = merge ? blocks_per_sm<1, false, true, true>(threads, smem, &per_sm)
                            : blocks_per_sm<1, false, false, true>(threads, smem, &per_sm);
      if (e != cudaSuccess) return e;
      if (per_sm >= 1)
        return merge ? launch_kernel<1, false, true, true>(p, threads, cfg.blocks_per_sm, s)
                     : launch_kernel<1, false, false, true>(p, threads, cfg.blocks_per_sm, s);
    }
  }
  return merge ? launch_kernel<NP, BATCH, true>(p, threads, cfg.blocks_per_sm, s)
               : launch_kernel<NP, BATCH, false>(p, threads, cfg.blocks_per_sm, s);
}

// a table of one reads its problem as uniform parameters; larger tables cache it per lane
template <int NP>
cudaError_t launch_np(const TransportParams &p, const TransportLaunch &cfg, cudaStream_t s) {
  return p.n_problems > 1 ? launch_b<NP, true>(p, cfg, s) : launch_b<NP, false>(p, cfg, s);
}

}  // namespace

unsigned order_bins(const ProblemDesc &d) {
  if (d.kind == MCR_LINE) return 1u << kLineBinsLog2;
  if (d.kind == kVolume)
    return (unsigned)(((d.nx + kOrderTile - 1) / kOrderTile) * ((d.nz + kOrderTile - 1) / kOrderTile));
  return 1u;
}

cudaError_t launch_order(const TransportParams &p, unsigned total_bins, unsigned *hist, unsigned *order,
                         cudaStream_t s) {
  if (p.total_packets == 0 || p.total_packets > 0xFFFFFFFFull) return cudaErrorInvalidValue;
  cudaError_t e = cudaMemsetAsync(hist, 0, (size_t)total_bins * sizeof(unsigned), s);
  if (e != cudaSuccess) return e;
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned long long want = (p.total_packets + 255) / 256;
  const unsigned grid = (unsigned)(want < (unsigned long long)sms * 8 ? want : (unsigned long long)sms * 8);
  k_order_count<<<grid, 256, 0, s>>>(p, hist);
  k_order_scan<<<1, 1024, 0, s>>>(hist, total_bins);
  k_order_place<<<grid, 256, 0, s>>>(p, hist, order);
  return cudaGetLastError();
}

size_t transport_smem_bytes(int row_stride, int threads, bool merge) {
  return (size_t)threads * row_stride * sizeof(float) * (merge ? 2 : 1);
}



cudaError_t launch_transport_records(const TransportParams &p, const TransportLaunch &cfg, cudaStream_t s) {
  if (p.n_problems != 1 || p.sectors > 0 || p.time_bins > 0 || !p.records) return cudaErrorInvalidValue;
  return launch_kernel<1, false, false, false, true>(p, cfg.threads_per_block > 0 ? cfg.threads_per_block : 128,
                                                    cfg.blocks_per_sm, s);
}

cudaError_t launch_transport(const TransportParams &p, const TransportLaunch &cfg, cudaStream_t s) {
  if (p.sectors > 0 || p.time_bins > 0) {  // discrete ordinates / time bins: one plain forward problem
    if (p.n_problems != 1) return cudaErrorInvalidValue;
    const int threads = cfg.threads_per_block > 0 ? cfg.threads_per_block : 128;
    return p.sectors > 0 ? launch_kernel<0, false, false>(p, threads, cfg.blocks_per_sm, s)
                         : launch_kernel<-1, false, false>(p, threads, cfg.blocks_per_sm, s);
  }
  // chunks of 32 coefficients deposited cooperatively (a remainder of <= 4 goes per lane)
  const int cw = (p.C & 31) <= 4 ? (p.C & ~31) : p.C;
  const int np = cw > 32 ? (cw + 31) / 32 : 1;
  switch (np) {
    case 1: return launch_np<1>(p, cfg, s);
    case 2: return launch_np<2>(p, cfg, s);
    case 3: return launch_np<3>(p, cfg, s);
    case 4: return launch_np<4>(p, cfg, s);
    case 5: return launch_np<5>(p, cfg, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mcr
