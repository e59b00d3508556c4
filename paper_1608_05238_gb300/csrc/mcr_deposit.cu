// mcr_deposit.cu -- the sorted-record deposit of the harmonic tally (Sec. 3.1, Eqs. 9-11) for
// tallies too large for L2 (e.g. 1024^2 pixels at K = 64: 1.2 GB).
//
// The direct deposit adds every segment's 2K+1 products into the pixel's tally row at once.  With
// packets spread over the whole domain the row is almost never in L2, so each segment costs a
// read and a write of the row in HBM (~2.3 KB at K = 64).  Here the transport (k_transport in
// record mode) only writes one 16-byte record per segment -- pixel, track weight x 2^q, direction --
// and counts it for its pixel.  Then:
//   1. an exclusive scan of the per-pixel counts gives each pixel's first slot;
//   2. one scatter puts the records in pixel order (a counting sort: the order within a pixel is
//      whatever the atomics give, which does not matter for an integer sum);
//   3. k_deposit_sorted walks the sorted records: each lane rebuilds the harmonic row of its
//      record with the transport's own harmonic_row (bit-identical coefficients), the warp sums
//      the rounded products round(t 2^q h_c) of a pixel's run in 64-bit registers, coefficient c
//      on lane c mod 32, and adds the run's sums to the tally row with one coalesced reduction
//      per coefficient when the pixel changes.
// Every product is rounded exactly as in the direct deposit and integer addition is exact, so the
// tally is bit-identical; HBM sees the records (written, read, scattered, read: ~100 B per
// segment) and each row once per chunk of packets.
#include "mcr_harmonics.cuh"
#include "mcr_internal.h"

namespace mcr {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kScanThreads = 256;

// Block-local exclusive scan of hist into cursor; block totals into block_sums.
__global__ void k_scan_local(const unsigned *__restrict__ hist, int n, unsigned *__restrict__ cursor,
                             unsigned *__restrict__ block_sums) {
  __shared__ unsigned warp_tot[kScanThreads / 32];
  const int i = blockIdx.x * kScanThreads + threadIdx.x;
  const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
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
    unsigned t = lane < kScanThreads / 32 ? warp_tot[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned u = __shfl_up_sync(kFull, t, o);
      if (lane >= o) t += u;
    }
    if (lane < kScanThreads / 32) warp_tot[lane] = t;
  }
  __syncthreads();
  const unsigned incl = v + (wid ? warp_tot[wid - 1] : 0u);
  if (i < n) cursor[i] = incl - x;
  if (threadIdx.x == kScanThreads - 1) block_sums[blockIdx.x] = incl;
}

// Exclusive scan of the block totals (one warp, chunks of 32 in order).
__global__ void k_scan_blocks(unsigned *block_sums, int nblocks) {
  const int lane = threadIdx.x;
  unsigned carry = 0;
  for (int base = 0; base < nblocks; base += 32) {
    const int i = base + lane;
    const unsigned x = i < nblocks ? block_sums[i] : 0u;
    unsigned v = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const unsigned t = __shfl_up_sync(kFull, v, o);
      if (lane >= o) v += t;
    }
    if (i < nblocks) block_sums[i] = carry + v - x;
    carry += __shfl_sync(kFull, v, 31);
  }
  if (lane == 0) block_sums[nblocks] = carry;  // the grand total: the number of records
}

__global__ void k_scan_add(unsigned *__restrict__ cursor, int n, const unsigned *__restrict__ block_sums) {
  const int i = blockIdx.x * kScanThreads + threadIdx.x;
  if (i < n) cursor[i] += block_sums[blockIdx.x];
}

// Records into pixel order: each takes the next slot of its pixel.
__global__ void k_scatter_records(const float4 *__restrict__ rec, unsigned long long n, unsigned *__restrict__ cursor,
                                  float4 *__restrict__ sorted, int npix, unsigned *flags) {
  for (unsigned long long i = blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x; i < n;
       i += (unsigned long long)gridDim.x * blockDim.x) {
    const float4 r = rec[i];
    if (__float_as_uint(r.x) == kRecSentinel) continue;  // an unused slot of a warp's block
    if (MCR_GUARD(flags, __float_as_uint(r.x) < (unsigned)npix)) {
      const unsigned slot = atomicAdd(cursor + __float_as_uint(r.x), 1u);
      if (MCR_GUARD(flags, slot < n)) sorted[slot] = r;
    }
  }
}

// Pixel runs of the sorted records into the tally.  Each warp owns a contiguous span of records;
// NPK = ceil((2K+1) / 32) coefficient chunks, coefficient j = 32 q + lane of chunk q.
template <int NPK>
__global__ void __launch_bounds__(128) k_deposit_sorted(const float4 *__restrict__ rec, const unsigned *n_records, int K,
                                                       int row_stride, int Cpad, int npix,
                                                       unsigned long long *__restrict__ tally, unsigned *flags) {
  extern __shared__ float smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned long long n = *n_records;  // the records the scan counted (sentinels excluded)
  float *const rows = smem + (size_t)warp * 32 * row_stride;  // the warp's 32 rows
  const int C = 2 * K + 1;
  const unsigned long long nwarps = (unsigned long long)gridDim.x * (blockDim.x >> 5);
  const unsigned long long gw = (unsigned long long)blockIdx.x * (blockDim.x >> 5) + warp;
  const unsigned long long per = ((n + nwarps - 1) / nwarps + 31) & ~31ull;
  const unsigned long long lo = gw * per, hi = lo + per < n ? lo + per : n;
  if (lo >= hi) return;

  long long acc[NPK];
#pragma unroll
  for (int q = 0; q < NPK; ++q) acc[q] = 0;
  unsigned cur = __float_as_uint(__ldg(&rec[lo].x));  // pixel of the current run
  auto flush = [&]() {
    if (!MCR_GUARD(flags, cur < (unsigned)npix)) return;
    unsigned long long *dst = tally + (size_t)cur * Cpad;
#pragma unroll
    for (int q = 0; q < NPK; ++q) {
      const int j = q * 32 + lane;
      if (j < C && acc[q] != 0) atomicAdd(dst + j, (unsigned long long)acc[q]);
      acc[q] = 0;
    }
  };
  for (unsigned long long b = lo; b < hi; b += 32) {
    const int nv = hi - b < 32 ? (int)(hi - b) : 32;
    float4 r = make_float4(0.f, 0.f, 0.f, 1.f);
    if (lane < nv) r = rec[b + lane];
    harmonic_row(rows + lane * row_stride, r.z, r.w, K);  // (s_x, s_z) of the record's flight
    __syncwarp();
    const unsigned key = __float_as_uint(r.x);
    for (int i = 0; i < nv; ++i) {
      const unsigned ki = __shfl_sync(kFull, key, i);
      const float ts = __shfl_sync(kFull, r.y, i);
      if (ki != cur) {  // warp-uniform: the run of `cur` ends
        flush();
        cur = ki;
      }
      const float *h = rows + i * row_stride + 1;
#pragma unroll
      for (int q = 0; q < NPK; ++q) {
        const int j = q * 32 + lane;
        if (j < C) acc[q] += (long long)__float2int_rn(ts * h[j]);
      }
    }
    __syncwarp();
  }
  flush();
}

int grid_for(unsigned long long n, int threads, int per_sm) {
  int dev = 0, sms = 148;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const unsigned long long want = (n + threads - 1) / threads;
  const unsigned long long cap = (unsigned long long)sms * per_sm;
  return (int)(want < 1 ? 1 : (want < cap ? want : cap));
}

template <int NPK>
cudaError_t launch_deposit(const float4 *sorted, unsigned long long n, const unsigned *n_records, int K, int Cpad,
                           int npix, unsigned long long *tally, unsigned *flags, cudaStream_t s) {
  const int row_stride = transport_row_stride(2 * K + 1);
  const int threads = 128;
  const size_t smem = (size_t)(threads / 32) * 32 * row_stride * sizeof(float);
  static bool configured[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !configured[dev]) {  // the largest rows (K = 64) need more than 48 KB per block
    cudaError_t e = cudaFuncSetAttribute(k_deposit_sorted<NPK>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)(4 * 32 * transport_row_stride(2 * MCR_MAX_K + 1) * sizeof(float)));
    if (e != cudaSuccess) return e;
    configured[dev] = true;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_deposit_sorted<NPK>, threads, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  // about 32 records per warp at least, so that a span is not shorter than one batch
  const int blocks = grid_for((n + 31) / 32, threads / 32, per_sm);
  k_deposit_sorted<NPK><<<blocks, threads, smem, s>>>(sorted, n_records, K, row_stride, Cpad, npix, tally, flags);
  return cudaGetLastError();
}

__global__ void k_add_stats(DevStats *dst, const DevStats *src) {
  dst->launched += src->launched;
  dst->flights += src->flights;
  dst->collisions += src->collisions;
  dst->segments += src->segments;
  dst->escapes += src->escapes;
  dst->rr_kill += src->rr_kill;
  dst->rr_survive += src->rr_survive;
  dst->scatter_limit += src->scatter_limit;
  dst->event_limit += src->event_limit;
  dst->launched_w += src->launched_w;
  dst->escaped_w += src->escaped_w;
  dst->rr_net_w += src->rr_net_w;
  dst->killed_w += src->killed_w;
}

}  // namespace

cudaError_t launch_add_stats(DevStats *dst, const DevStats *src, cudaStream_t s) {
  k_add_stats<<<1, 1, 0, s>>>(dst, src);
  return cudaGetLastError();
}

cudaError_t launch_sort_and_deposit(const float4 *records, unsigned long long n, const unsigned *hist,
                                    unsigned *cursor, unsigned *block_sums, int npix, float4 *sorted, int K, int Cpad,
                                    unsigned long long *tally, unsigned *flags, cudaStream_t s) {
  if (n == 0) return cudaSuccess;
  const int nblocks = (npix + kScanThreads - 1) / kScanThreads;
  k_scan_local<<<nblocks, kScanThreads, 0, s>>>(hist, npix, cursor, block_sums);
  k_scan_blocks<<<1, 32, 0, s>>>(block_sums, nblocks);
  k_scan_add<<<nblocks, kScanThreads, 0, s>>>(cursor, npix, block_sums);
  k_scatter_records<<<grid_for(n, 256, 8), 256, 0, s>>>(records, n, cursor, sorted, npix, flags);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  switch ((2 * K + 1 + 31) / 32) {
    case 1: return launch_deposit<1>(sorted, n, block_sums + nblocks, K, Cpad, npix, tally, flags, s);
    case 2: return launch_deposit<2>(sorted, n, block_sums + nblocks, K, Cpad, npix, tally, flags, s);
    case 3: return launch_deposit<3>(sorted, n, block_sums + nblocks, K, Cpad, npix, tally, flags, s);
    case 4: return launch_deposit<4>(sorted, n, block_sums + nblocks, K, Cpad, npix, tally, flags, s);
    case 5: return launch_deposit<5>(sorted, n, block_sums + nblocks, K, Cpad, npix, tally, flags, s);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace mcr
