// mcr_noalloc.cu -- mc_forward_noalloc: the forward transport with its scratch memory (packed
// medium, 64-bit fixed-point tally, counters) in a fixed-size array that is part of the loaded
// library, so that the call performs no device allocation at all.
//
// Who needs this: callers that may not call cudaMalloc on the path where they run the forward
// model -- code whose device memory is entirely owned by another allocator or memory pool (the
// library's own grow-only workspace would compete with it), latency-critical loops where the
// implicit device synchronisation of cudaMalloc/cudaFree is not acceptable, and hosts that
// forbid allocation after start-up.  They pass their own input and output buffers; everything
// else the kernels need lives in g_scratch below.
#include <math.h>
#include <string.h>

#include <mutex>

#include "mcr_internal.h"

namespace {

// Every GPU that loads libmcr holds this array (16 MiB) until the process exits.
constexpr size_t kScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

// Layout inside g_scratch: [0, 512) counters and flags, then the packed medium, then the tally.
// The flags word holds the current call's error bits (the transport reads its medium bit);
// the latched word collects the bits of every call until mc_check reads and clears it.
constexpr size_t kOffWork = 0, kOffStats = 64, kOffFlags = 256, kOffLatched = 260, kSmall = 512;

// Moves the previous call's error bits into the latched word and clears them for this call.
__global__ void k_latch_flags(unsigned *flags, unsigned *latched) {
  *latched |= *flags;
  *flags = 0u;
}

constexpr int kMaxDev = 64;
std::mutex g_setup_mu;
unsigned char *g_scratch_ptr[kMaxDev];  // device address of g_scratch, per device

// Device address of g_scratch on the current device.  In host code `g_scratch` names a host-side
// stand-in, not device memory, so the address is asked from the runtime once per device (with
// that device current) and cached.  With lookup = false only an address already cached is
// returned (nullptr if this device never ran the entry point).
int scratch_address(unsigned char **out, bool lookup = true) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDev) return MCR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mu);
  if (!g_scratch_ptr[dev] && lookup) {
    void *p = nullptr;
    if (cudaGetSymbolAddress(&p, g_scratch) != cudaSuccess || !p) {
      cudaGetLastError();
      return MCR_ERR_CUDA;
    }
    g_scratch_ptr[dev] = static_cast<unsigned char *>(p);
  }
  *out = g_scratch_ptr[dev];
  return MCR_OK;
}

size_t round256(size_t b) { return (b + 255) & ~size_t(255); }

}  // namespace

extern "C" {

int mc_forward_noalloc(const mcr_medium *med, const mcr_source *src, const mcr_run *run, float *coeff,
                       void *stream) {
  using namespace mcr;
  // the same argument checks as mc_forward
  int rc;
  if ((rc = check_medium(med)) || (rc = check_run(run))) return rc;
  if (!coeff) return MCR_ERR_ARG;
  if (run->sectors || run->time_bins) return MCR_ERR_ARG;  // these tallies run through mc_forward only
  float dirx = 0.f, dirz = 1.f;
  if (!src) return MCR_ERR_ARG;
  if ((rc = check_source(src, &dirx, &dirz))) return rc;
  // size limits of the fixed scratch: one transport launch (no FP64 chunk accumulator)
  if (run->n_packets > kChunkPackets) return MCR_ERR_SCRATCH;
  const int64_t npix = (int64_t)med->nx * med->nz;
  const int C = 2 * run->K + 1, Cpad = tally_row_words(C);
  const size_t mu_bytes = round256((size_t)npix * sizeof(float4));
  const size_t tally_bytes = (size_t)npix * Cpad * 8;
  if (kSmall + mu_bytes + tally_bytes > kScratchBytes) return MCR_ERR_SCRATCH;

  unsigned char *base = nullptr;
  if ((rc = scratch_address(&base))) return rc;
  unsigned long long *work = reinterpret_cast<unsigned long long *>(base + kOffWork);
  DevStats *stats = reinterpret_cast<DevStats *>(base + kOffStats);
  unsigned *flags = reinterpret_cast<unsigned *>(base + kOffFlags);
  unsigned *latched = reinterpret_cast<unsigned *>(base + kOffLatched);
  float4 *mu = reinterpret_cast<float4 *>(base + kSmall);
  unsigned long long *tally = reinterpret_cast<unsigned long long *>(base + kSmall + mu_bytes);

  cudaStream_t s = (cudaStream_t)stream;
  // the array keeps the previous call's contents: clear the counters and the tally, and move the
  // previous call's error bits into the latched word (read by mc_check)
  if (cudaMemsetAsync(base, 0, kOffFlags, s) != cudaSuccess) return MCR_ERR_CUDA;
  k_latch_flags<<<1, 1, 0, s>>>(flags, latched);
  if (cudaGetLastError() != cudaSuccess) return MCR_ERR_CUDA;
  if (cudaMemsetAsync(tally, 0, tally_bytes, s) != cudaSuccess) return MCR_ERR_CUDA;
  if (launch_pack_medium(med->mua, med->mus, mu, npix, flags, s) != cudaSuccess) return MCR_ERR_CUDA;

  // a transport launch with a one-problem table (the table lives in kernel parameter space)
  TransportParams p;
  memset(&p, 0, sizeof(p));
  p.n_problems = 1;
  p.K = run->K;
  p.C = C;
  p.Cpad = Cpad;
  p.row_stride = transport_row_stride(C);
  p.max_scatter = run->max_scatter;
  p.max_events = run->max_events;
  p.w_threshold = run->w_threshold;
  p.rr_p = run->roulette_p;
  p.rr_inv_p = 1.f / run->roulette_p;
  p.total_packets = run->n_packets;
  p.work = work;
  p.stats = stats;
  p.flags = flags;
  ProblemDesc &d = p.prob[0];
  d.mu = mu;
  d.tally = tally + tally_row_offset(C);  // dense harmonic rows start 15 words into their slot
  d.first_packet = run->first_packet;
  d.end = run->n_packets;
  d.nx = med->nx;
  d.nz = med->nz;
  d.dx = med->dx;
  d.hg_c = (1.f - med->g) / (1.f + med->g);
  const int qexp = tally_exponent(med->dx, run->w_threshold, run->roulette_p);
  d.qscale = ldexpf(1.f, qexp);
  d.kind = src->kind;
  d.x0 = src->x0;
  d.z0 = src->z0;
  d.x1 = src->x1;
  d.z1 = src->z1;
  d.dir_x = dirx;
  d.dir_z = dirz;
  set_angular(d, *src);
  d.key0 = (unsigned)run->seed;
  d.key1 = (unsigned)(run->seed >> 32) ^ run->stream_id;
  if (run->n_packets && launch_transport(p, TransportLaunch{0, 0, 0, 0}, s) != cudaSuccess) return MCR_ERR_CUDA;
  const double area = (double)med->dx * (double)med->dx;
  const double fixed_scale = run->n_packets ? (double)src->power / ((double)run->n_packets * area) : 0.0;
  if (launch_finalize(tally + tally_row_offset(C), nullptr, npix, C, Cpad, ldexp(1.0, -qexp), fixed_scale, false, nullptr, nullptr,
                      (double)(run->n_packets ? run->n_packets : 1), false, run->accumulate != 0, coeff, flags,
                      s) != cudaSuccess)
    return MCR_ERR_CUDA;
  return MCR_OK;
}

}  // extern "C"

namespace mcr {

int noalloc_take_flags(cudaStream_t s) {
  unsigned char *base = nullptr;
  if (scratch_address(&base, false) != MCR_OK || !base) return MCR_OK;
  unsigned w[2] = {0u, 0u};  // the last call's bits and the latched bits of the earlier calls
  if (cudaMemcpyAsync(w, base + kOffFlags, sizeof(w), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaStreamSynchronize(s) != cudaSuccess)
    return MCR_ERR_CUDA;
  if ((w[0] | w[1]) && (cudaMemsetAsync(base + kOffFlags, 0, sizeof(w), s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
    return MCR_ERR_CUDA;
  return status_from_flags(w[0] | w[1]);
}

}  // namespace mcr
