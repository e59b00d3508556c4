// mcr_api.cu -- the C ABI of libmcr (declared in include/mcr.h): argument checks, the per-device
// workspace, and the launch sequences of mc_forward / mc_adjoint / mc_h_eps /
// mc_adjoint_source / mc_gradient.
#include <math.h>
#include <string.h>

#include <mutex>

#include "mcr_internal.h"

using namespace mcr;

namespace {

constexpr int kMaxDevices = 64;
Workspace g_ws[kMaxDevices];
std::mutex g_mu;

#define MCR_TRY_CUDA(expr)                  \
  do {                                      \
    cudaError_t e_ = (expr);                \
    if (e_ != cudaSuccess) return MCR_ERR_CUDA; \
  } while (0)

int grow(void **ptr, size_t *cap, size_t need) {
  if (*cap >= need && *ptr) return MCR_OK;
  if (*ptr) {
    cudaFree(*ptr);
    *ptr = nullptr;
    *cap = 0;
  }
  if (cudaMalloc(ptr, need) != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return MCR_ERR_NOMEM;
  }
  *cap = need;
  return MCR_OK;
}

// Workspace of the current device, grown to hold a problem of npix pixels and C channels.
int workspace(int64_t npix, int C, bool chunked, bool volumetric, Workspace **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCR_ERR_CUDA;
  Workspace &w = g_ws[dev];
  w.device = dev;
  const int Cpad = (C + 3) & ~3;
  int rc;
  if (!w.small) {
    if (cudaMalloc(&w.small, kSmallBytes) != cudaSuccess) {
      w.small = nullptr;
      return MCR_ERR_NOMEM;
    }
    if (cudaMemset(w.small, 0, kSmallBytes) != cudaSuccess) return MCR_ERR_CUDA;
    for (int k = 0; k < 2; ++k)
      if (cudaEventCreate(&w.ev_start[k]) != cudaSuccess || cudaEventCreate(&w.ev_stop[k]) != cudaSuccess)
        return MCR_ERR_CUDA;
  }
  if ((rc = grow((void **)&w.tally, &w.tally_bytes, (size_t)npix * Cpad * 8))) return rc;
  if ((rc = grow((void **)&w.mu, &w.mu_bytes, (size_t)npix * sizeof(float4)))) return rc;
  if ((rc = grow((void **)&w.partials, &w.partials_bytes, (size_t)4096 * sizeof(double)))) return rc;
  if (chunked && (rc = grow((void **)&w.acc, &w.acc_bytes, (size_t)npix * C * sizeof(double)))) return rc;
  if (volumetric) {
    if ((rc = grow((void **)&w.cdf, &w.cdf_bytes, (size_t)npix * 8))) return rc;
    if ((rc = grow((void **)&w.block_sums, &w.block_sums_bytes, (size_t)((npix + 255) / 256) * 8))) return rc;
  }
  *out = &w;
  return MCR_OK;
}

bool finite_f(float v) { return isfinite(v) != 0; }

int check_medium(const mcr_medium *m) {
  if (!m || !m->mua || !m->mus) return MCR_ERR_ARG;
  if (m->nx <= 0 || m->nz <= 0 || (int64_t)m->nx * m->nz > (int64_t)1 << 30) return MCR_ERR_ARG;
  if (!(m->dx > 0.f) || !finite_f(m->dx)) return MCR_ERR_ARG;
  if (!(m->g > -1.f && m->g < 1.f)) return MCR_ERR_ARG;
  return MCR_OK;
}

int check_run(const mcr_run *r) {
  if (!r) return MCR_ERR_ARG;
  if (r->K < 0 || r->K > MCR_MAX_K) return MCR_ERR_ARG;
  if (!(r->roulette_p > 0.f && r->roulette_p <= 1.f)) return MCR_ERR_ARG;
  if (!(r->w_threshold >= 0.f) || !finite_f(r->w_threshold)) return MCR_ERR_ARG;
  if (r->first_packet + r->n_packets < r->first_packet) return MCR_ERR_ARG;  // id overflow
  return MCR_OK;
}

void fill_stats(const DevStats &d, mcr_stats *s) {
  s->launched = d.launched;
  s->flights = d.flights;
  s->collisions = d.collisions;
  s->segments = d.segments;
  s->escapes = d.escapes;
  s->rr_kill = d.rr_kill;
  s->rr_survive = d.rr_survive;
  s->scatter_limit = d.scatter_limit;
  s->event_limit = d.event_limit;
  s->launched_w = d.launched_w;
  s->escaped_w = d.escaped_w;
  s->rr_net_w = d.rr_net_w;
  s->killed_w = d.killed_w;
  s->absorbed_w = d.launched_w + d.rr_net_w - d.escaped_w - d.killed_w;
}

// Reads and clears the latched flags (synchronises the stream).
int take_flags(Workspace *w, cudaStream_t s) {
  unsigned flags = 0;
  MCR_TRY_CUDA(cudaMemcpyAsync(&flags, w->flags(), sizeof(unsigned), cudaMemcpyDeviceToHost, s));
  MCR_TRY_CUDA(cudaStreamSynchronize(s));
  if (flags) MCR_TRY_CUDA(cudaMemsetAsync(w->flags(), 0, sizeof(unsigned), s));
  MCR_TRY_CUDA(cudaStreamSynchronize(s));
  if (flags & kFlagMedium) return MCR_ERR_MEDIUM;
  if (flags & kFlagOverflow) return MCR_ERR_TALLY_OVERFLOW;
  if (flags & kFlagEventLimit) return MCR_ERR_EVENT_LIMIT;
  return MCR_OK;
}

// The shared body of mc_forward and mc_adjoint.
int run_mc(const mcr_medium *med, const mcr_source *src, const float *qstar, const mcr_run *run, float *coeff,
           mcr_stats *stats, cudaStream_t s) {
  int rc;
  if ((rc = check_medium(med)) || (rc = check_run(run))) return rc;
  if (!coeff) return MCR_ERR_ARG;
  const bool volumetric = qstar != nullptr;
  float dirx = 0.f, dirz = 1.f;
  if (!volumetric) {
    if (!src || src->kind < MCR_PENCIL || src->kind > MCR_ISO_POINT) return MCR_ERR_ARG;
    if (!finite_f(src->x0) || !finite_f(src->z0) || !finite_f(src->x1) || !finite_f(src->z1) ||
        !finite_f(src->power))
      return MCR_ERR_ARG;
    if (src->kind != MCR_ISO_POINT) {
      const double nrm = sqrt((double)src->dir_x * src->dir_x + (double)src->dir_z * src->dir_z);
      if (!(nrm > 0.0) || !isfinite(nrm)) return MCR_ERR_ARG;
      dirx = (float)(src->dir_x / nrm);
      dirz = (float)(src->dir_z / nrm);
    }
  }
  const int64_t npix = (int64_t)med->nx * med->nz;
  const int C = 2 * run->K + 1, Cpad = (C + 3) & ~3;
  const bool chunked = run->n_packets > kChunkPackets;
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace *w = nullptr;
  if ((rc = workspace(npix, C, chunked, volumetric, &w))) return rc;

  MCR_TRY_CUDA(launch_pack_medium(med->mua, med->mus, w->mu, npix, w->flags(), s));
  const int slot = volumetric ? 1 : 0;
  MCR_TRY_CUDA(cudaMemsetAsync(w->stats(slot), 0, sizeof(DevStats), s));
  if (volumetric)
    MCR_TRY_CUDA(launch_source_cdf(qstar, npix, w->cdf, w->block_sums, w->block_sums_bytes / 8, w->qmax_bits(), s));
  if (chunked) MCR_TRY_CUDA(cudaMemsetAsync(w->acc, 0, (size_t)npix * C * sizeof(double), s));

  TransportParams p{};
  p.nx = med->nx;
  p.nz = med->nz;
  p.dx = med->dx;
  p.hg_c = (1.f - med->g) / (1.f + med->g);
  p.mu = w->mu;
  p.kind = volumetric ? kVolume : src->kind;
  if (!volumetric) {
    p.x0 = src->x0;
    p.z0 = src->z0;
    p.x1 = src->x1;
    p.z1 = src->z1;
  }
  p.dir_x = dirx;
  p.dir_z = dirz;
  p.cdf = volumetric ? w->cdf : nullptr;
  p.q = qstar;
  p.K = run->K;
  p.C = C;
  p.Cpad = Cpad;
  p.row_stride = Cpad + 2;  // = 2 mod 4 words: conflict-free 8-byte row stores
  const int qexp = tally_exponent(med->dx, run->w_threshold, run->roulette_p);
  p.qscale = ldexpf(1.f, qexp);
  const double quantum = ldexp(1.0, -qexp);
  p.key0 = (unsigned)run->seed;
  p.key1 = (unsigned)(run->seed >> 32) ^ run->stream_id;
  p.max_scatter = run->max_scatter;
  p.max_events = run->max_events;
  p.w_threshold = run->w_threshold;
  p.rr_p = run->roulette_p;
  p.rr_inv_p = 1.f / run->roulette_p;
  p.tally = w->tally;
  p.work = w->work();
  p.stats = w->stats(slot);
  p.flags = w->flags();

  // packets in chunks of at most kChunkPackets; n = 0 runs no transport and gives zeros
  const uint64_t n = run->n_packets;
  uint64_t done = 0;
  MCR_TRY_CUDA(cudaEventRecord(w->ev_start[slot], s));
  do {
    const uint64_t this_n = n - done < kChunkPackets ? n - done : kChunkPackets;
    MCR_TRY_CUDA(cudaMemsetAsync(w->tally, 0, (size_t)npix * Cpad * 8, s));
    MCR_TRY_CUDA(cudaMemsetAsync(w->work(), 0, 8, s));
    p.first_packet = run->first_packet + done;
    p.n_packets = this_n;
    if (this_n) MCR_TRY_CUDA(launch_transport(p, s));
    if (chunked) MCR_TRY_CUDA(launch_accumulate(w->tally, npix, C, Cpad, quantum, w->acc, s));
    done += this_n;
  } while (done < n);
  MCR_TRY_CUDA(cudaEventRecord(w->ev_stop[slot], s));
  w->ran[slot] = true;
  const double area = (double)med->dx * (double)med->dx;
  const double fixed_scale = (!volumetric && n) ? (double)src->power / ((double)n * area) : 0.0;
  MCR_TRY_CUDA(launch_finalize(w->tally, chunked ? w->acc : nullptr, npix, C, Cpad, chunked ? 1.0 : quantum, fixed_scale,
                               volumetric && n > 0, w->qmax_bits(), volumetric ? w->cdf + (npix - 1) : nullptr,
                               (double)(n ? n : 1), volumetric, coeff, w->flags(), s));
  if (stats) {
    DevStats d;
    MCR_TRY_CUDA(cudaMemcpyAsync(&d, w->stats(slot), sizeof(DevStats), cudaMemcpyDeviceToHost, s));
    MCR_TRY_CUDA(cudaStreamSynchronize(s));
    fill_stats(d, stats);
    rc = take_flags(w, s);
    if (rc == MCR_OK && d.event_limit) rc = MCR_ERR_EVENT_LIMIT;
    return rc;
  }
  return MCR_OK;
}

}  // namespace

extern "C" {

int mc_forward(const mcr_medium *med, const mcr_source *src, const mcr_run *run, float *coeff, mcr_stats *stats,
               void *stream) {
  if (!src) return MCR_ERR_ARG;
  return run_mc(med, src, nullptr, run, coeff, stats, (cudaStream_t)stream);
}

int mc_adjoint(const mcr_medium *med, const float *qstar, const mcr_run *run, float *coeff_adj, mcr_stats *stats,
               void *stream) {
  if (!qstar) return MCR_ERR_ARG;
  return run_mc(med, nullptr, qstar, run, coeff_adj, stats, (cudaStream_t)stream);
}

int mc_h_eps(const mcr_medium *med, const float *coeff, const float *Hmeas, float *H, float *dL_dH, double *eps,
             void *stream) {
  int rc;
  if ((rc = check_medium(med))) return rc;
  if (!coeff || (!Hmeas && (dL_dH || eps))) return MCR_ERR_ARG;
  const int64_t npix = (int64_t)med->nx * med->nz;
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace *w = nullptr;
  if ((rc = workspace(npix, 1, false, false, &w))) return rc;
  MCR_TRY_CUDA(launch_h_eps(med->mua, coeff, Hmeas, npix, (double)med->dx * (double)med->dx, H, dL_dH, w->partials,
                            w->partials_bytes / sizeof(double), eps, (cudaStream_t)stream));
  return MCR_OK;
}

int mc_adjoint_source(const mcr_medium *med, const float *dL_dH, float *qstar, void *stream) {
  int rc;
  if ((rc = check_medium(med))) return rc;
  if (!dL_dH || !qstar) return MCR_ERR_ARG;
  MCR_TRY_CUDA(launch_adjoint_source(med->mua, dL_dH, (int64_t)med->nx * med->nz, (double)med->dx * (double)med->dx, qstar,
                                     (cudaStream_t)stream));
  return MCR_OK;
}

int mc_gradient(const mcr_medium *med, int32_t K, const float *coeff, const float *coeff_adj, const float *dL_dH,
                double *d_mua, double *d_mus, void *stream) {
  int rc;
  if ((rc = check_medium(med))) return rc;
  if (K < 0 || K > MCR_MAX_K || !coeff || !coeff_adj || !dL_dH || !d_mua) return MCR_ERR_ARG;
  MCR_TRY_CUDA(launch_gradient(coeff, coeff_adj, dL_dH, (int64_t)med->nx * med->nz, K, (double)med->g,
                               (double)med->dx * (double)med->dx, d_mua, d_mus, (cudaStream_t)stream));
  return MCR_OK;
}

int mc_check(void *stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace &w = g_ws[dev];
  if (!w.small) {
    MCR_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
    return MCR_OK;
  }
  return take_flags(&w, (cudaStream_t)stream);
}

int mc_last_run_info(int32_t which, mcr_stats *stats, float *transport_ms) {
  int dev = 0;
  if (which < 0 || which > 1) return MCR_ERR_ARG;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace &w = g_ws[dev];
  if (!w.small || !w.ran[which]) return MCR_ERR_ARG;
  MCR_TRY_CUDA(cudaEventSynchronize(w.ev_stop[which]));
  if (transport_ms) MCR_TRY_CUDA(cudaEventElapsedTime(transport_ms, w.ev_start[which], w.ev_stop[which]));
  if (stats) {
    DevStats d;
    MCR_TRY_CUDA(cudaMemcpy(&d, w.stats(which), sizeof(DevStats), cudaMemcpyDeviceToHost));
    fill_stats(d, stats);
  }
  return MCR_OK;
}

int mc_release_workspace(void) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCR_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_mu);
  MCR_TRY_CUDA(cudaDeviceSynchronize());
  Workspace &w = g_ws[dev];
  void *ptrs[] = {w.tally, w.acc, w.mu, w.cdf, w.block_sums, w.partials, w.small};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int k = 0; k < 2; ++k) {
    if (w.ev_start[k]) cudaEventDestroy(w.ev_start[k]);
    if (w.ev_stop[k]) cudaEventDestroy(w.ev_stop[k]);
  }
  w = Workspace{};
  return MCR_OK;
}

const char *mc_status_string(int status) {
  switch (status) {
    case MCR_OK: return "ok";
    case MCR_ERR_ARG: return "invalid argument";
    case MCR_ERR_CUDA: return "CUDA runtime error";
    case MCR_ERR_NOMEM: return "device memory allocation failed";
    case MCR_ERR_EVENT_LIMIT: return "a packet reached max_events flights and was ended";
    case MCR_ERR_TALLY_OVERFLOW: return "fixed-point tally near overflow";
    case MCR_ERR_MEDIUM: return "medium holds a negative or non-finite coefficient";
    case MCR_ERR_SCRATCH: return "problem exceeds the fixed 16 MiB scratch of mc_forward_noalloc";
    default: return "unknown status";
  }
}

const char *mc_version(void) { return "mcr 1.0 sm_103a"; }

}  // extern "C"

namespace mcr {

// q such that every deposit |t h| 2^q stays below 2^30 (< 2^31 with margin for |h| rounding):
// t <= W l with l <= dx sqrt 2 inside one pixel, and |W| <= max(1, w_threshold / p) because the
// weight only decreases except for roulette survivors, which are below the threshold before.
int tally_exponent(float dx, float w_threshold, float roulette_p) {
  const double wmax = fmax(1.0, (double)w_threshold / (double)roulette_p);
  const double tmax = wmax * (double)dx * 1.41421356237309515 * 1.001;
  int q = (int)floor(30.0 - log2(tmax));
  if (q > 60) q = 60;
  if (q < -60) q = -60;
  return q;
}

}  // namespace mcr
