// mcr_api.cu -- the C ABI of libmcr (declared in include/mcr.h): argument checks, the per-device
// workspace, and the launch sequences of mc_forward / mc_adjoint / mc_run_batch / mc_h_eps /
// mc_eps / mc_adjoint_source / mc_gradient.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "mcr_internal.h"

using namespace mcr;

namespace {

constexpr int kMaxDevices = 64;
Workspace g_ws[kMaxDevices];
std::mutex g_mu;

#define MCR_TRY_CUDA(expr)                      \
  do {                                          \
    cudaError_t e_ = (expr);                    \
    if (e_ != cudaSuccess) return MCR_ERR_CUDA; \
  } while (0)

int grow(void **ptr, size_t *cap, size_t need) {
  if (need == 0) need = 256;
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

// Sizes the workspace of one launch needs (all problems together).
struct Need {
  size_t tally = 0, acc = 0, mu = 0, cdf = 0, block_sums = 0, order = 0, order_hist = 0;
  size_t records = 0, rec_hist = 0;  // sorted-record deposit (records: each of the two buffers)
};

// Workspace of the current device, grown to `need`.
int workspace(const Need &need, Workspace **out) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCR_ERR_CUDA;
  Workspace &w = g_ws[dev];
  w.device = dev;
  int rc;
  if (!w.small) {
    if (cudaMalloc(&w.small, kSmallBytes) != cudaSuccess) {
      w.small = nullptr;
      return MCR_ERR_NOMEM;
    }
    if (cudaMemset(w.small, 0, kSmallBytes) != cudaSuccess) return MCR_ERR_CUDA;
    for (int k = 0; k < 3; ++k)
      if (cudaEventCreate(&w.ev_start[k]) != cudaSuccess || cudaEventCreate(&w.ev_stop[k]) != cudaSuccess)
        return MCR_ERR_CUDA;
  }
  if ((rc = grow((void **)&w.partials, &w.partials_bytes, (size_t)4096 * sizeof(double)))) return rc;
  if (need.tally && (rc = grow((void **)&w.tally, &w.tally_bytes, need.tally))) return rc;
  if (need.mu && (rc = grow((void **)&w.mu, &w.mu_bytes, need.mu))) return rc;
  if (need.acc && (rc = grow((void **)&w.acc, &w.acc_bytes, need.acc))) return rc;
  if (need.cdf && (rc = grow((void **)&w.cdf, &w.cdf_bytes, need.cdf))) return rc;
  if (need.block_sums && (rc = grow((void **)&w.block_sums, &w.block_sums_bytes, need.block_sums))) return rc;
  if (need.order && (rc = grow((void **)&w.order, &w.order_bytes, need.order))) return rc;
  if (need.order_hist && (rc = grow((void **)&w.order_hist, &w.order_hist_bytes, need.order_hist))) return rc;
  if (need.records) {
    if ((rc = grow((void **)&w.records, &w.records_bytes, need.records))) return rc;
    if ((rc = grow((void **)&w.sorted, &w.sorted_bytes, need.records))) return rc;
    if ((rc = grow((void **)&w.rec_hdr, &w.rec_hdr_bytes, sizeof(RecordHeader)))) return rc;
    if ((rc = grow((void **)&w.rec_hist, &w.rec_hist_bytes, need.rec_hist))) return rc;
  }
  *out = &w;
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
  return status_from_flags(flags);
}

// One problem as the host sees it.
struct HostProblem {
  const mcr_medium *med;
  const mcr_source *src;  // forward source, or null
  const float *qstar;     // volumetric (adjoint) source, or null
  uint64_t n_packets, first_packet, seed;
  uint32_t stream_id;
  float *coeff;
  float dirx, dirz;
};

// Enqueues the whole sequence for `probs` on stream s: pack media, source CDFs, zero tallies,
// transport launch(es), finalize per problem.  `slot` selects the run counters / events.
// With raw_out (one problem of at most kChunkPackets packets) the run's fixed-point sums are
// exported channel-major instead of being finalised.
int enqueue(const std::vector<HostProblem> &probs, const mcr_run *common, const TransportLaunch &cfg, int slot,
            mcr_stats *stats, cudaStream_t s, long long *raw_out = nullptr) {
  const int np = (int)probs.size();
  const int C = common->time_bins ? (int)common->time_bins : common->sectors ? (int)common->sectors : 2 * common->K + 1;
  const int Cpad = tally_row_words(C);
  // words from a pixel's slot to its row (dense harmonic rows; folded into tally_off)
  const int roff = (common->time_bins || common->sectors) ? 0 : tally_row_offset(C);
  // a single problem may exceed one launch's packet budget (chunks + FP64 flush); a batch may not
  const bool chunked = np == 1 && probs[0].n_packets > kChunkPackets;
  Need need;
  std::vector<size_t> mu_off(np), tally_off(np), cdf_off(np), bs_off(np);
  for (int i = 0; i < np; ++i) {
    const int64_t npix = (int64_t)probs[i].med->nx * probs[i].med->nz;
    mu_off[i] = need.mu / sizeof(float4);
    need.mu += ((size_t)npix * sizeof(float4) + 255) & ~size_t(255);
    tally_off[i] = need.tally / 8 + roff;
    need.tally += ((size_t)npix * Cpad * 8 + 255) & ~size_t(255);
    if (probs[i].qstar) {
      cdf_off[i] = need.cdf / 8;
      need.cdf += ((size_t)npix * 8 + 255) & ~size_t(255);
      bs_off[i] = need.block_sums / 8;
      need.block_sums += (size_t)((npix + 255) / 256) * 8;
    }
    if (chunked) need.acc = (size_t)npix * C * sizeof(double);
  }
  // launch order: by default once the tallies no longer fit in L2, for the kinds it orders
  bool ordered = false;
  unsigned total_bins = 0;
  {
    bool orderable = false;
    uint64_t packets = 0;
    for (int i = 0; i < np; ++i) {
      orderable |= probs[i].qstar != nullptr || (probs[i].src && probs[i].src->kind == MCR_LINE);
      packets += chunked ? kChunkPackets : probs[i].n_packets;
      ProblemDesc d{};
      d.kind = probs[i].qstar ? kVolume : probs[i].src->kind;
      d.nx = probs[i].med->nx;
      d.nz = probs[i].med->nz;
      total_bins += order_bins(d);
    }
    ordered = orderable && packets > 0 && packets <= 0xFFFFFFFFull && !common->sectors && !common->time_bins &&
              (cfg.launch_order == 2 || (cfg.launch_order == 0 && (double)need.tally > kOrderTallyBytes));
    if (ordered) {
      need.order = (size_t)packets * sizeof(unsigned);
      need.order_hist = (size_t)total_bins * sizeof(unsigned);
    }
  }
  // sorted-record deposit: one harmonic problem whose tally does not fit in L2 (not while a graph
  // is being captured: the chunk sizes are read back from the device)
  cudaStreamCaptureStatus cap0 = cudaStreamCaptureStatusNone;
  MCR_TRY_CUDA(cudaStreamIsCapturing(s, &cap0));
  bool rec_mode = np == 1 && !common->sectors && !common->time_bins && cap0 == cudaStreamCaptureStatusNone &&
                        probs[0].n_packets > 0 &&
                        (cfg.deposit == 2 || (cfg.deposit == 0 && (double)need.tally > kRecordTallyBytes));
  const unsigned long long rec_cap = cfg.record_capacity > 0 ? (unsigned long long)cfg.record_capacity : kRecordCapacity;
  if (rec_mode) {
    const int64_t npix = (int64_t)probs[0].med->nx * probs[0].med->nz;
    need.records = (size_t)rec_cap * sizeof(float4);
    need.rec_hist = ((size_t)npix * 2 + (npix + 255) / 256 + 1) * sizeof(unsigned);
  }
  Workspace *w = nullptr;
  int rc = workspace(need, &w);
  if (rc == MCR_ERR_NOMEM && rec_mode) {  // no room for the record buffers: deposit directly
    rec_mode = false;
    need.records = need.rec_hist = 0;
    rc = workspace(need, &w);
  }
  if (rc) return rc;

  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  MCR_TRY_CUDA(cudaStreamIsCapturing(s, &cap));
  const bool timed = cap == cudaStreamCaptureStatusNone;

  MCR_TRY_CUDA(cudaMemsetAsync(w->stats(slot), 0, sizeof(DevStats), s));
  TransportParams p;
  memset(&p, 0, sizeof(p));
  p.n_problems = np;
  p.K = common->K;
  p.C = C;
  p.Cpad = Cpad;
  // no harmonic rows for the sector and time tallies
  p.row_stride = (common->sectors || common->time_bins) ? 1 : transport_row_stride(C);
  p.sectors = (int)common->sectors;
  p.sector_scale = (float)(common->sectors / (2.0 * 3.14159265358979323846));
  p.time_bins = (int)common->time_bins;
  p.time_bin_mm = common->time_bin_mm;
  p.inv_time_bin = common->time_bins ? 1.f / common->time_bin_mm : 0.f;
  p.max_scatter = common->max_scatter;
  p.max_events = common->max_events;
  p.w_threshold = common->w_threshold;
  p.rr_p = common->roulette_p;
  p.rr_inv_p = 1.f / common->roulette_p;
  p.work = w->work();
  p.stats = w->stats(slot);
  p.flags = w->flags();
  std::vector<int> qexp(np);
  uint64_t end = 0;
  unsigned bin_base = 0;
  for (int i = 0; i < np; ++i) {
    const HostProblem &h = probs[i];
    const int64_t npix = (int64_t)h.med->nx * h.med->nz;
    float4 *mu = w->mu + mu_off[i];
    MCR_TRY_CUDA(launch_pack_medium(h.med->mua, h.med->mus, mu, npix, w->flags(), s));
    ProblemDesc &d = p.prob[i];
    d.mu = mu;
    d.tally = w->tally + tally_off[i];
    d.nx = h.med->nx;
    d.nz = h.med->nz;
    d.dx = h.med->dx;
    d.hg_c = (1.f - h.med->g) / (1.f + h.med->g);
    qexp[i] = tally_exponent(h.med->dx, common->w_threshold, common->roulette_p);
    d.qscale = ldexpf(1.f, qexp[i]);
    d.key0 = (unsigned)h.seed;
    d.key1 = (unsigned)(h.seed >> 32) ^ h.stream_id;
    d.first_packet = h.first_packet;
    if (h.qstar) {
      d.kind = kVolume;
      d.cdf = w->cdf + cdf_off[i];
      d.q = h.qstar;
      MCR_TRY_CUDA(launch_source_cdf(h.qstar, npix, w->cdf + cdf_off[i], w->block_sums + bs_off[i],
                                     (size_t)((npix + 255) / 256), w->qmax_bits(i), s));
    } else {
      d.kind = h.src->kind;
      d.x0 = h.src->x0;
      d.z0 = h.src->z0;
      d.x1 = h.src->x1;
      d.z1 = h.src->z1;
      d.dir_x = h.dirx;
      d.dir_z = h.dirz;
      set_angular(d, *h.src);
    }
    end += chunked ? 0 : h.n_packets;
    d.end = end;
    d.bin_base = bin_base;
    bin_base += order_bins(d);
  }
  p.order = ordered ? w->order : nullptr;
  MCR_TRY_CUDA(cudaMemsetAsync(w->tally, 0, need.tally, s));
  if (chunked) MCR_TRY_CUDA(cudaMemsetAsync(w->acc, 0, need.acc, s));
  if (timed) MCR_TRY_CUDA(cudaEventRecord(w->ev_start[slot], s));
  // one problem's packets [first, first + count) added into the tally: directly ...
  auto direct = [&](uint64_t first, uint64_t count) -> int {
    MCR_TRY_CUDA(cudaMemsetAsync(w->work(), 0, 8, s));
    p.prob[0].first_packet = first;
    p.prob[0].end = count;
    p.total_packets = count;
    if (ordered) MCR_TRY_CUDA(launch_order(p, total_bins, w->order_hist, w->order, s));
    MCR_TRY_CUDA(launch_transport(p, cfg, s));
    return MCR_OK;
  };
  // ... or by sorted records, in chunks sized so that their records fit the buffer (from the most
  // records per packet seen so far); a chunk whose records overflow runs again directly
  double rec_per_packet = 0.0;
  auto by_records = [&](uint64_t first, uint64_t count) -> int {
    const int64_t npix = (int64_t)probs[0].med->nx * probs[0].med->nz;
    unsigned *hist = w->rec_hist, *cursor = w->rec_hist + npix, *bsums = w->rec_hist + 2 * npix;
    for (uint64_t done = 0; done < count;) {
      // first chunk: room for 2048 records per packet; then from the most records per packet seen
      uint64_t chunk = rec_per_packet > 0.0 ? (uint64_t)((double)rec_cap / (1.25 * rec_per_packet)) : rec_cap / 2048;
      chunk = chunk < 1 ? 1 : (chunk > kChunkPackets ? kChunkPackets : chunk);
      const uint64_t this_n = count - done < chunk ? count - done : chunk;
      TransportParams q = p;
      q.prob[0].first_packet = first + done;
      q.prob[0].end = this_n;
      q.total_packets = this_n;
      q.order = nullptr;
      q.records = w->records;
      q.rec_count = &w->rec_hdr->count;
      q.rec_overflow = &w->rec_hdr->overflow;
      q.rec_capacity = rec_cap;
      q.rec_hist = hist;
      q.stats = &w->rec_hdr->stats;
      MCR_TRY_CUDA(cudaMemsetAsync(w->work(), 0, 8, s));
      MCR_TRY_CUDA(cudaMemsetAsync(w->rec_hdr, 0, sizeof(RecordHeader), s));
      MCR_TRY_CUDA(cudaMemsetAsync(hist, 0, (size_t)npix * sizeof(unsigned), s));
      MCR_TRY_CUDA(launch_transport_records(q, cfg, s));
      RecordHeader hdr;
      MCR_TRY_CUDA(cudaMemcpyAsync(&hdr, w->rec_hdr, sizeof(hdr), cudaMemcpyDeviceToHost, s));
      MCR_TRY_CUDA(cudaStreamSynchronize(s));
      if (hdr.overflow) {
        int rc2 = direct(first + done, this_n);
        if (rc2) return rc2;
      } else {
        // slots reserved past the capacity (a warp's last block may straddle it) were never written
        const unsigned long long n_slots = hdr.count < rec_cap ? hdr.count : rec_cap;
        MCR_TRY_CUDA(launch_sort_and_deposit(w->records, n_slots, hist, cursor, bsums, (int)npix, w->sorted,
                                             common->K, Cpad, w->tally + tally_off[0], w->flags(), s));
        MCR_TRY_CUDA(launch_add_stats(p.stats, &w->rec_hdr->stats, s));
      }
      const double r = (double)hdr.count / (double)this_n;
      if (r > rec_per_packet) rec_per_packet = r;
      done += this_n;
    }
    return MCR_OK;
  };
  auto run_range = [&](uint64_t first, uint64_t count) -> int {
    return rec_mode ? by_records(first, count) : direct(first, count);
  };
  if (!chunked) {
    p.total_packets = end;
    if (rec_mode) {
      if ((rc = run_range(probs[0].first_packet, probs[0].n_packets))) return rc;
    } else {
      MCR_TRY_CUDA(cudaMemsetAsync(w->work(), 0, 8, s));
      if (end && ordered) MCR_TRY_CUDA(launch_order(p, total_bins, w->order_hist, w->order, s));
      if (end) MCR_TRY_CUDA(launch_transport(p, cfg, s));
    }
  } else {
    const HostProblem &h = probs[0];
    const int64_t npix = (int64_t)h.med->nx * h.med->nz;
    for (uint64_t done = 0; done < h.n_packets;) {
      const uint64_t this_n = h.n_packets - done < kChunkPackets ? h.n_packets - done : kChunkPackets;
      if (done) MCR_TRY_CUDA(cudaMemsetAsync(w->tally, 0, need.tally, s));
      if ((rc = run_range(h.first_packet + done, this_n))) return rc;
      MCR_TRY_CUDA(launch_accumulate(w->tally + tally_off[0], npix, C, Cpad, ldexp(1.0, -qexp[0]), w->acc, s));
      done += this_n;
    }
  }
  if (timed) {
    MCR_TRY_CUDA(cudaEventRecord(w->ev_stop[slot], s));
    w->ran[slot] = true;
  }
  if (raw_out) {
    const int64_t npix = (int64_t)probs[0].med->nx * probs[0].med->nz;
    MCR_TRY_CUDA(launch_export_raw(w->tally + tally_off[0], npix, C, Cpad, common->accumulate != 0, raw_out, s));
  }
  for (int i = 0; i < np && !raw_out; ++i) {
    const HostProblem &h = probs[i];
    const int64_t npix = (int64_t)h.med->nx * h.med->nz;
    const double area = (double)h.med->dx * (double)h.med->dx;
    const bool vol = h.qstar != nullptr;
    const double fixed_scale = (!vol && h.n_packets) ? (double)h.src->power / ((double)h.n_packets * area) : 0.0;
    MCR_TRY_CUDA(launch_finalize(w->tally + tally_off[i], chunked ? w->acc : nullptr, npix, C, Cpad,
                                 chunked ? 1.0 : ldexp(1.0, -qexp[i]), fixed_scale, vol && h.n_packets > 0,
                                 w->qmax_bits(i), vol ? w->cdf + cdf_off[i] + (npix - 1) : nullptr,
                                 (double)(h.n_packets ? h.n_packets : 1), vol, common->accumulate != 0, h.coeff,
                                 w->flags(), s));
  }
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

// The shared body of mc_forward and mc_adjoint (and of their raw forms, raw != NULL).
int run_mc(const mcr_medium *med, const mcr_source *src, const float *qstar, const mcr_run *run, float *coeff,
           mcr_stats *stats, cudaStream_t s, long long *raw = nullptr) {
  int rc;
  if ((rc = check_medium(med)) || (rc = check_run(run))) return rc;
  if (!coeff && !raw) return MCR_ERR_ARG;
  if (qstar && (run->sectors || run->time_bins)) return MCR_ERR_ARG;  // forward-only tallies
  // raw sums: harmonic tallies of one launch (longer runs add ranges with accumulate)
  if (raw && (run->sectors || run->time_bins || run->n_packets > kChunkPackets)) return MCR_ERR_ARG;
  HostProblem h{med, src, qstar, run->n_packets, run->first_packet, run->seed, run->stream_id, coeff, 0.f, 1.f};
  if (!qstar && (rc = check_source(src, &h.dirx, &h.dirz))) return rc;
  std::lock_guard<std::mutex> lock(g_mu);
  return enqueue({h}, run, TransportLaunch{0, 0, 0, 0}, qstar ? 1 : 0, stats, s, raw);
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

int mc_forward_raw(const mcr_medium *med, const mcr_source *src, const mcr_run *run, int64_t *tally,
                   mcr_stats *stats, void *stream) {
  if (!src || !tally) return MCR_ERR_ARG;
  return run_mc(med, src, nullptr, run, nullptr, stats, (cudaStream_t)stream, reinterpret_cast<long long *>(tally));
}

int mc_adjoint_raw(const mcr_medium *med, const float *qstar, const mcr_run *run, int64_t *tally, mcr_stats *stats,
                   void *stream) {
  if (!qstar || !tally) return MCR_ERR_ARG;
  return run_mc(med, nullptr, qstar, run, nullptr, stats, (cudaStream_t)stream, reinterpret_cast<long long *>(tally));
}

int mc_finalize(const mcr_medium *med, const mcr_source *src, const float *qstar, const mcr_run *run,
                const int64_t *tally, float *coeff, void *stream) {
  int rc;
  if ((rc = check_medium(med)) || (rc = check_run(run))) return rc;
  if (!tally || !coeff || run->sectors || run->time_bins || (src == nullptr) == (qstar == nullptr)) return MCR_ERR_ARG;
  float dirx, dirz;
  if (src && (rc = check_source(src, &dirx, &dirz))) return rc;
  const int64_t npix = (int64_t)med->nx * med->nz;
  const int C = 2 * run->K + 1;
  const double area = (double)med->dx * (double)med->dx;
  const double quantum = ldexp(1.0, -tally_exponent(med->dx, run->w_threshold, run->roulette_p));
  const double n = (double)(run->n_packets ? run->n_packets : 1);
  cudaStream_t s = (cudaStream_t)stream;
  std::lock_guard<std::mutex> lock(g_mu);
  Need need;
  if (qstar) {
    need.cdf = ((size_t)npix * 8 + 255) & ~size_t(255);
    need.block_sums = (size_t)((npix + 255) / 256) * 8;
  }
  Workspace *w = nullptr;
  if ((rc = workspace(need, &w))) return rc;
  if (qstar) {  // the source strength S of the adjoint run, from q* as mc_adjoint computes it
    MCR_TRY_CUDA(launch_source_cdf(qstar, npix, w->cdf, w->block_sums, (size_t)((npix + 255) / 256),
                                   w->qmax_bits(0), s));
  }
  const double fixed_scale = (src && run->n_packets) ? (double)src->power / (n * area) : 0.0;
  MCR_TRY_CUDA(launch_finalize_raw(reinterpret_cast<const long long *>(tally), npix, C, quantum, fixed_scale,
                                   qstar != nullptr && run->n_packets > 0, w->qmax_bits(0),
                                   qstar ? w->cdf + (npix - 1) : nullptr, n, qstar != nullptr, run->accumulate != 0,
                                   coeff, w->flags(), s));
  return MCR_OK;
}

int mc_run_batch(const mcr_problem *problems, int32_t n_problems, const mcr_run *common, const mcr_launch *launch,
                 mcr_stats *stats, void *stream) {
  int rc;
  if (!problems || n_problems < 1 || n_problems > MCR_MAX_BATCH) return MCR_ERR_ARG;
  if ((rc = check_run(common))) return rc;
  if (common->sectors || common->time_bins) return MCR_ERR_ARG;  // these tallies run through mc_forward only
  TransportLaunch cfg{0, 0, 0, 0, 0, 0, 0};
  if (launch) {
    if (launch->threads_per_block < 0 || launch->threads_per_block > 256 || launch->threads_per_block % 32 ||
        launch->blocks_per_sm < 0 || launch->merge_collisions < 0 || launch->merge_collisions > 2 ||
        launch->shared_tally < 0 || launch->shared_tally > 2 || launch->launch_order < 0 || launch->launch_order > 2 ||
        launch->deposit < 0 || launch->deposit > 2 || launch->record_capacity < 0)
      return MCR_ERR_ARG;
    cfg = TransportLaunch{launch->threads_per_block, launch->blocks_per_sm, launch->merge_collisions,
                          launch->shared_tally, launch->launch_order, launch->deposit, launch->record_capacity};
  }
  std::vector<HostProblem> probs;
  uint64_t total = 0;
  for (int i = 0; i < n_problems; ++i) {
    const mcr_problem &q = problems[i];
    if ((rc = check_medium(&q.medium))) return rc;
    if (!q.coeff || q.n_packets > kChunkPackets || q.first_packet + q.n_packets < q.first_packet) return MCR_ERR_ARG;
    HostProblem h{&q.medium, q.qstar ? nullptr : &q.source, q.qstar, q.n_packets, q.first_packet, q.seed,
                  q.stream_id, q.coeff, 0.f, 1.f};
    if (!q.qstar && (rc = check_source(&q.source, &h.dirx, &h.dirz))) return rc;
    total += q.n_packets;
    probs.push_back(h);
  }
  (void)total;
  std::lock_guard<std::mutex> lock(g_mu);
  return enqueue(probs, common, cfg, 2, stats, (cudaStream_t)stream);
}

int mc_h_eps(const mcr_medium *med, const float *coeff, const float *Hmeas, float *H, float *dL_dH, double *eps,
             void *stream) {
  int rc;
  if ((rc = check_medium(med))) return rc;
  if (!coeff || (!Hmeas && (dL_dH || eps))) return MCR_ERR_ARG;
  const int64_t npix = (int64_t)med->nx * med->nz;
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace *w = nullptr;
  if ((rc = workspace(Need{}, &w))) return rc;
  MCR_TRY_CUDA(launch_h_eps(med->mua, coeff, Hmeas, npix, (double)med->dx * (double)med->dx, H, dL_dH, w->partials,
                            w->partials_bytes / sizeof(double), eps, (cudaStream_t)stream));
  return MCR_OK;
}

int mc_eps(int64_t npix, double pixel_area, const float *H, const float *Hmeas, float *dL_dH, double *eps,
           void *stream) {
  if (npix <= 0 || !(pixel_area > 0.0) || !isfinite(pixel_area) || !H || !Hmeas || !eps) return MCR_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace *w = nullptr;
  int rc;
  if ((rc = workspace(Need{}, &w))) return rc;
  MCR_TRY_CUDA(launch_h_eps(nullptr, H, Hmeas, npix, pixel_area, nullptr, dL_dH, w->partials,
                            w->partials_bytes / sizeof(double), eps, (cudaStream_t)stream));
  return MCR_OK;
}

int mc_dot(int64_t n, const float *a, const float *b, double *out, void *stream) {
  if (n <= 0 || !a || !b || !out) return MCR_ERR_ARG;
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace *w = nullptr;
  int rc;
  if ((rc = workspace(Need{}, &w))) return rc;
  MCR_TRY_CUDA(launch_dot(a, b, n, w->partials, w->partials_bytes / sizeof(double), out, (cudaStream_t)stream));
  return MCR_OK;
}

int mc_adjoint_source(const mcr_medium *med, const float *dL_dH, float *qstar, void *stream) {
  int rc;
  if ((rc = check_medium(med))) return rc;
  if (!dL_dH || !qstar) return MCR_ERR_ARG;
  MCR_TRY_CUDA(launch_adjoint_source(med->mua, dL_dH, (int64_t)med->nx * med->nz,
                                     (double)med->dx * (double)med->dx, qstar, (cudaStream_t)stream));
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

int mc_gradient_f32(const mcr_medium *med, int32_t K, const float *coeff, const float *coeff_adj, const float *dL_dH,
                    float *d_mua, float *d_mus, void *stream) {
  int rc;
  if ((rc = check_medium(med))) return rc;
  if (K < 0 || K > MCR_MAX_K || !coeff || !coeff_adj || !dL_dH || !d_mua) return MCR_ERR_ARG;
  MCR_TRY_CUDA(launch_gradient_f32(coeff, coeff_adj, dL_dH, (int64_t)med->nx * med->nz, K, (double)med->g,
                                   (double)med->dx * (double)med->dx, d_mua, d_mus, (cudaStream_t)stream));
  return MCR_OK;
}

int mc_check(void *stream) {
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return MCR_ERR_CUDA;
  // the no-allocation entry point latches its errors in its own scratch
  const int rc_noalloc = noalloc_take_flags((cudaStream_t)stream);
  std::lock_guard<std::mutex> lock(g_mu);
  Workspace &w = g_ws[dev];
  int rc = MCR_OK;
  if (!w.small) {
    MCR_TRY_CUDA(cudaStreamSynchronize((cudaStream_t)stream));
  } else {
    rc = take_flags(&w, (cudaStream_t)stream);
  }
  return rc != MCR_OK ? rc : rc_noalloc;
}

int mc_last_run_info(int32_t which, mcr_stats *stats, float *transport_ms) {
  int dev = 0;
  if (which < 0 || which > 2) return MCR_ERR_ARG;
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
  void *ptrs[] = {w.tally, w.acc, w.mu, w.cdf, w.block_sums, w.partials, w.small, w.order, w.order_hist,
                  w.records, w.sorted, w.rec_hdr, w.rec_hist};
  for (void *p : ptrs)
    if (p) cudaFree(p);
  for (int k = 0; k < 3; ++k) {
    if (w.ev_start[k]) cudaEventDestroy(w.ev_start[k]);
    if (w.ev_stop[k]) cudaEventDestroy(w.ev_stop[k]);
  }
  w = Workspace{};
  return release_workspace3(dev);
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
    case MCR_ERR_CHECK: return "checked build: out-of-range index or non-finite weight on the device";
    default: return "unknown status";
  }
}

#ifdef MCR_CHECKED
const char *mc_version(void) { return "mcr 1.1 sm_103a checked"; }
#else
const char *mc_version(void) { return "mcr 1.1 sm_103a"; }
#endif

}  // extern "C"

namespace mcr {

int check_medium(const mcr_medium *m) {
  if (!m || !m->mua || !m->mus) return MCR_ERR_ARG;
  // the deposit key packs (pixel + 1) into 26 bits
  if (m->nx <= 0 || m->nz <= 0 || (int64_t)m->nx * m->nz >= (int64_t)1 << 26) return MCR_ERR_ARG;
  if (!(m->dx > 0.f) || !isfinite(m->dx)) return MCR_ERR_ARG;
  if (!(m->g > -1.f && m->g < 1.f)) return MCR_ERR_ARG;
  return MCR_OK;
}

int check_run(const mcr_run *r) {
  if (!r) return MCR_ERR_ARG;
  if (r->K < 0 || r->K > MCR_MAX_K) return MCR_ERR_ARG;
  if (!(r->roulette_p > 0.f && r->roulette_p <= 1.f)) return MCR_ERR_ARG;
  if (!(r->w_threshold >= 0.f) || !isfinite(r->w_threshold)) return MCR_ERR_ARG;
  if (r->first_packet + r->n_packets < r->first_packet) return MCR_ERR_ARG;  // id overflow
  if (r->accumulate > 1u) return MCR_ERR_ARG;
  if (r->sectors > 1024u) return MCR_ERR_ARG;
  if (r->time_bins > 1024u) return MCR_ERR_ARG;
  if (r->time_bins && (r->sectors || !(r->time_bin_mm > 0.f) || !isfinite(r->time_bin_mm))) return MCR_ERR_ARG;
  return MCR_OK;
}

// Normalised launch direction of a boundary source, or MCR_ERR_ARG.
int check_source(const mcr_source *src, float *dirx, float *dirz) {
  if (!src || src->kind < MCR_PENCIL || src->kind > MCR_ANGULAR_POINT) return MCR_ERR_ARG;
  if (src->kind == MCR_ANGULAR_POINT && !angular_density_ok(*src)) return MCR_ERR_ARG;
  if (!isfinite(src->x0) || !isfinite(src->z0) || !isfinite(src->x1) || !isfinite(src->z1) ||
      !isfinite(src->power))
    return MCR_ERR_ARG;
  *dirx = 0.f;
  *dirz = 1.f;
  if (src->kind == MCR_PENCIL || src->kind == MCR_LINE) {
    const double nrm = sqrt((double)src->dir_x * src->dir_x + (double)src->dir_z * src->dir_z);
    if (!(nrm > 0.0) || !isfinite(nrm)) return MCR_ERR_ARG;
    *dirx = (float)(src->dir_x / nrm);
    *dirz = (float)(src->dir_z / nrm);
  }
  return MCR_OK;
}

int status_from_flags(unsigned flags) {
  if (flags & kFlagChecked) return MCR_ERR_CHECK;
  if (flags & kFlagMedium) return MCR_ERR_MEDIUM;
  if (flags & kFlagOverflow) return MCR_ERR_TALLY_OVERFLOW;
  if (flags & kFlagEventLimit) return MCR_ERR_EVENT_LIMIT;
  return MCR_OK;
}

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

bool angular_density_ok(const mcr_source &src) {
  if (src.n_ang < 0 || src.n_ang > MCR_MAX_ANG) return false;
  for (int n = 0; n < src.n_ang; ++n)
    if (!isfinite(src.ang_c[n]) || !isfinite(src.ang_s[n])) return false;
  for (int i = 0; i < 4096; ++i) {  // 2 pi p(theta) = 1 + sum_n c_n cos n theta + s_n sin n theta
    const double th = 2.0 * 3.14159265358979323846 * i / 4096.0;
    double v = 1.0;
    for (int n = 1; n <= src.n_ang; ++n) v += src.ang_c[n - 1] * cos(n * th) + src.ang_s[n - 1] * sin(n * th);
    if (v < -1e-6) return false;
  }
  return true;
}

}  // namespace mcr
