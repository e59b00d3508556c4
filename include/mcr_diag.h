/*
 * mcr_diag.h -- measurement and test entry points of libmcr.  They are not part of the method's
 * interface (include/mcr.h): one measures a hardware ceiling that the transport is compared
 * with, the other exposes the random-number function that the transport kernels use, so that
 * tests can hold it to the generator's published known answers.
 */
#ifndef MCR_DIAG_H
#define MCR_DIAG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/*
 * mc_reduction_probe -- measurement kernel (the paper has no counterpart): the rate of the
 * deposit step of Sec. 3.1 (Eqs. 9-11), one 64-bit reduction per coefficient per pixel segment,
 * with no transport work around it.  blocks x threads threads (threads a multiple of 32,
 * <= 1024) run `iters` iterations per warp; each picks a pseudo-random row of `tally` (device,
 * rows x row_words uint64, 8-byte aligned, caller-owned) and adds 1 to its words [0, C) in 32-lane
 * coalesced chunks, as the transport's warp-cooperative deposit does.  Afterwards the words of
 * the tally sum to (blocks threads / 32) iters C more than before.  Asynchronous on `stream`;
 * time it with events around the call.  The payload rate is 8 C (blocks threads / 32) iters
 * bytes per duration.  Returns MCR_ERR_ARG for a bad shape or a misaligned tally.
 */
int mc_reduction_probe(void *tally, int64_t rows, int32_t row_words, int32_t C, int64_t iters, int32_t blocks,
                       int32_t threads, void *stream);

/*
 * mc_philox_blocks -- test hook (the paper has no counterpart): n Philox4x32-10 blocks computed
 * on the current device by the same device function the transport kernels draw their random
 * numbers from (Salmon, Moraes, Dror & Shaw, SC'11).  ctr (host, [n][4] words), key (host,
 * [n][2] words) in; out (host, [n][4] words) receives the blocks.  The transport uses the
 * counter (packet_lo, packet_hi, event, 0) and the key (seed_lo, seed_hi ^ stream_id).
 * Synchronous (legacy default stream); allocates and frees a small device buffer.
 * 1 <= n <= 2^20, else MCR_ERR_ARG.
 */
int mc_philox_blocks(const uint32_t *ctr, const uint32_t *key, int32_t n, uint32_t *out);

/*
 * dn_wait_probe -- test hook (the paper has no counterpart): the denoiser kernels' bounded
 * mbarrier wait made to run out.  One warp waits, with the same wait function the tensor-core
 * kernels use but limited to `spins` polls (1 <= spins <= 2^24, else MCR_ERR_ARG), on an mbarrier
 * that nothing arrives at; when the wait gives up it latches the kernels' wait-failure bit in the
 * denoiser's device error word -- the status dn_check returns (MCR_ERR_CUDA, then cleared) -- and
 * *timed_out (host) is 1.  Nothing is left in flight, so the context stays usable.  Synchronises
 * `stream`.
 */
int dn_wait_probe(uint32_t spins, int32_t *timed_out, void *stream);

#ifdef __cplusplus
}
#endif

#endif /* MCR_DIAG_H */
