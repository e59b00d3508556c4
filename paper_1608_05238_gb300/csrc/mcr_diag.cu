// mcr_diag.cu -- measurement and test entry points of libmcr (include/mcr_diag.h), not part of
// the method's interface.
//
// mc_reduction_probe: the rate at which this GPU absorbs the tally's 64-bit
// reductions when nothing else runs, the ceiling of the track-length deposit (the deposit of
// Sec. 3.1, Eqs. 9-11, is one 64-bit fixed-point reduction per harmonic coefficient per pixel
// segment).  Each warp repeatedly picks a pseudo-random pixel row of a tally laid out like the
// transport's (rows of row_words 64-bit words) and adds 1 to its first C words in the deposit's
// access pattern: 32-lane coalesced chunks of consecutive words.  Rows are uniform over the
// tally, so the probe has none of the hot-pixel contention a real source has: an upper bound.
#include <stdlib.h>

#include "mcr_internal.h"
#include "mcr_rng.cuh"
#include "../../include/mcr_diag.h"

namespace {

__device__ __forceinline__ unsigned long long mix64(unsigned long long z) {  // splitmix64 finaliser
  z += 0x9E3779B97F4A7C15ull;
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

__global__ void k_reduction_probe(unsigned long long *__restrict__ tally, long long rows, int row_words, int C,
                                  long long iters) {
  const int lane = threadIdx.x & 31;
  const unsigned long long warp = (blockIdx.x * (unsigned long long)blockDim.x + threadIdx.x) >> 5;
  // four rows per step, so that the reductions of several rows are in flight together; the row is
  // the high half of a 64-bit hash scaled to [0, rows) (a multiply, no division)
  long long it = 0;
  for (; it + 4 <= iters; it += 4) {
    unsigned long long *r[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
      const unsigned long long h = mix64(warp * 0x100000001ull + (unsigned long long)(it + k));
      r[k] = tally + (long long)__umul64hi(h, (unsigned long long)rows) * row_words;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
      for (int j = lane; j < C; j += 32) atomicAdd(r[k] + j, 1ull);
  }
  for (; it < iters; ++it) {
    const unsigned long long h = mix64(warp * 0x100000001ull + (unsigned long long)it);
    unsigned long long *r = tally + (long long)__umul64hi(h, (unsigned long long)rows) * row_words;
    for (int j = lane; j < C; j += 32) atomicAdd(r + j, 1ull);
  }
}

// One Philox4x32-10 block per thread, with the transport kernels' own device function.
__global__ void k_philox_blocks(const unsigned *__restrict__ ctr, const unsigned *__restrict__ key, int n,
                                unsigned *__restrict__ out) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const uint4 c = make_uint4(ctr[4 * i], ctr[4 * i + 1], ctr[4 * i + 2], ctr[4 * i + 3]);
  const uint4 r = mcr::philox4x32_10_block(c, key[2 * i], key[2 * i + 1]);
  out[4 * i] = r.x;
  out[4 * i + 1] = r.y;
  out[4 * i + 2] = r.z;
  out[4 * i + 3] = r.w;
}

}  // namespace

extern "C" int mc_philox_blocks(const uint32_t *ctr, const uint32_t *key, int32_t n, uint32_t *out) {
  if (!ctr || !key || !out || n <= 0 || n > (1 << 20)) return MCR_ERR_ARG;
  unsigned *d = nullptr;
  const size_t words = (size_t)n * 10;  // [n][4] counters, [n][2] keys, [n][4] outputs
  if (cudaMalloc(&d, words * sizeof(unsigned)) != cudaSuccess) {
    cudaGetLastError();
    return MCR_ERR_NOMEM;
  }
  int rc = MCR_OK;
  if (cudaMemcpy(d, ctr, (size_t)n * 4 * sizeof(unsigned), cudaMemcpyHostToDevice) != cudaSuccess ||
      cudaMemcpy(d + 4 * (size_t)n, key, (size_t)n * 2 * sizeof(unsigned), cudaMemcpyHostToDevice) != cudaSuccess) {
    rc = MCR_ERR_CUDA;
  } else {
    k_philox_blocks<<<(n + 127) / 128, 128>>>(d, d + 4 * (size_t)n, n, d + 6 * (size_t)n);
    if (cudaGetLastError() != cudaSuccess ||
        cudaMemcpy(out, d + 6 * (size_t)n, (size_t)n * 4 * sizeof(unsigned), cudaMemcpyDeviceToHost) != cudaSuccess)
      rc = MCR_ERR_CUDA;
  }
  cudaFree(d);
  return rc;
}

extern "C" int mc_reduction_probe(void *tally, int64_t rows, int32_t row_words, int32_t C, int64_t iters,
                                  int32_t blocks, int32_t threads, void *stream) {
  if (!tally || rows <= 0 || C <= 0 || row_words < C || iters < 0 || blocks <= 0 || threads <= 0 || threads % 32 ||
      threads > 1024)
    return MCR_ERR_ARG;
  if ((reinterpret_cast<uintptr_t>(tally) & 7) != 0) return MCR_ERR_ARG;
  k_reduction_probe<<<blocks, threads, 0, (cudaStream_t)stream>>>(static_cast<unsigned long long *>(tally), rows,
                                                                  row_words, C, iters);
  return cudaGetLastError() == cudaSuccess ? MCR_OK : MCR_ERR_CUDA;
}
