// mcr_probe.cu -- mc_reduction_probe: the rate at which this GPU absorbs the tally's 64-bit
// reductions when nothing else runs, the ceiling of the track-length deposit (the deposit of
// Sec. 3.1, Eqs. 9-11, is one 64-bit fixed-point reduction per harmonic coefficient per pixel
// segment).  Each warp repeatedly picks a pseudo-random pixel row of a tally laid out like the
// transport's (rows of row_words 64-bit words) and adds 1 to its first C words in the deposit's
// access pattern: 32-lane coalesced chunks of consecutive words.  Rows are uniform over the
// tally, so the probe has none of the hot-pixel contention a real source has: an upper bound.
#include "mcr_internal.h"

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

}  // namespace

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
