// Test helper: evaluates curand's Philox4x32-10 (NVIDIA's device API, called
// as a black box) so the tests can compare it with the oracle's and the
// library's Philox.  curand_init(seed, subsequence, offset) sets key = seed,
// counter words 2,3 = subsequence and words 0,1 = offset / 4; curand4 then
// returns the generator's output for that counter.
#include <cstdint>
#include <curand_kernel.h>

__global__ void k_probe(unsigned long long seed, unsigned long long subseq,
                        unsigned long long offset4, unsigned n, unsigned* out) {
  const unsigned i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  curandStatePhilox4_32_10_t st;
  curand_init(seed, subseq, 4ull * (offset4 + i), &st);
  const uint4 v = curand4(&st);
  out[4 * i + 0] = v.x;
  out[4 * i + 1] = v.y;
  out[4 * i + 2] = v.z;
  out[4 * i + 3] = v.w;
}

extern "C" int curand_philox_probe(unsigned long long seed, unsigned long long subseq,
                                   unsigned long long offset4, unsigned n, unsigned* d_out) {
  k_probe<<<(n + 127) / 128, 128>>>(seed, subseq, offset4, n, d_out);
  return static_cast<int>(cudaDeviceSynchronize());
}
