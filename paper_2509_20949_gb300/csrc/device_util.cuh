// device_util.cuh -- small device helpers shared by the kernels.
#pragma once

#include "smcx_common.cuh"

namespace smcx {

// Warp-reduce the trial statistics and add them (order-free integer atomics,
// hence exact) to this call's and the cumulative counters.
__device__ __forceinline__ void warp_reduce_add_stats(unsigned long long* stats, uint64_t att,
                                                      uint64_t unl, uint64_t acc, int64_t de) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    att += __shfl_down_sync(0xffffffffu, att, off);
    unl += __shfl_down_sync(0xffffffffu, unl, off);
    acc += __shfl_down_sync(0xffffffffu, acc, off);
    de += __shfl_down_sync(0xffffffffu, de, off);
  }
  if ((threadIdx.x & 31) == 0 && (att | unl | acc | static_cast<uint64_t>(de)) != 0) {
    atomicAdd(stats + kStatCall + 0, att);
    atomicAdd(stats + kStatCall + 1, unl);
    atomicAdd(stats + kStatCall + 2, acc);
    atomicAdd(stats + kStatCall + 3, static_cast<unsigned long long>(de));
    atomicAdd(stats + kStatCum + 0, att);
    atomicAdd(stats + kStatCum + 1, unl);
    atomicAdd(stats + kStatCum + 2, acc);
    atomicAdd(stats + kStatCum + 3, static_cast<unsigned long long>(de));
  }
}

}  // namespace smcx
