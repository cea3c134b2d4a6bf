// kernels.h -- host-side launchers of the library's CUDA kernels.
#pragma once

#include "smcx_common.cuh"

namespace smcx {

cudaError_t launch_sweep_generic(const Geom& g, const PhaseArgs& a, const ShellParam& sp,
                                 const Tables& tab, uint8_t* occ, const int64_t* V,
                                 unsigned long long* stats, cudaStream_t st);

cudaError_t launch_pair_count_generic(const Geom& g, const ShellParam& sp, int n_shells,
                                      const uint8_t* occ, unsigned long long* counts, uint32_t N,
                                      int n_sm, cudaStream_t st);

cudaError_t launch_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t key,
                               uint32_t n, uint32_t* out, cudaStream_t st);

}  // namespace smcx
