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

// One-hot species count of a shell neighbour with storage code c: 1 << c,
// and 0 for c = 32 (the species whose field shifts out of the word).
__device__ __forceinline__ uint32_t onehot(uint32_t c) { return __funnelshift_lc(0u, 1u, c); }

// dp4a with an unsigned first and a signed second operand: c + sum of the
// four byte products
__device__ __forceinline__ int dp4a_us(uint32_t a, uint32_t b, int c) {
  int d;
  asm("dp4a.u32.s32 %0, %1, %2, %3;" : "=r"(d) : "r"(a), "r"(b), "r"(c));
  return d;
}

// Energy change of a swap (EPI model) from the one-hot species counts of
// the anchor's and the partner's shells, for storage codes 8 sigma (K <= 5):
// byte s of a count word counts species s in that shell (species 4, code
// 32, shifts out).  F_m = 0x80808080 + acc_i[m] - acc_j[m] holds 128 + n_i -
// n_j in byte s (no borrows: counts <= 24).  The (p, q) difference row holds,
// per shell m and byte t, the bytes t of D'_{m,s} for s = 0..3 in one word
// (D' = D_{m,s} - D_{m,4}, D_{m,s} = V_m(q,s) - V_m(p,s); the species-4
// column folds away because every shell has as many sites around i as
// around j), and at byte offset DOFF_C the int64 constant C = 128 sum D' +
// the i-j bond term.  Then dE = sum_t 2^{8t} P_t - C with P_t = sum_m
// dp4a(F_m, word (m, t)) (|P_t| < 2^20).
template <int M, int DOFF_C>
__device__ __forceinline__ long long delta_e_dp4a(const uint32_t* acc_i, const uint32_t* acc_j,
                                                  const uint8_t* row) {
  uint32_t p0 = 0, p1 = 0, p2 = 0;
  int p3 = 0;
#pragma unroll
  for (int m = 0; m < M; ++m) {
    const uint4 d = reinterpret_cast<const uint4*>(row)[m];
    const uint32_t F = 0x80808080u + acc_i[m] - acc_j[m];
    p0 = __dp4a(F, d.x, p0);
    p1 = __dp4a(F, d.y, p1);
    p2 = __dp4a(F, d.z, p2);
    p3 = dp4a_us(F, d.w, p3);
  }
  const uint32_t lo = p0 + (p1 << 8);                          // < 2^29
  const int hi = static_cast<int>(p2) + p3 * 256;              // |hi| < 2^29
  return (static_cast<long long>(hi) << 16) + lo - *reinterpret_cast<const long long*>(row + DOFF_C);
}

}  // namespace smcx
