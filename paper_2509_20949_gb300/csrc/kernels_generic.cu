// kernels_generic.cu -- global-memory sweep and pair-count kernels for any
// lattice size (including lattices so small that a site is its own
// neighbour).  One thread runs all trials of one link cell of the active
// colour (Sec. 2.2: cells of one colour never interact); every neighbour
// index is computed from coordinates with periodic wrap.
#include "kernels.h"

namespace smcx {

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

__device__ __forceinline__ uint32_t occ_get(const uint8_t* occ, uint32_t i, int pack4) {
  if (!pack4) return occ[i];
  return (occ[i >> 1] >> ((i & 1u) * 4u)) & 15u;
}

__device__ __forceinline__ void occ_set(uint8_t* occ, uint32_t i, uint32_t v, int pack4) {
  if (!pack4) {
    occ[i] = static_cast<uint8_t>(v);
    return;
  }
  uint8_t* p = occ + (i >> 1);
  const uint32_t sh = (i & 1u) * 4u;
  *p = static_cast<uint8_t>((*p & ~(15u << sh)) | (v << sh));
}

struct SiteXYZ {
  int x, y, z, b;
};

__device__ __forceinline__ uint32_t site_of(const Geom& g, int x, int y, int z, int b) {
  return ((static_cast<uint32_t>(z) * g.n[1] + y) * g.n[0] + x) * g.nb + b;
}

__device__ __forceinline__ SiteXYZ xyz_of(const Geom& g, uint32_t i) {
  SiteXYZ s;
  s.b = static_cast<int>(i % g.nb);
  uint32_t c = i / g.nb;
  s.x = static_cast<int>(c % g.n[0]);
  c /= g.n[0];
  s.y = static_cast<int>(c % g.n[1]);
  s.z = static_cast<int>(c / g.n[1]);
  return s;
}

__device__ __forceinline__ uint32_t neighbour(const Geom& g, const SiteXYZ& s, int dx, int dy,
                                              int dz) {
  const int hx = pmod(2 * s.x + basis_comp(g.kind, s.b, 0) + dx, 2 * g.n[0]);
  const int hy = pmod(2 * s.y + basis_comp(g.kind, s.b, 1) + dy, 2 * g.n[1]);
  const int hz = pmod(2 * s.z + basis_comp(g.kind, s.b, 2) + dz, 2 * g.n[2]);
  const int bp = basis_of_parity(g.kind, hx & 1, hy & 1, hz & 1);
  return site_of(g, hx >> 1, hy >> 1, hz >> 1, bp);
}

__device__ __forceinline__ void warp_reduce_add_stats(unsigned long long* stats, uint64_t att,
                                                      uint64_t unl, uint64_t acc, int64_t de) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) {
    att += __shfl_down_sync(0xffffffffu, att, off);
    unl += __shfl_down_sync(0xffffffffu, unl, off);
    acc += __shfl_down_sync(0xffffffffu, acc, off);
    de += __shfl_down_sync(0xffffffffu, de, off);
  }
  if ((threadIdx.x & 31) == 0) {
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

// One colour phase.  Thread -> active cell (cx, cy, cz) with c_d = 2 a_d + bit_d
// (or 0 where m_d == 1); trials in raster order: basis fastest, then shifted
// x, y, z.  The energy change leaves out every occurrence of the two swapped
// sites (exact on any periodic lattice).
__global__ void __launch_bounds__(128) k_sweep_generic(const Geom g, const PhaseArgs a,
                                                      const ShellParam sp,
                                                      const __grid_constant__ Tables tab,
                                                      uint8_t* __restrict__ occ,
                                                      const int64_t* __restrict__ V,
                                                      unsigned long long* __restrict__ stats,
                                                      uint32_t n_active, uint32_t ax_n,
                                                      uint32_t ay_n) {
  __shared__ uint32_t s_tab[kTabWords];
  for (int w = threadIdx.x; w < kTabWords; w += blockDim.x) s_tab[w] = tab.w[w];
  __syncthreads();

  uint64_t att = 0, unl = 0, acc = 0;
  int64_t sum_de = 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < n_active) {
    const uint32_t axi = tid % ax_n, ayi = (tid / ax_n) % ay_n, azi = tid / (ax_n * ay_n);
    const int c[3] = {
        g.m[0] == 1 ? 0 : static_cast<int>(2 * axi + (a.colour & 1)),
        g.m[1] == 1 ? 0 : static_cast<int>(2 * ayi + ((a.colour >> 1) & 1)),
        g.m[2] == 1 ? 0 : static_cast<int>(2 * azi + ((a.colour >> 2) & 1))};
    const uint32_t cid = (static_cast<uint32_t>(c[2]) * g.m[1] + c[1]) * g.m[0] + c[0];
    int lo[3], hi[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      lo[d] = static_cast<int>((static_cast<int64_t>(c[d]) * g.n[d]) / g.m[d]);
      hi[d] = static_cast<int>((static_cast<int64_t>(c[d] + 1) * g.n[d]) / g.m[d]);
    }
    const int K = g.K;
    uint32_t k = 0;
    U4 w = {0, 0, 0, 0};
    for (int zs = lo[2]; zs < hi[2]; ++zs)
      for (int ys = lo[1]; ys < hi[1]; ++ys)
        for (int xs = lo[0]; xs < hi[0]; ++xs)
          for (int b = 0; b < g.nb; ++b, ++k) {
            SiteXYZ si;
            si.x = pmod(xs + a.shift[0], g.n[0]);
            si.y = pmod(ys + a.shift[1], g.n[1]);
            si.z = pmod(zs + a.shift[2], g.n[2]);
            si.b = b;
            const uint32_t i = site_of(g, si.x, si.y, si.z, b);
            if ((k & 1u) == 0) w = philox4x32_10(k >> 1, cid, a.t, 0u, g.seed_lo, g.seed_hi);
            const uint32_t wa = (k & 1u) ? w.z : w.x;
            const uint32_t wb = (k & 1u) ? w.w : w.y;
            const uint32_t dir = mulhi32(wa, static_cast<uint32_t>(g.z1));
            const uint32_t j = neighbour(g, si, sp.v[dir][0], sp.v[dir][1], sp.v[dir][2]);
            const SiteXYZ sj = xyz_of(g, j);
            const uint32_t p = occ_get(occ, i, g.pack4), q = occ_get(occ, j, g.pack4);
            ++att;
            if (p == q) continue;
            ++unl;
            int64_t de = 0;
            for (int m = 0; m < g.M; ++m) {
              const int64_t* Vm = V + static_cast<int64_t>(m) * K * K;
              for (int t = sp.start[m]; t < sp.start[m + 1]; ++t) {
                const uint32_t ki = neighbour(g, si, sp.v[t][0], sp.v[t][1], sp.v[t][2]);
                if (ki != i && ki != j) {
                  const uint32_t sk = occ_get(occ, ki, g.pack4);
                  de += Vm[q * K + sk] - Vm[p * K + sk];
                }
                const uint32_t kj = neighbour(g, sj, sp.v[t][0], sp.v[t][1], sp.v[t][2]);
                if (kj != i && kj != j) {
                  const uint32_t sk = occ_get(occ, kj, g.pack4);
                  de += Vm[p * K + sk] - Vm[q * K + sk];
                }
              }
            }
            bool accept;
            if (de <= 0) {
              accept = true;
            } else if (a.mode == kModeZeroT) {
              accept = false;
            } else if (a.mode == kModeAcceptAll) {
              accept = true;
            } else {
              const uint64_t idx = static_cast<uint64_t>(de) >> a.s;
              if (idx >= (1ull << 27)) {
                accept = false;
              } else {
                const uint32_t thr = compose_threshold(s_tab[idx & 511u], s_tab[512 + ((idx >> 9) & 511u)],
                                                       s_tab[1024 + (idx >> 18)]);
                accept = wb < thr;
              }
            }
            if (accept) {
              occ_set(occ, i, q, g.pack4);
              occ_set(occ, j, p, g.pack4);
              ++acc;
              sum_de += de;
            }
          }
  }
  warp_reduce_add_stats(stats, att, unl, acc, sum_de);
}

// Directed pair counts N_m[p'][p] over every site (Sec. 3.2, Eq. 9), shared
// memory accumulators for K <= 32, global atomics otherwise.
__global__ void __launch_bounds__(256) k_pair_count_generic(const Geom g, const ShellParam sp,
                                                           int n_shells,
                                                           const uint8_t* __restrict__ occ,
                                                           unsigned long long* __restrict__ counts,
                                                           uint32_t N) {
  extern __shared__ uint32_t s_cnt[];
  const int K = g.K;
  const bool in_smem = K <= 32;
  const int n_cnt = n_shells * K * K;
  if (in_smem)
    for (int c = threadIdx.x; c < n_cnt; c += blockDim.x) s_cnt[c] = 0;
  __syncthreads();
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < N; i += gridDim.x * blockDim.x) {
    const SiteXYZ s = xyz_of(g, i);
    const uint32_t pc = occ_get(occ, i, g.pack4);
    for (int m = 0; m < n_shells; ++m)
      for (int t = sp.start[m]; t < sp.start[m + 1]; ++t) {
        const uint32_t k = neighbour(g, s, sp.v[t][0], sp.v[t][1], sp.v[t][2]);
        const uint32_t p = occ_get(occ, k, g.pack4);
        const int slot = (m * K + pc) * K + p;
        if (in_smem)
          atomicAdd(&s_cnt[slot], 1u);
        else
          atomicAdd(&counts[slot], 1ull);
      }
  }
  __syncthreads();
  if (in_smem)
    for (int c = threadIdx.x; c < n_cnt; c += blockDim.x)
      if (s_cnt[c]) atomicAdd(&counts[c], static_cast<unsigned long long>(s_cnt[c]));
}

cudaError_t launch_sweep_generic(const Geom& g, const PhaseArgs& a, const ShellParam& sp,
                                 const Tables& tab, uint8_t* occ, const int64_t* V,
                                 unsigned long long* stats, cudaStream_t st) {
  uint32_t cnt[3];
  for (int d = 0; d < 3; ++d) {
    const int bit = (a.colour >> d) & 1;
    if (g.m[d] == 1) {
      if (bit) return cudaSuccess;  // no cell of this colour
      cnt[d] = 1;
    } else {
      cnt[d] = static_cast<uint32_t>(g.m[d] / 2);
    }
  }
  const uint32_t n_active = cnt[0] * cnt[1] * cnt[2];
  const uint32_t blocks = (n_active + 127) / 128;
  k_sweep_generic<<<blocks, 128, 0, st>>>(g, a, sp, tab, occ, V, stats, n_active, cnt[0], cnt[1]);
  return cudaGetLastError();
}

cudaError_t launch_pair_count_generic(const Geom& g, const ShellParam& sp, int n_shells,
                                      const uint8_t* occ, unsigned long long* counts, uint32_t N,
                                      int n_sm, cudaStream_t st) {
  const int K = g.K;
  const size_t smem = K <= 32 ? sizeof(uint32_t) * n_shells * K * K : 0;
  uint32_t blocks = (N + 255) / 256;
  const uint32_t cap = static_cast<uint32_t>(n_sm) * 8u;
  if (blocks > cap) blocks = cap;
  if (blocks == 0) blocks = 1;
  k_pair_count_generic<<<blocks, 256, smem, st>>>(g, sp, n_shells, occ, counts, N);
  return cudaGetLastError();
}

__global__ void k_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint32_t k0,
                              uint32_t k1, uint32_t n, uint32_t* __restrict__ out) {
  const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const U4 w = philox4x32_10(c0 + i, c1, c2, c3, k0, k1);
  out[4 * i + 0] = w.x;
  out[4 * i + 1] = w.y;
  out[4 * i + 2] = w.z;
  out[4 * i + 3] = w.w;
}

cudaError_t launch_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t key,
                               uint32_t n, uint32_t* out, cudaStream_t st) {
  if (n == 0) return cudaSuccess;
  k_philox_fill<<<(n + 255) / 256, 256, 0, st>>>(c0, c1, c2, c3, static_cast<uint32_t>(key),
                                                 static_cast<uint32_t>(key >> 32), n, out);
  return cudaGetLastError();
}

}  // namespace smcx
