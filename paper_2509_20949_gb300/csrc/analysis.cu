// analysis.cu -- analyses of a lattice's occupancy used in Sec. 3.2 of the
// paper: composition profiles along a cylinder (its atom-probe-like
// cylinders, r = 12a and l = 72a there) and connected clusters of chosen
// species (precipitate sizes).  All integer arithmetic; positions in half
// units h = a/2 of the conventional cell.
#include "kernels.h"

namespace smcx {
namespace {

__device__ __forceinline__ uint32_t species_at(const Geom& g, const uint8_t* occ, int b, int z,
                                               int y, int x) {
  if (!g.pack4) return occ[dev_row(g, b, z, y) + x] / static_cast<uint32_t>(g.W);
  const uint8_t v = occ[dev_row(g, b >> 1, z, y) + x];
  return (b & 1) ? static_cast<uint32_t>(v >> 4) : static_cast<uint32_t>(v & 15);
}

__device__ __forceinline__ int pmod_h(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// Species counts per bin of a cylinder: axis `axis`, base point o (h units),
// radius^2 r2max and length `length` (h units).  A site at h is inside when
// t = (h_axis - o_axis) mod 2n_axis < length and the squared minimum-image
// distance to the axis (components in (-n, n], periodic images of 2n)
// is <= r2max; bin = t * n_bins / length.  Block histograms in shared memory.
__global__ void k_profile(const Geom g, const uint8_t* __restrict__ occ, int axis, int o0, int o1,
                          int o2, unsigned long long r2max, uint32_t length, uint32_t n_bins,
                          unsigned long long* __restrict__ counts, uint32_t n_cells) {
  extern __shared__ uint32_t s_h[];
  const uint32_t nh = n_bins * static_cast<uint32_t>(g.K);
  for (uint32_t i = threadIdx.x; i < nh; i += blockDim.x) s_h[i] = 0;
  __syncthreads();
  const int o[3] = {o0, o1, o2};
  for (uint32_t cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n_cells;
       cell += gridDim.x * blockDim.x) {
    const int c[3] = {static_cast<int>(cell % g.n[0]), static_cast<int>((cell / g.n[0]) % g.n[1]),
                      static_cast<int>(cell / (static_cast<uint32_t>(g.n[0]) * g.n[1]))};
    for (int b = 0; b < g.nb; ++b) {
      int h[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) h[d] = 2 * c[d] + basis_comp(g.kind, b, d);
      const int t = pmod_h(h[axis] - o[axis], 2 * g.n[axis]);
      if (t >= static_cast<int>(length)) continue;
      unsigned long long r2 = 0;
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        if (d == axis) continue;
        int dd = pmod_h(h[d] - o[d], 2 * g.n[d]);
        if (dd > g.n[d]) dd -= 2 * g.n[d];
        r2 += static_cast<unsigned long long>(static_cast<long long>(dd) * dd);
      }
      if (r2 > r2max) continue;
      const uint32_t bin = static_cast<uint32_t>(static_cast<unsigned long long>(t) * n_bins / length);
      atomicAdd(&s_h[bin * g.K + species_at(g, occ, b, c[2], c[1], c[0])], 1u);
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nh; i += blockDim.x)
    if (s_h[i]) atomicAdd(&counts[i], static_cast<unsigned long long>(s_h[i]));
}

// The same counts, a warp per conventional row (z, y) and a lane per 4
// cells of it (32-bit loads per row group, up to 8 in flight; bytes past
// n_x are the row padding and masked).  The origin is brought into [0, 2n) once, so a
// periodic difference takes one conditional add; bin_of[t] (shared, one
// entry per half-unit position along the axis, 0xFFFF past `length`)
// replaces the per-site division, and lanes of a warp that add to the same
// (bin, species) counter combine first (__match_any_sync), so a row of one
// bin costs one shared atomic per species present.  2 n_axis <= kBinTab.
constexpr int kBinTab = 16384;

__global__ void k_profile_rows(const Geom g, const uint8_t* __restrict__ occ, int axis, int o0,
                               int o1, int o2, unsigned long long r2max, uint32_t length,
                               uint32_t n_bins, unsigned long long* __restrict__ counts) {
  extern __shared__ uint32_t s_h[];
  const uint32_t K = static_cast<uint32_t>(g.K);
  const uint32_t nh = n_bins * K;
  uint16_t* const bin_of = reinterpret_cast<uint16_t*>(s_h + nh);
  const int n2[3] = {2 * g.n[0], 2 * g.n[1], 2 * g.n[2]};
  for (uint32_t i = threadIdx.x; i < nh; i += blockDim.x) s_h[i] = 0;
  for (int t = threadIdx.x; t < n2[axis]; t += blockDim.x)
    bin_of[t] = static_cast<uint32_t>(t) < length
                    ? static_cast<uint16_t>(static_cast<unsigned long long>(t) * n_bins / length)
                    : static_cast<uint16_t>(0xFFFF);
  __syncthreads();
  const int o[3] = {o0, o1, o2};  // in [0, 2n)
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const uint32_t rows = static_cast<uint32_t>(ny) * nz;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  const uint32_t chunks = static_cast<uint32_t>(nx + 3) / 4;
  const uint32_t inv = (65536u + static_cast<uint32_t>(g.W) - 1u) / static_cast<uint32_t>(g.W);
  const bool reg_count = axis != 0 && K <= 8u && nx < 65536;
  for (uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const int y = static_cast<int>(r % ny), z = static_cast<int>(r / ny);
    for (int b = 0; b < g.nb; ++b) {
      // this row's y and z parts (h = 2c + basis; differences to o in [0, 2n))
      int d[3];
      d[1] = 2 * y + basis_comp(g.kind, b, 1) - o[1];
      d[2] = 2 * z + basis_comp(g.kind, b, 2) - o[2];
      d[1] += d[1] < 0 ? n2[1] : 0;
      d[2] += d[2] < 0 ? n2[2] : 0;
      unsigned long long r2row = 0;
      uint32_t row_bin = 0xFFFFu;
#pragma unroll
      for (int e = 1; e < 3; ++e) {
        if (e == axis) {
          row_bin = bin_of[d[e]];
        } else {
          const long long dd = d[e] > g.n[e] ? d[e] - n2[e] : d[e];
          r2row += static_cast<unsigned long long>(dd * dd);
        }
      }
      if (axis != 0 && (row_bin == 0xFFFFu || r2row > r2max)) continue;  // warp-uniform
      const int bx = basis_comp(g.kind, b, 0);
      const uint8_t* row = occ + dev_row(g, g.pack4 ? b >> 1 : b, z, y);
      const uint32_t shift = g.pack4 ? 4u * (b & 1) : 0u;
      // along y or z the row has one bin: with K <= 8 and rows shorter than
      // 2^16 cells each lane counts species in 16-bit fields (species s in
      // field s & 3 of reg[s >> 2]; a field's sum over the warp is at most
      // n_x), and the warp adds the row's counts once
      if (reg_count) {
        unsigned long long reg[2] = {0ull, 0ull};
        for (uint32_t c8 = 0; c8 < chunks; c8 += 256) {
          uint32_t wv[8];
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint32_t c = c8 + 32u * k + lane;
            wv[k] = c < chunks ? *reinterpret_cast<const uint32_t*>(row + 4 * c) : 0u;
          }
#pragma unroll
          for (int k = 0; k < 8; ++k) {
            const uint32_t c = c8 + 32u * k + lane;
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int x = static_cast<int>(4 * c) + e;
              if (c >= chunks || x >= nx) continue;
              int dx = 2 * x + bx - o[0];
              dx += dx < 0 ? n2[0] : 0;
              const long long dd = dx > nx ? dx - n2[0] : dx;
              if (r2row + static_cast<unsigned long long>(dd * dd) > r2max) continue;
              const uint32_t code = (wv[k] >> (8 * e)) & 0xFFu;
              const uint32_t sp = g.pack4 ? (code >> shift) & 15u : (code * inv) >> 16;
              const unsigned long long one = 1ull << (16 * (sp & 3u));
              if (sp < 4u) reg[0] += one;
              else reg[1] += one;
            }
          }
        }
        uint32_t f[4];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          f[2 * h] = __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(reg[h]));
          f[2 * h + 1] = __reduce_add_sync(0xffffffffu, static_cast<uint32_t>(reg[h] >> 32));
        }
        if (lane == 0)
          for (uint32_t sp = 0; sp < K; ++sp) {
            const uint32_t v = (f[sp >> 1] >> (16 * (sp & 1u))) & 0xFFFFu;
            if (v) atomicAdd(&s_h[row_bin * K + sp], v);
          }
        continue;
      }
      // up to 8 loads of the row in flight before their sites are counted
      for (uint32_t c8 = 0; c8 < chunks; c8 += 256) {
        uint32_t wv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const uint32_t c = c8 + 32u * k + lane;
          wv[k] = c < chunks ? *reinterpret_cast<const uint32_t*>(row + 4 * c) : 0u;  // rows pad to 16 B
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (c8 + 32u * k >= chunks) break;  // warp-uniform
          const uint32_t c = c8 + 32u * k + lane;
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int x = static_cast<int>(4 * c) + e;
            uint32_t key = 0xFFFFFFFFu;
            if (c < chunks && x < nx) {
              int dx = 2 * x + bx - o[0];
              dx += dx < 0 ? n2[0] : 0;
              uint32_t bin = row_bin;
              unsigned long long r2 = r2row;
              if (axis == 0) {
                bin = bin_of[dx];
              } else {
                const long long dd = dx > nx ? dx - n2[0] : dx;
                r2 += static_cast<unsigned long long>(dd * dd);
              }
              if (bin != 0xFFFFu && r2 <= r2max) {
                const uint32_t code = (wv[k] >> (8 * e)) & 0xFFu;
                const uint32_t sp = g.pack4 ? (code >> shift) & 15u : (code * inv) >> 16;
                key = bin * K + sp;
              }
            }
            const unsigned act = __ballot_sync(0xffffffffu, key != 0xFFFFFFFFu);
            if (key != 0xFFFFFFFFu) {
              const unsigned same = __match_any_sync(act, key);
              if (lane == static_cast<uint32_t>(__ffs(same) - 1)) atomicAdd(&s_h[key], __popc(same));
            }
          }
        }
      }
    }
  }
  __syncthreads();
  for (uint32_t i = threadIdx.x; i < nh; i += blockDim.x)
    if (s_h[i]) atomicAdd(&counts[i], static_cast<unsigned long long>(s_h[i]));
}

}  // namespace

cudaError_t launch_profile(const Geom& g, const uint8_t* occ, int axis, const int* origin_h,
                           unsigned long long r2max, uint32_t length, uint32_t n_bins,
                           unsigned long long* counts, int n_sm, cudaStream_t st) {
  const uint32_t n_cells = static_cast<uint32_t>(g.n[0]) * g.n[1] * g.n[2];
  if (2 * g.n[axis] <= kBinTab) {
    const uint32_t rows = static_cast<uint32_t>(g.n[1]) * g.n[2];
    uint32_t grid = (rows + 7) / 8;  // a warp per row
    if (grid > static_cast<uint32_t>(n_sm) * 8) grid = static_cast<uint32_t>(n_sm) * 8;
    if (grid == 0) grid = 1;
    const size_t smem = sizeof(uint32_t) * n_bins * static_cast<uint32_t>(g.K) +
                        sizeof(uint16_t) * 2 * g.n[axis];
    int o[3];
    for (int d = 0; d < 3; ++d) {
      const int m = 2 * g.n[d];
      o[d] = ((origin_h[d] % m) + m) % m;
    }
    if (smem > 48 * 1024) {
      const cudaError_t e = cudaFuncSetAttribute(k_profile_rows,
                                                 cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                 static_cast<int>(smem));
      if (e != cudaSuccess) return e;
    }
    k_profile_rows<<<grid, 256, smem, st>>>(g, occ, axis, o[0], o[1], o[2], r2max, length, n_bins,
                                            counts);
    return cudaGetLastError();
  }
  uint32_t grid = (n_cells + 255) / 256;
  if (grid > static_cast<uint32_t>(n_sm) * 8) grid = static_cast<uint32_t>(n_sm) * 8;
  if (grid == 0) grid = 1;
  const size_t smem = sizeof(uint32_t) * n_bins * static_cast<uint32_t>(g.K);
  k_profile<<<grid, 256, smem, st>>>(g, occ, axis, origin_h[0], origin_h[1], origin_h[2], r2max,
                                     length, n_bins, counts, n_cells);
  return cudaGetLastError();
}

}  // namespace smcx

// ---- clusters: connected components of member sites (species in a mask)
// through first-shell neighbours, periodic.  Union-find on canonical site
// indices (((z n_y + y) n_x + x) nb + b): hooking links the larger root
// under the smaller with a compare-and-swap (lock-free), finds halve paths;
// every loop is capped and reports through *err instead of spinning on.
namespace smcx {
namespace {

constexpr uint32_t kNone = 0xFFFFFFFFu;
constexpr uint32_t kLoopCap = 1u << 26;

struct SiteGeom {
  int n[3], nb, kind;
};

__device__ __forceinline__ bool member(const Geom& g, const uint8_t* occ, uint32_t mask,
                                       uint32_t i) {
  const int b = static_cast<int>(i % g.nb);
  const uint32_t cell = i / g.nb;
  const int x = static_cast<int>(cell % g.n[0]);
  const int y = static_cast<int>((cell / g.n[0]) % g.n[1]);
  const int z = static_cast<int>(cell / (static_cast<uint32_t>(g.n[0]) * g.n[1]));
  return (mask >> species_at(g, occ, b, z, y, x)) & 1u;
}

// canonical index of the site at h = 2c + basis_b + v (periodic)
__device__ __forceinline__ uint32_t site_plus(const Geom& g, uint32_t i, int vx, int vy, int vz) {
  const int b = static_cast<int>(i % g.nb);
  const uint32_t cell = i / g.nb;
  const int c[3] = {static_cast<int>(cell % g.n[0]), static_cast<int>((cell / g.n[0]) % g.n[1]),
                    static_cast<int>(cell / (static_cast<uint32_t>(g.n[0]) * g.n[1]))};
  const int v[3] = {vx, vy, vz};
  int q[3], par[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int h = 2 * c[d] + basis_comp(g.kind, b, d) + v[d];
    par[d] = h & 1;
    q[d] = pmod_h((h - par[d]) / 2, g.n[d]);
  }
  const int bp = basis_of_parity(g.kind, par[0], par[1], par[2]);
  return ((static_cast<uint32_t>(q[2]) * g.n[1] + q[1]) * g.n[0] + q[0]) * g.nb + bp;
}

__device__ __forceinline__ uint32_t find_root(uint32_t* lab, uint32_t x, unsigned int* err) {
  for (uint32_t it = 0; it < kLoopCap; ++it) {
    const uint32_t p = *reinterpret_cast<volatile uint32_t*>(lab + x);
    if (p == x) return x;
    const uint32_t gp = *reinterpret_cast<volatile uint32_t*>(lab + p);
    if (gp != p) atomicCAS(lab + x, p, gp);  // path halving (labels only move to ancestors)
    x = gp;
  }
  atomicOr(err, 1u);
  return x;
}

__global__ void k_cc_init(const Geom g, const uint8_t* __restrict__ occ, uint32_t mask,
                          uint32_t* __restrict__ lab, uint32_t* __restrict__ cnt, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    lab[i] = member(g, occ, mask, i) ? i : kNone;
    cnt[i] = 0;
  }
}

__global__ void k_cc_hook(const Geom g, uint32_t* lab, uint32_t n, unsigned int* err) {
  // lexicographically positive first-shell vectors: every bond once
  constexpr int kBcc[4][3] = {{1, 1, 1}, {1, 1, -1}, {1, -1, 1}, {1, -1, -1}};
  constexpr int kFcc[6][3] = {{1, 1, 0}, {1, -1, 0}, {1, 0, 1}, {1, 0, -1}, {0, 1, 1}, {0, 1, -1}};
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (*reinterpret_cast<volatile uint32_t*>(lab + i) == kNone) continue;
    const int nv = g.kind == 0 ? 4 : 6;
    for (int k = 0; k < nv; ++k) {
      const int* v = g.kind == 0 ? kBcc[k] : kFcc[k];
      const uint32_t j = site_plus(g, i, v[0], v[1], v[2]);
      if (*reinterpret_cast<volatile uint32_t*>(lab + j) == kNone) continue;
      uint32_t a = i, b = j;
      for (uint32_t it = 0;; ++it) {
        if (it >= kLoopCap) {
          atomicOr(err, 2u);
          break;
        }
        a = find_root(lab, a, err);
        b = find_root(lab, b, err);
        if (a == b) break;
        if (a < b) {
          const uint32_t t = a;
          a = b;
          b = t;
        }
        if (atomicCAS(lab + a, a, b) == a) break;  // root a now under b
      }
    }
  }
}

__global__ void k_cc_count(uint32_t* lab, uint32_t* __restrict__ cnt, uint32_t n,
                           unsigned int* err) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    if (lab[i] == kNone) continue;
    atomicAdd(cnt + find_root(lab, i, err), 1u);
  }
}

// sizes of the clusters (nonzero counts) appended to out
__global__ void k_cc_compact(const uint32_t* __restrict__ cnt, uint32_t* __restrict__ out,
                             unsigned long long* __restrict__ n_out, uint32_t n) {
  for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
    if (cnt[i]) out[atomicAdd(n_out, 1ull)] = cnt[i];
}

}  // namespace

cudaError_t launch_clusters(const Geom& g, const uint8_t* occ, uint32_t mask, uint32_t* lab,
                            uint32_t* cnt, unsigned long long* n_out, unsigned int* err,
                            uint32_t n_sites, int n_sm, cudaStream_t st) {
  uint32_t grid = (n_sites + 255) / 256;
  if (grid > static_cast<uint32_t>(n_sm) * 16) grid = static_cast<uint32_t>(n_sm) * 16;
  if (grid == 0) grid = 1;
  k_cc_init<<<grid, 256, 0, st>>>(g, occ, mask, lab, cnt, n_sites);
  k_cc_hook<<<grid, 256, 0, st>>>(g, lab, n_sites, err);
  k_cc_count<<<grid, 256, 0, st>>>(lab, cnt, n_sites, err);
  // the labels are no longer needed: the sizes go to their array
  k_cc_compact<<<grid, 256, 0, st>>>(cnt, lab, n_out, n_sites);
  return cudaGetLastError();
}

}  // namespace smcx
