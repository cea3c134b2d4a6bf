// kernels_generic.cu -- global-memory sweep and pair-count kernels for any
// lattice size (including lattices so small that a site is its own
// neighbour), plus the conversions between the canonical occupancy and the
// device storage.  In the sweep, one thread runs all trials of one link cell
// of the active colour (Sec. 2.2: cells of one colour never interact);
// every neighbour is located from coordinates with periodic wrap.
#include <vector>
#include <cstddef>
#include <type_traits>
#include "device_util.cuh"
#include "kernels.h"

namespace smcx {

__device__ __forceinline__ int pmod(int a, int n) {
  int r = a % n;
  return r < 0 ? r + n : r;
}

struct SiteXYZ {
  int x, y, z, b;
};

__device__ __forceinline__ uint32_t occ_get(const Geom& g, const uint8_t* occ, const SiteXYZ& s) {
  if (!g.pack4) return static_cast<uint32_t>(occ[dev_row(g, s.b, s.z, s.y) + s.x]) / g.W;
  return (occ[dev_row(g, s.b >> 1, s.z, s.y) + s.x] >> ((s.b & 1) * 4)) & 15u;
}

__device__ __forceinline__ void occ_set(const Geom& g, uint8_t* occ, const SiteXYZ& s, uint32_t v) {
  if (!g.pack4) {
    occ[dev_row(g, s.b, s.z, s.y) + s.x] = static_cast<uint8_t>(v * g.W);
    return;
  }
  uint8_t* p = occ + dev_row(g, s.b >> 1, s.z, s.y) + s.x;
  const uint32_t sh = (s.b & 1) * 4u;
  *p = static_cast<uint8_t>((*p & ~(15u << sh)) | (v << sh));
}

// canonical site index ((z*ny + y)*nx + x)*nb + b: the identity of a site
__device__ __forceinline__ uint32_t site_id(const Geom& g, const SiteXYZ& s) {
  return ((static_cast<uint32_t>(s.z) * g.n[1] + s.y) * g.n[0] + s.x) * g.nb + s.b;
}

__device__ __forceinline__ SiteXYZ neighbour(const Geom& g, const SiteXYZ& s, int dx, int dy,
                                             int dz) {
  const int hx = pmod(2 * s.x + basis_comp(g.kind, s.b, 0) + dx, 2 * g.n[0]);
  const int hy = pmod(2 * s.y + basis_comp(g.kind, s.b, 1) + dy, 2 * g.n[1]);
  const int hz = pmod(2 * s.z + basis_comp(g.kind, s.b, 2) + dz, 2 * g.n[2]);
  SiteXYZ r;
  r.x = hx >> 1;
  r.y = hy >> 1;
  r.z = hz >> 1;
  r.b = basis_of_parity(g.kind, hx & 1, hy & 1, hz & 1);
  return r;
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
    const uint32_t axi = tid % ax_n, ayi = (tid / ax_n) % ay_n,
                   azi = tid / (ax_n * ay_n) + static_cast<uint32_t>(a.az0);
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
            const uint32_t i = site_id(g, si);
            if ((k & 1u) == 0) w = philox4x32_10(k >> 1, cid, a.t, 0u, g.seed_lo, g.seed_hi);
            const uint32_t wa = (k & 1u) ? w.z : w.x;
            const uint32_t wb = (k & 1u) ? w.w : w.y;
            const uint32_t dir = mulhi32(wa, static_cast<uint32_t>(g.z1));
            const SiteXYZ sj = neighbour(g, si, sp.v[dir][0], sp.v[dir][1], sp.v[dir][2]);
            const uint32_t j = site_id(g, sj);
            const uint32_t p = occ_get(g, occ, si), q = occ_get(g, occ, sj);
            ++att;
            if (p == q) continue;
            ++unl;
            int64_t de = 0;
            for (int m = 0; m < g.M; ++m) {
              const int64_t* Vm = V + static_cast<int64_t>(m) * K * K;
              for (int t = sp.start[m]; t < sp.start[m + 1]; ++t) {
                const SiteXYZ ki = neighbour(g, si, sp.v[t][0], sp.v[t][1], sp.v[t][2]);
                const uint32_t ik = site_id(g, ki);
                if (ik != i && ik != j) {
                  const uint32_t sk = occ_get(g, occ, ki);
                  de += Vm[q * K + sk] - Vm[p * K + sk];
                }
                const SiteXYZ kj = neighbour(g, sj, sp.v[t][0], sp.v[t][1], sp.v[t][2]);
                const uint32_t jk = site_id(g, kj);
                if (jk != i && jk != j) {
                  const uint32_t sk = occ_get(g, occ, kj);
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
                const uint32_t thr = compose_threshold(
                    s_tab[idx & 511u], s_tab[512 + ((idx >> 9) & 511u)], s_tab[1024 + (idx >> 18)]);
                accept = wb < thr;
              }
            }
            if (accept) {
              occ_set(g, occ, si, q);
              occ_set(g, occ, sj, p);
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
                                                           uint32_t n_cells) {
  extern __shared__ uint32_t s_cnt[];
  const int K = g.K;
  const bool in_smem = K <= 32;
  const int n_cnt = n_shells * K * K;
  if (in_smem)
    for (int c = threadIdx.x; c < n_cnt; c += blockDim.x) s_cnt[c] = 0;
  __syncthreads();
  for (uint32_t cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n_cells;
       cell += gridDim.x * blockDim.x) {
    SiteXYZ s;
    s.x = static_cast<int>(cell % g.n[0]);
    s.y = static_cast<int>((cell / g.n[0]) % g.n[1]);
    s.z = static_cast<int>(cell / (static_cast<uint32_t>(g.n[0]) * g.n[1]));
    for (int b = 0; b < g.nb; ++b) {
      s.b = b;
      const uint32_t pc = occ_get(g, occ, s);
      for (int m = 0; m < n_shells; ++m)
        for (int t = sp.start[m]; t < sp.start[m + 1]; ++t) {
          const SiteXYZ k = neighbour(g, s, sp.v[t][0], sp.v[t][1], sp.v[t][2]);
          const uint32_t p = occ_get(g, occ, k);
          const int slot = (m * K + pc) * K + p;
          if (in_smem)
            atomicAdd(&s_cnt[slot], 1u);
          else
            atomicAdd(&counts[slot], 1ull);
        }
    }
  }
  __syncthreads();
  if (in_smem)
    for (int c = threadIdx.x; c < n_cnt; c += blockDim.x)
      if (s_cnt[c]) atomicAdd(&counts[c], static_cast<unsigned long long>(s_cnt[c]));
}

// Layout conversions.  Canonical row r = z n_y + y holds n_x cells of nb
// bytes; the device row of group grp of that (z, y) starts at
// (grp * n_y n_z + r) * px (dev_row).  Blocks stride over rows and threads
// over x, so there is no per-cell division; one load or store of nb bytes per
// cell on the canonical side, one byte per group on the device side.

// canonical -> device storage (codes sigma * W, or two 4-bit ids per byte);
// writes the row padding [n_x, px) as zeros.  Returns at once when *skip is
// non-zero (the validation of this upload failed).
template <int NB, bool PACK4>
__global__ void k_canon_to_dev(const Geom g, const uint8_t* __restrict__ canon,
                               uint8_t* __restrict__ occ, const unsigned int* __restrict__ skip) {
  if (skip && *skip) return;
  using Cell = typename std::conditional<NB == 2, uint16_t, uint32_t>::type;
  const uint32_t rows = static_cast<uint32_t>(g.n[1]) * g.n[2];
  const int nx = g.n[0], px = g.px;
  const uint32_t W = static_cast<uint32_t>(g.W);
  for (uint32_t r = blockIdx.x; r < rows; r += gridDim.x) {
    const Cell* src = reinterpret_cast<const Cell*>(canon + static_cast<size_t>(r) * nx * NB);
    for (int x = threadIdx.x; x < px; x += blockDim.x) {
      const uint32_t c = x < nx ? static_cast<uint32_t>(src[x]) : 0u;
      if constexpr (!PACK4) {
#pragma unroll
        for (int b = 0; b < NB; ++b)
          occ[(static_cast<size_t>(b) * rows + r) * px + x] =
              static_cast<uint8_t>(((c >> (8 * b)) & 0xFFu) * W);
      } else {
#pragma unroll
        for (int b = 0; b < NB; b += 2)
          occ[(static_cast<size_t>(b >> 1) * rows + r) * px + x] =
              static_cast<uint8_t>(((c >> (8 * b)) & 0x0Fu) | (((c >> (8 * b + 8)) & 0x0Fu) << 4));
      }
    }
  }
}

// device storage -> canonical.  Codes are sigma * W <= 255, so sigma =
// (code * ceil(2^16 / W)) >> 16 exactly (the rounding error is sigma * e / 2^16
// with e < W).
template <int NB, bool PACK4>
__global__ void k_dev_to_canon(const Geom g, const uint8_t* __restrict__ occ,
                               uint8_t* __restrict__ canon) {
  using Cell = typename std::conditional<NB == 2, uint16_t, uint32_t>::type;
  const uint32_t rows = static_cast<uint32_t>(g.n[1]) * g.n[2];
  const int nx = g.n[0], px = g.px;
  const uint32_t inv = (65536u + static_cast<uint32_t>(g.W) - 1u) / static_cast<uint32_t>(g.W);
  for (uint32_t r = blockIdx.x; r < rows; r += gridDim.x) {
    Cell* dst = reinterpret_cast<Cell*>(canon + static_cast<size_t>(r) * nx * NB);
    for (int x = threadIdx.x; x < nx; x += blockDim.x) {
      uint32_t c = 0;
      if constexpr (!PACK4) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const uint32_t code = occ[(static_cast<size_t>(b) * rows + r) * px + x];
          c |= ((code * inv) >> 16) << (8 * b);
        }
      } else {
#pragma unroll
        for (int b = 0; b < NB; b += 2) {
          const uint32_t v = occ[(static_cast<size_t>(b >> 1) * rows + r) * px + x];
          c |= ((v & 0x0Fu) << (8 * b)) | ((v >> 4) << (8 * b + 8));
        }
      }
      dst[x] = static_cast<Cell>(c);
    }
  }
}

// Vector forms for rows of n_x % 4 == 0 (the canonical rows are then
// 4 NB-byte aligned, the device rows are 16-byte aligned): a warp takes a
// row (warps stride over rows), its lanes 4 cells at a time -- one 4 NB-byte
// canonical access, one 4-byte access per device row group -- and the bytes
// are (de)interleaved with byte permutes.  Chunks past n_x are the row
// padding (zeros).

// the 4 cells' byte of basis b from their canonical words (NB = 4: w0..w3;
// NB = 2: lo = cells 0, 1 and hi = cells 2, 3)
__device__ __forceinline__ void split4(const uint4 w, uint32_t (&o)[4]) {
  const uint32_t t01 = __byte_perm(w.x, w.y, 0x5140), t23 = __byte_perm(w.z, w.w, 0x5140);
  const uint32_t u01 = __byte_perm(w.x, w.y, 0x7362), u23 = __byte_perm(w.z, w.w, 0x7362);
  o[0] = __byte_perm(t01, t23, 0x5410);
  o[1] = __byte_perm(t01, t23, 0x7632);
  o[2] = __byte_perm(u01, u23, 0x5410);
  o[3] = __byte_perm(u01, u23, 0x7632);
}

template <int NB, bool PACK4>
__global__ void k_canon_to_dev_v4(const Geom g, const uint8_t* __restrict__ canon,
                                  uint8_t* __restrict__ occ, const unsigned int* __restrict__ skip) {
  if (skip && *skip) return;
  const uint32_t rows = static_cast<uint32_t>(g.n[1]) * g.n[2];
  const uint32_t nxc = static_cast<uint32_t>(g.n[0]) / 4, pxc = static_cast<uint32_t>(g.px) / 4;
  const uint32_t W = static_cast<uint32_t>(g.W);
  const size_t grp_words = static_cast<size_t>(rows) * pxc;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const uint8_t* src_row = canon + static_cast<size_t>(r) * nxc * 4 * NB;
    uint32_t* dst_row = reinterpret_cast<uint32_t*>(occ) + static_cast<size_t>(r) * pxc;
    for (uint32_t c = lane; c < pxc; c += 32) {
      uint32_t o[4] = {0u, 0u, 0u, 0u};  // per basis: the 4 cells' ids
      if (c < nxc) {
        if constexpr (NB == 4) {
          split4(*reinterpret_cast<const uint4*>(src_row + 16 * c), o);
        } else {
          const uint2 v = *reinterpret_cast<const uint2*>(src_row + 8 * c);
          o[0] = __byte_perm(v.x, v.y, 0x6420);
          o[1] = __byte_perm(v.x, v.y, 0x7531);
        }
      }
      if constexpr (!PACK4) {
        // ids * W <= 255: the bytewise products do not carry
#pragma unroll
        for (int b = 0; b < NB; ++b) dst_row[b * grp_words + c] = o[b] * W;
      } else {
#pragma unroll
        for (int b = 0; b < NB; b += 2) dst_row[(b >> 1) * grp_words + c] = o[b] | (o[b + 1] << 4);
      }
    }
  }
}

template <int NB, bool PACK4>
__global__ void k_dev_to_canon_v4(const Geom g, const uint8_t* __restrict__ occ,
                                  uint8_t* __restrict__ canon) {
  const uint32_t rows = static_cast<uint32_t>(g.n[1]) * g.n[2];
  const uint32_t nxc = static_cast<uint32_t>(g.n[0]) / 4, pxc = static_cast<uint32_t>(g.px) / 4;
  const uint32_t W = static_cast<uint32_t>(g.W);
  const uint32_t inv = (65536u + W - 1u) / W;
  const size_t grp_words = static_cast<size_t>(rows) * pxc;
  const uint32_t lane = threadIdx.x & 31u;
  const uint32_t warps = gridDim.x * (blockDim.x >> 5);
  for (uint32_t r = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); r < rows; r += warps) {
    const uint32_t* src_row = reinterpret_cast<const uint32_t*>(occ) + static_cast<size_t>(r) * pxc;
    uint8_t* dst_row = canon + static_cast<size_t>(r) * nxc * 4 * NB;
    for (uint32_t c = lane; c < nxc; c += 32) {
      uint32_t o[4];  // per basis: the 4 cells' ids
      if constexpr (!PACK4) {
#pragma unroll
        for (int b = 0; b < NB; ++b) {
          const uint32_t v = src_row[b * grp_words + c];
          if (W == 8u) {
            o[b] = (v >> 3) & 0x1F1F1F1Fu;
          } else {  // codes are sigma * W <= 255: sigma = (code * ceil(2^16 / W)) >> 16 exactly
            uint32_t w = 0;
#pragma unroll
            for (int e = 0; e < 4; ++e) w |= ((((v >> (8 * e)) & 0xFFu) * inv) >> 16) << (8 * e);
            o[b] = w;
          }
        }
      } else {
#pragma unroll
        for (int b = 0; b < NB; b += 2) {
          const uint32_t v = src_row[(b >> 1) * grp_words + c];
          o[b] = v & 0x0F0F0F0Fu;
          o[b + 1] = (v >> 4) & 0x0F0F0F0Fu;
        }
      }
      if constexpr (NB == 4) {
        // cell k = bytes k of o[0..3]: the transpose split4 is its own inverse
        uint32_t w[4];
        split4(make_uint4(o[0], o[1], o[2], o[3]), w);
        *reinterpret_cast<uint4*>(dst_row + 16 * c) = make_uint4(w[0], w[1], w[2], w[3]);
      } else {
        *reinterpret_cast<uint2*>(dst_row + 8 * c) =
            make_uint2(__byte_perm(o[0], o[1], 0x5140), __byte_perm(o[0], o[1], 0x7362));
      }
    }
  }
}

// flag[0] |= 1 when a canonical byte is >= K: 16 bytes per thread, bytewise
// compare of four bytes per word (__vcmpgeu4); the unaligned head and the
// tail bytewise
__global__ void k_validate(const uint8_t* __restrict__ canon, uint64_t n, uint32_t K,
                           unsigned int* __restrict__ flag) {
  const uint64_t head = (16u - (reinterpret_cast<uintptr_t>(canon) & 15u)) & 15u;
  const uint64_t h = head < n ? head : n;
  const uint64_t n16 = (n - h) / 16;
  const uint4* body = reinterpret_cast<const uint4*>(canon + h);
  const uint32_t k4 = (K > 255u ? 255u : K) * 0x01010101u;
  const uint64_t tid = blockIdx.x * static_cast<uint64_t>(blockDim.x) + threadIdx.x;
  const uint64_t stride = static_cast<uint64_t>(gridDim.x) * blockDim.x;
  uint32_t bad = 0;
  for (uint64_t i = tid; i < n16; i += stride) {
    const uint4 v = body[i];
    bad |= __vcmpgeu4(v.x, k4) | __vcmpgeu4(v.y, k4) | __vcmpgeu4(v.z, k4) | __vcmpgeu4(v.w, k4);
  }
  if (K > 255u) bad = 0;  // every byte is a valid id
  for (uint64_t i = tid; i < h; i += stride) bad |= canon[i] >= K;
  for (uint64_t i = h + 16 * n16 + tid; i < n; i += stride) bad |= canon[i] >= K;
  if (__any_sync(0xffffffffu, bad != 0) && (threadIdx.x & 31) == 0) atomicOr(flag, 1u);
}

static uint32_t grid_for(uint64_t work, int threads, int n_sm) {
  uint64_t b = (work + threads - 1) / threads;
  const uint64_t cap = static_cast<uint64_t>(n_sm > 0 ? n_sm : 148) * 16;
  if (b > cap) b = cap;
  return static_cast<uint32_t>(b < 1 ? 1 : b);
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
  if (a.naz <= 0 || static_cast<uint32_t>(a.az0 + a.naz) > cnt[2]) return cudaErrorInvalidValue;
  const uint32_t n_active = cnt[0] * cnt[1] * static_cast<uint32_t>(a.naz);
  const uint32_t blocks = (n_active + 127) / 128;
  k_sweep_generic<<<blocks, 128, 0, st>>>(g, a, sp, tab, occ, V, stats, n_active, cnt[0], cnt[1]);
  return cudaGetLastError();
}

cudaError_t launch_pair_count_generic(const Geom& g, const ShellParam& sp, int n_shells,
                                      const uint8_t* occ, unsigned long long* counts,
                                      uint32_t n_cells, int n_sm, cudaStream_t st) {
  const int K = g.K;
  const size_t smem = K <= 32 ? sizeof(uint32_t) * n_shells * K * K : 0;
  k_pair_count_generic<<<grid_for(n_cells, 256, n_sm), 256, smem, st>>>(g, sp, n_shells, occ,
                                                                         counts, n_cells);
  return cudaGetLastError();
}

cudaError_t launch_canon_to_dev(const Geom& g, const uint8_t* canon, uint8_t* occ,
                                uint32_t n_cells, int n_sm, cudaStream_t st,
                                const unsigned int* skip) {
  (void)n_cells;
  const uint32_t rows = static_cast<uint32_t>(g.n[1]) * g.n[2];
  if (g.n[0] % 4 == 0) {
    const uint32_t vb = grid_for(rows, 8, n_sm);  // a warp per row
    if (g.nb == 2) {
      if (g.pack4) k_canon_to_dev_v4<2, true><<<vb, 256, 0, st>>>(g, canon, occ, skip);
      else k_canon_to_dev_v4<2, false><<<vb, 256, 0, st>>>(g, canon, occ, skip);
    } else {
      if (g.pack4) k_canon_to_dev_v4<4, true><<<vb, 256, 0, st>>>(g, canon, occ, skip);
      else k_canon_to_dev_v4<4, false><<<vb, 256, 0, st>>>(g, canon, occ, skip);
    }
    return cudaGetLastError();
  }
  const uint32_t blocks = grid_for(rows, 1, n_sm);
  if (g.nb == 2) {
    if (g.pack4) k_canon_to_dev<2, true><<<blocks, 256, 0, st>>>(g, canon, occ, skip);
    else k_canon_to_dev<2, false><<<blocks, 256, 0, st>>>(g, canon, occ, skip);
  } else {
    if (g.pack4) k_canon_to_dev<4, true><<<blocks, 256, 0, st>>>(g, canon, occ, skip);
    else k_canon_to_dev<4, false><<<blocks, 256, 0, st>>>(g, canon, occ, skip);
  }
  return cudaGetLastError();
}

cudaError_t launch_dev_to_canon(const Geom& g, const uint8_t* occ, uint8_t* canon,
                                uint32_t n_cells, int n_sm, cudaStream_t st) {
  (void)n_cells;
  const uint32_t rows = static_cast<uint32_t>(g.n[1]) * g.n[2];
  if (g.n[0] % 4 == 0) {
    const uint32_t vb = grid_for(rows, 8, n_sm);  // a warp per row
    if (g.nb == 2) {
      if (g.pack4) k_dev_to_canon_v4<2, true><<<vb, 256, 0, st>>>(g, occ, canon);
      else k_dev_to_canon_v4<2, false><<<vb, 256, 0, st>>>(g, occ, canon);
    } else {
      if (g.pack4) k_dev_to_canon_v4<4, true><<<vb, 256, 0, st>>>(g, occ, canon);
      else k_dev_to_canon_v4<4, false><<<vb, 256, 0, st>>>(g, occ, canon);
    }
    return cudaGetLastError();
  }
  const uint32_t blocks = grid_for(rows, 1, n_sm);
  if (g.nb == 2) {
    if (g.pack4) k_dev_to_canon<2, true><<<blocks, 256, 0, st>>>(g, occ, canon);
    else k_dev_to_canon<2, false><<<blocks, 256, 0, st>>>(g, occ, canon);
  } else {
    if (g.pack4) k_dev_to_canon<4, true><<<blocks, 256, 0, st>>>(g, occ, canon);
    else k_dev_to_canon<4, false><<<blocks, 256, 0, st>>>(g, occ, canon);
  }
  return cudaGetLastError();
}

cudaError_t launch_validate(const uint8_t* canon, uint64_t n, uint32_t K, unsigned int* flag,
                            int n_sm, cudaStream_t st) {
  k_validate<<<grid_for((n + 15) / 16, 256, n_sm), 256, 0, st>>>(canon, n, K, flag);
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

// ---- local-energy model (the nonlinear short-range model of Sec. 3) ------
//
// One thread per active link cell, trials in the raster order and Philox
// keying of the EPI kernels.  A trial's energy change is the sum over the
// distinct sites k of U (LocalParam::u, displacements from i) of eps_after(k)
// - eps_before(k).  For k = i and k = j every shell is recounted before and
// after the swap (5-bit one-hot fields of a 64-bit word; the swapped sites are
// recognised by their site ids).  Any other k keeps its species, and its
// shell m+1 changes only when exactly one of i, j lies in it (i turns p -> q,
// j turns q -> p; both together cancel): only those shells are scanned, for
// the counts of p and q, and four table entries change.  Integer throughout.

__device__ __forceinline__ uint32_t count_field(uint64_t c, int s) {
  return static_cast<uint32_t>((c >> (5 * s)) & 31u);
}

// neighbour for displacements shorter than the period (|d| < 2 n_d half
// units): one conditional wrap per axis instead of a modulo
__device__ __forceinline__ SiteXYZ neighbour_near(const Geom& g, const SiteXYZ& s, int dx, int dy,
                                                  int dz) {
  int hx = 2 * s.x + basis_comp(g.kind, s.b, 0) + dx;
  int hy = 2 * s.y + basis_comp(g.kind, s.b, 1) + dy;
  int hz = 2 * s.z + basis_comp(g.kind, s.b, 2) + dz;
  hx += hx < 0 ? 2 * g.n[0] : (hx >= 2 * g.n[0] ? -2 * g.n[0] : 0);
  hy += hy < 0 ? 2 * g.n[1] : (hy >= 2 * g.n[1] ? -2 * g.n[1] : 0);
  hz += hz < 0 ? 2 * g.n[2] : (hz >= 2 * g.n[2] ? -2 * g.n[2] : 0);
  SiteXYZ r;
  r.x = hx >> 1;
  r.y = hy >> 1;
  r.z = hz >> 1;
  r.b = basis_of_parity(g.kind, hx & 1, hy & 1, hz & 1);
  return r;
}

// eps_after(k) - eps_before(k) for k = i or j (species cb before, ca after);
// TT: the shared table's type (int32 when every entry fits, else int64)
template <typename TT>
__device__ __forceinline__ int64_t local_eps_change(const Geom& g, const LocalParam& lp,
                                                    const TT* T, const uint8_t* occ,
                                                    const SiteXYZ& sk, uint32_t cb, uint32_t ca,
                                                    uint32_t ii, uint32_t jj, uint32_t p,
                                                    uint32_t q) {
  int64_t de = 0;
  const int K = lp.K, zt = lp.zt;
  for (int m = 0; m < lp.M; ++m) {
    uint64_t nb_b = 0, nb_a = 0;
    for (int t = lp.start[m]; t < lp.start[m + 1]; ++t) {
      const SiteXYZ sn = neighbour_near(g, sk, lp.v[t][0], lp.v[t][1], lp.v[t][2]);
      const uint32_t nn = site_id(g, sn);
      const uint32_t sb = occ_get(g, occ, sn);
      const uint32_t sa = nn == ii ? q : (nn == jj ? p : sb);
      nb_b += 1ull << (5 * sb);
      nb_a += 1ull << (5 * sa);
    }
    const TT* row_b = T + (static_cast<size_t>(m) * K + cb) * K * zt;
    const TT* row_a = T + (static_cast<size_t>(m) * K + ca) * K * zt;
    for (int s = 0; s < K; ++s)
      de += static_cast<int64_t>(row_a[s * zt + count_field(nb_a, s)]) -
            static_cast<int64_t>(row_b[s * zt + count_field(nb_b, s)]);
  }
  return de;
}

// eps change of a site k other than i and j (species c): in each shell m+1
// holding exactly one of them, the counts of p and q move by one
template <typename TT>
__device__ __forceinline__ int64_t local_bystander_change(const Geom& g, const LocalParam& lp,
                                                          const TT* T, const uint8_t* occ,
                                                          const SiteXYZ& sk, uint32_t c,
                                                          uint32_t shells_i, uint32_t shells_j,
                                                          uint32_t p, uint32_t q) {
  int64_t de = 0;
  const int K = lp.K, zt = lp.zt;
  const uint32_t one = shells_i ^ shells_j;
  for (int m = 0; m < lp.M; ++m) {
    if (!((one >> m) & 1u)) continue;
    int np = 0, nq = 0;
    for (int t = lp.start[m]; t < lp.start[m + 1]; ++t) {
      const uint32_t sn = occ_get(g, occ, neighbour_near(g, sk, lp.v[t][0], lp.v[t][1], lp.v[t][2]));
      np += sn == p;
      nq += sn == q;
    }
    const int dp = ((shells_i >> m) & 1u) ? -1 : 1;  // i: p -> q; j: q -> p
    const TT* row = T + (static_cast<size_t>(m) * K + c) * K * zt;
    de += static_cast<int64_t>(row[p * zt + np + dp]) - row[p * zt + np] +
          static_cast<int64_t>(row[q * zt + nq - dp]) - row[q * zt + nq];
  }
  return de;
}

// the part of LocalParam the kernels keep in shared memory: counts, shell
// ranges and shell vectors (the displacement lists of U, their shell masks
// and the item lists are read from global memory, through L1: by the seam
// path and once per block)
constexpr int kLocalParamCopy = (offsetof(LocalParam, u) + 3) / 4 * 4;
constexpr int kLocalParamBytes = (kLocalParamCopy + 15) / 16 * 16;

// Fast path of the local kernel (8-bit storage, a cell whose sites and their
// reads, up to 3 conventional cells away, do not cross the periodic seam):
// every site is a byte address in device storage and a displacement adds a
// fixed delta for a given basis.  Per block: dv[b][t] / bv[b][t] = delta and
// basis reached by shell vector t from a basis-b site, du[b][dir][e] /
// di[b][dir][x] / bi[b][dir][x] the same for the site of item x, and
// im[dir][x] its shell and sign; sized for the lattice's basis count,
// first-shell size and item count (the unified L1 keeps the rest).
__host__ __device__ inline int local_fast_bytes(int nb, int z1, int n_items) {
  return 5 * nb * kLocalMaxV + 5 * nb * z1 * n_items + z1 * n_items;
}

// Order of the cells of one launch: the interior cells (the product of one
// circular run of active cell indices per axis, a_d = (s0_d + i) mod A_d),
// then the seam cells as three slabs, so that a warp's lanes take one path.
// on = 0: plain raster order.
struct LocalSplit {
  int on;
  int A[3], s0[3], I[3];
};

__device__ __forceinline__ void split_cell(const LocalSplit& sp, uint32_t tid, uint32_t* a) {
  const uint32_t A0 = sp.A[0], A1 = sp.A[1], A2 = sp.A[2];
  const uint32_t I0 = sp.I[0], I1 = sp.I[1], I2 = sp.I[2];
  const uint32_t n_int = I0 * I1 * I2;
  uint32_t i0, i1, i2;  // offsets from s0 along each axis
  if (tid < n_int) {
    i0 = tid % I0;
    i1 = (tid / I0) % I1;
    i2 = tid / (I0 * I1);
  } else {
    uint32_t r = tid - n_int;
    const uint32_t S0 = A0 - I0, S1 = A1 - I1;
    if (r < S0 * A1 * A2) {  // x seam: every y, z
      i0 = I0 + r % S0;
      i1 = (r / S0) % A1;
      i2 = r / (S0 * A1);
    } else if ((r -= S0 * A1 * A2) < I0 * S1 * A2) {  // y seam, x interior, every z
      i0 = r % I0;
      i1 = I1 + (r / I0) % S1;
      i2 = r / (I0 * S1);
    } else {  // z seam, x and y interior
      r -= I0 * S1 * A2;
      i0 = r % I0;
      i1 = (r / I0) % I1;
      i2 = I2 + r / (I0 * I1);
    }
  }
  a[0] = (sp.s0[0] + i0) % A0;
  a[1] = (sp.s0[1] + i1) % A1;
  a[2] = (sp.s0[2] + i2) % A2;
}

__device__ __forceinline__ int fast_delta(const Geom& g, int b, int dx, int dy, int dz, int* bn) {
  const int hx = basis_comp(g.kind, b, 0) + dx, hy = basis_comp(g.kind, b, 1) + dy,
            hz = basis_comp(g.kind, b, 2) + dz;
  *bn = basis_of_parity(g.kind, hx & 1, hy & 1, hz & 1);
  const int plane = g.n[1] * g.px;
  return (*bn - b) * (g.n[2] * plane) + (hz >> 1) * plane + (hy >> 1) * g.px + (hx >> 1);
}

template <typename TT>
__device__ void load_local(unsigned char* smem, const LocalParam* lp_g, const int64_t* T_g,
                           int n_T) {
  const uint32_t* src = reinterpret_cast<const uint32_t*>(lp_g);
  uint32_t* dst = reinterpret_cast<uint32_t*>(smem);
  for (int w = threadIdx.x; w < kLocalParamCopy / 4; w += blockDim.x) dst[w] = src[w];
  TT* t = reinterpret_cast<TT*>(smem + kLocalParamBytes);
  for (int w = threadIdx.x; w < n_T; w += blockDim.x) t[w] = static_cast<TT>(T_g[w]);
}

template <typename TT>
__global__ void __launch_bounds__(128, 6) k_sweep_local(const __grid_constant__ Geom g,
                                                    const PhaseArgs a,
                                                    const __grid_constant__ Tables tab,
                                                    uint8_t* __restrict__ occ,
                                                    const LocalParam* __restrict__ lp_g,
                                                    const int64_t* __restrict__ T_g, int n_T,
                                                    unsigned long long* __restrict__ stats,
                                                    uint32_t n_active, uint32_t ax_n,
                                                    uint32_t ay_n, const LocalSplit split) {
  extern __shared__ __align__(16) unsigned char smem[];
  load_local<TT>(smem, lp_g, T_g, n_T);
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem + kLocalParamBytes +
                                                (sizeof(TT) * n_T + 15) / 16 * 16);
  for (int w = threadIdx.x; w < kTabWords; w += blockDim.x) s_tab[w] = tab.w[w];
  const int n_items = lp_g->n_items;
  int* dv = reinterpret_cast<int*>(s_tab + kTabWords);
  int* di = dv + g.nb * kLocalMaxV;
  uint8_t* bv = reinterpret_cast<uint8_t*>(di + g.nb * g.z1 * n_items);
  uint8_t* bi = bv + g.nb * kLocalMaxV;
  uint8_t* im = bi + g.nb * g.z1 * n_items;
  // the fast path needs 8-bit storage and byte addresses (hence deltas) that
  // fit int32
  const bool fast_ok = !g.pack4 && static_cast<int64_t>(g.nb) * g.n[2] * g.n[1] * g.px < (1ll << 31);
  __syncthreads();
  const LocalParam& lp = *reinterpret_cast<const LocalParam*>(smem);
  const TT* T = reinterpret_cast<const TT*>(smem + kLocalParamBytes);
  if (fast_ok) {
    for (int w = threadIdx.x; w < g.nb * lp.total; w += blockDim.x) {
      const int b = w / lp.total, t = w % lp.total;
      int bn;
      dv[b * kLocalMaxV + t] = fast_delta(g, b, lp.v[t][0], lp.v[t][1], lp.v[t][2], &bn);
      bv[b * kLocalMaxV + t] = static_cast<uint8_t>(bn);
    }
    const int n_dir = g.z1 * n_items;
    for (int w = threadIdx.x; w < g.nb * n_dir; w += blockDim.x) {
      const int b = w / n_dir, r = w % n_dir, dir = r / n_items, x = r % n_items;
      const int e = lp_g->item_e[dir][x];
      int bn;
      di[w] = fast_delta(g, b, lp_g->u[dir][e][0], lp_g->u[dir][e][1], lp_g->u[dir][e][2], &bn);
      bi[w] = static_cast<uint8_t>(bn);
      if (b == 0) im[r] = lp_g->item_m[dir][x];
    }
  }
  __syncthreads();
  // species of a stored code sigma * W: exact multiply-shift
  const uint32_t invW = (65536u + static_cast<uint32_t>(g.W) - 1u) / static_cast<uint32_t>(g.W);
  const int K = lp.K, zt = lp.zt;

  uint64_t att = 0, unl = 0, acc = 0;
  int64_t sum_de = 0;
  const uint32_t tid = blockIdx.x * blockDim.x + threadIdx.x;
  if (tid < n_active) {
    uint32_t axi, ayi, azi;
    if (split.on) {
      uint32_t av[3];
      split_cell(split, tid, av);
      axi = av[0];
      ayi = av[1];
      azi = av[2] + static_cast<uint32_t>(a.az0);
    } else {
      axi = tid % ax_n;
      ayi = (tid / ax_n) % ay_n;
      azi = tid / (ax_n * ay_n) + static_cast<uint32_t>(a.az0);
    }
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
    // every site of the cell and every site its trials read, within 3
    // conventional cells, stays clear of the periodic seam
    bool fast = fast_ok;
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      const int x0 = pmod(lo[d] + a.shift[d], g.n[d]);
      fast = fast && x0 >= 3 && x0 + (hi[d] - lo[d]) + 3 <= g.n[d];
    }
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
            if ((k & 1u) == 0) w = philox4x32_10(k >> 1, cid, a.t, 0u, g.seed_lo, g.seed_hi);
            const uint32_t wa = (k & 1u) ? w.z : w.x;
            const uint32_t wb = (k & 1u) ? w.w : w.y;
            const uint32_t dir = __umulhi(wa, static_cast<uint32_t>(g.z1));
            if (fast) {
              ++att;
              const int ai = static_cast<int>(dev_row(g, b, si.z, si.y)) + si.x;
              const int aj = ai + dv[b * kLocalMaxV + dir];
              const int bj = bv[b * kLocalMaxV + dir];
              const uint32_t cp = occ[ai], cq = occ[aj];
              if (cp == cq) continue;
              ++unl;
              const uint32_t p = (cp * invW) >> 16, q = (cq * invW) >> 16;
              int64_t de = 0;
              // i and j: every shell recounted before and after
              auto full = [&](int ak, int bk, uint32_t cb, uint32_t ca) {
                for (int m = 0; m < lp.M; ++m) {
                  uint64_t nb_b = 0, nb_a = 0;
                  for (int t = lp.start[m]; t < lp.start[m + 1]; ++t) {
                    const int an = ak + dv[bk * kLocalMaxV + t];
                    const uint32_t sb = (occ[an] * invW) >> 16;
                    const uint32_t sa = an == ai ? q : (an == aj ? p : sb);
                    nb_b += 1ull << (5 * sb);
                    nb_a += 1ull << (5 * sa);
                  }
                  const TT* row_b = T + (static_cast<size_t>(m) * K + cb) * K * zt;
                  const TT* row_a = T + (static_cast<size_t>(m) * K + ca) * K * zt;
                  for (int s = 0; s < K; ++s)
                    de += static_cast<int64_t>(row_a[s * zt + count_field(nb_a, s)]) -
                          static_cast<int64_t>(row_b[s * zt + count_field(nb_b, s)]);
                }
              };
              full(ai, b, p, q);
              full(aj, bj, q, p);
              // bystanders: item x scans the same shell for every lane
              const int ib = (b * g.z1 + static_cast<int>(dir)) * n_items;
              const uint8_t* imd = im + static_cast<int>(dir) * n_items;
              for (int x = 0; x < n_items; ++x) {
                const int ak = ai + di[ib + x], bk = bi[ib + x];
                const int m = imd[x] & 3;
                const int dp = (imd[x] >> 2) ? 1 : -1;  // i: p -> q; j: q -> p
                const uint32_t c = (occ[ak] * invW) >> 16;
                int np = 0, nq = 0;
                for (int t = lp.start[m]; t < lp.start[m + 1]; ++t) {
                  const uint32_t sn = occ[ak + dv[bk * kLocalMaxV + t]];
                  np += sn == cp;
                  nq += sn == cq;
                }
                const TT* row = T + (static_cast<size_t>(m) * K + c) * K * zt;
                de += static_cast<int64_t>(row[p * zt + np + dp]) - row[p * zt + np] +
                      static_cast<int64_t>(row[q * zt + nq - dp]) - row[q * zt + nq];
              }
              bool accept;
              if (de <= 0 || a.mode == kModeAcceptAll) {
                accept = true;
              } else if (a.mode == kModeZeroT) {
                accept = false;
              } else {
                const uint64_t idx = static_cast<uint64_t>(de) >> a.s;
                accept = idx < (1ull << 27) &&
                         wb < compose_threshold(s_tab[idx & 511u], s_tab[512 + ((idx >> 9) & 511u)],
                                                s_tab[1024 + (idx >> 18)]);
              }
              if (accept) {
                occ[ai] = static_cast<uint8_t>(cq);
                occ[aj] = static_cast<uint8_t>(cp);
                ++acc;
                sum_de += de;
              }
              continue;
            }
            const SiteXYZ sj = neighbour_near(g, si, lp.v[dir][0], lp.v[dir][1], lp.v[dir][2]);
            const uint32_t p = occ_get(g, occ, si), q = occ_get(g, occ, sj);
            ++att;
            if (p == q) continue;
            ++unl;
            const uint32_t ii = site_id(g, si), jj = site_id(g, sj);
            int64_t de = 0;
            de += local_eps_change(g, lp, T, occ, si, p, q, ii, jj, p, q) +
                  local_eps_change(g, lp, T, occ, sj, q, p, ii, jj, p, q);
            for (int e = 2; e < lp.n_u[dir]; ++e) {
              const uint32_t mi = lp_g->shells_i[dir][e], mj = lp_g->shells_j[dir][e];
              if (mi == mj) continue;  // no shell holds exactly one of i, j
              const SiteXYZ sk = neighbour_near(g, si, lp_g->u[dir][e][0], lp_g->u[dir][e][1],
                                                lp_g->u[dir][e][2]);
              de += local_bystander_change(g, lp, T, occ, sk, occ_get(g, occ, sk), mi, mj, p, q);
            }
            bool accept;
            if (de <= 0 || a.mode == kModeAcceptAll) {
              accept = true;
            } else if (a.mode == kModeZeroT) {
              accept = false;
            } else {
              const uint64_t idx = static_cast<uint64_t>(de) >> a.s;
              accept = idx < (1ull << 27) &&
                       wb < compose_threshold(s_tab[idx & 511u], s_tab[512 + ((idx >> 9) & 511u)],
                                              s_tab[1024 + (idx >> 18)]);
            }
            if (accept) {
              occ_set(g, occ, si, q);
              occ_set(g, occ, sj, p);
              ++acc;
              sum_de += de;
            }
          }
  }
  warp_reduce_add_stats(stats, att, unl, acc, sum_de);
}

// Total local energy: per-block int64 partial sums (the host adds them in
// int128); one thread per conventional cell, grid-stride
__global__ void __launch_bounds__(256) k_local_energy(const Geom g,
                                                      const LocalParam* __restrict__ lp_g,
                                                      const int64_t* __restrict__ T_g, int n_T,
                                                      const uint8_t* __restrict__ occ,
                                                      long long* __restrict__ partial,
                                                      uint32_t n_cells) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ long long s_red[8];
  load_local<int64_t>(smem, lp_g, T_g, n_T);
  __syncthreads();
  const LocalParam& lp = *reinterpret_cast<const LocalParam*>(smem);
  const int64_t* T = reinterpret_cast<const int64_t*>(smem + kLocalParamBytes);
  const int K = lp.K, zt = lp.zt;
  long long e = 0;
  for (uint32_t cell = blockIdx.x * blockDim.x + threadIdx.x; cell < n_cells;
       cell += gridDim.x * blockDim.x) {
    SiteXYZ s;
    s.x = static_cast<int>(cell % g.n[0]);
    s.y = static_cast<int>((cell / g.n[0]) % g.n[1]);
    s.z = static_cast<int>(cell / (static_cast<uint32_t>(g.n[0]) * g.n[1]));
    for (int b = 0; b < g.nb; ++b) {
      s.b = b;
      const uint32_t c = occ_get(g, occ, s);
      for (int m = 0; m < lp.M; ++m) {
        uint64_t nb = 0;
        for (int t = lp.start[m]; t < lp.start[m + 1]; ++t)
          nb += 1ull << (5 * occ_get(g, occ, neighbour(g, s, lp.v[t][0], lp.v[t][1], lp.v[t][2])));
        const int64_t* row = T + (static_cast<size_t>(m) * K + c) * K * zt;
        for (int sp = 0; sp < K; ++sp) e += row[sp * zt + count_field(nb, sp)];
      }
    }
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) e += __shfl_down_sync(0xffffffffu, e, o);
  if ((threadIdx.x & 31) == 0) s_red[threadIdx.x >> 5] = e;
  __syncthreads();
  if (threadIdx.x == 0) {
    long long t = 0;
    for (int w = 0; w < static_cast<int>(blockDim.x >> 5); ++w) t += s_red[w];
    partial[blockIdx.x] = t;
  }
}

size_t local_smem_bytes(int n_T, size_t entry = 8) {
  return kLocalParamBytes + (entry * static_cast<size_t>(n_T) + 15) / 16 * 16;
}

cudaError_t launch_sweep_local(const Geom& g, const PhaseArgs& a, const Tables& tab,
                               uint8_t* occ, const LocalParam* lp, const int64_t* T, int n_T,
                               bool t32, int n_items, unsigned long long* stats, cudaStream_t st) {
  uint32_t cnt[2];
  for (int d = 0; d < 2; ++d) {
    if (g.m[d] == 1 && ((a.colour >> d) & 1)) return cudaSuccess;
    cnt[d] = g.m[d] == 1 ? 1u : static_cast<uint32_t>(g.m[d] / 2);
  }
  if (a.naz <= 0) return cudaErrorInvalidValue;
  const uint32_t n_active = cnt[0] * cnt[1] * static_cast<uint32_t>(a.naz);
  const size_t smem = local_smem_bytes(n_T, t32 ? 4 : 8) + 4 * kTabWords +
                      local_fast_bytes(g.nb, g.z1, n_items);
  auto kern = t32 ? k_sweep_local<int32_t> : k_sweep_local<int64_t>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  // interior cells first (a cell is interior when its sites and their reads,
  // 3 conventional cells either way, stay clear of the periodic seam); the
  // interior indices along each axis must form one circular run, else the
  // plain order is kept (the kernel checks every cell itself either way)
  LocalSplit sp{};
  sp.on = !g.pack4 && static_cast<int64_t>(g.nb) * g.n[2] * g.n[1] * g.px < (1ll << 31);
  const int Ad[3] = {static_cast<int>(cnt[0]), static_cast<int>(cnt[1]), a.naz};
  for (int d = 0; d < 3 && sp.on; ++d) {
    const int A = Ad[d], bit = (a.colour >> d) & 1;
    std::vector<char> in(A);
    int n_in = 0;
    for (int i = 0; i < A; ++i) {
      const int ai = d == 2 ? a.az0 + i : i;
      const int c = g.m[d] == 1 ? 0 : 2 * ai + bit;
      const int lo = static_cast<int>((static_cast<int64_t>(c) * g.n[d]) / g.m[d]);
      const int hi = static_cast<int>((static_cast<int64_t>(c + 1) * g.n[d]) / g.m[d]);
      int x0 = (lo + a.shift[d]) % g.n[d];
      x0 += x0 < 0 ? g.n[d] : 0;
      in[i] = x0 >= 3 && x0 + (hi - lo) + 3 <= g.n[d];
      n_in += in[i];
    }
    int s0 = 0;
    if (n_in > 0 && n_in < A)
      for (int i = 0; i < A; ++i)
        if (in[i] && !in[(i + A - 1) % A]) s0 = i;
    int run = 0;
    while (run < n_in && in[(s0 + run) % A]) ++run;
    if (run != n_in) sp.on = 0;
    sp.A[d] = A;
    sp.s0[d] = s0;
    sp.I[d] = n_in;
  }
  kern<<<(n_active + 127) / 128, 128, smem, st>>>(g, a, tab, occ, lp, T, n_T, stats, n_active,
                                                 cnt[0], cnt[1], sp);
  return cudaGetLastError();
}

cudaError_t launch_local_energy(const Geom& g, const LocalParam* lp, const int64_t* T, int n_T,
                                const uint8_t* occ, long long* partial, int n_blocks,
                                cudaStream_t st) {
  const size_t smem = local_smem_bytes(n_T);
  cudaError_t e = cudaFuncSetAttribute(k_local_energy, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const uint32_t n_cells = static_cast<uint32_t>(g.n[0]) * g.n[1] * g.n[2];
  k_local_energy<<<n_blocks, 256, smem, st>>>(g, lp, T, n_T, occ, partial, n_cells);
  return cudaGetLastError();
}

}  // namespace smcx
