// kernels_pair.cuh -- tiled directed shell pair counts (Warren-Cowley SRO,
// Sec. 3.2, Eq. 9, and the EPI energy, Sec. 3).
//
// H_m[p'][p] = #{(i, d): d in S_m+, sigma_i = p', sigma_{i+d} = p} over the
// lexicographically positive half S_m+ of every shell; the directed counts
// over the whole shell are N_m = H_m + H_m^T (substitute i -> i - d), which
// the host forms.  A persistent grid walks boxes of 64 x 8 x 8 conventional
// cells; each box plus its halo (+2 cells in x, +-2 in y and z: half-shell
// vectors never point to smaller x) is staged into shared memory with
// asynchronous 8-byte copies, the next box prefetched while one is counted.  One thread per x column sums, for each site and shell, a one-hot
// 64-bit word over the neighbour species (FW-bit fields), masked into the
// row of the centre's species; the fields are warp-reduced and added to
// shared counters once per box (twice for FCC with 10-bit fields).
#pragma once

#include <utility>

#include "device_util.cuh"
#include "kernels.h"
#include "kernels_tiled.cuh"

namespace smcx {
namespace pairs {

using tiled::floordiv2;
using tiled::round_up;

__host__ __device__ constexpr bool lex_pos(ShellVec v) {
  return v.x > 0 || (v.x == 0 && (v.y > 0 || (v.y == 0 && v.z > 0)));
}

// index of the k-th positive vector of shell m (compile-time)
__host__ __device__ constexpr int pos_vec(int kind, int m, int k) {
  const int s = shell_start(kind, m);
  for (int i = 0; i < shell_z(kind, m); ++i)
    if (lex_pos(shell_vec(kind, s + i))) {
      if (k == 0) return s + i;
      --k;
    }
  return -1;
}

template <int KIND_, int M_, int KMAX_, bool PACK4_>
struct PCfg {
  static constexpr int KIND = KIND_, M = M_, KMAX = KMAX_;
  static constexpr bool PACK4 = PACK4_;
  static constexpr int NB = KIND == 0 ? 2 : 4;
  static constexpr int BXC = 64, BYC = 8, BZC = 8;  // box of conventional cells
  static constexpr int HX = 2, HYZ = 2;             // halo: x on the + side only
  static constexpr int TX = BXC + HX, TY = BYC + 2 * HYZ, TZ = BZC + 2 * HYZ;
  static constexpr int XW = round_up(TX, 8);
  static constexpr int RS = NB * XW;
  static constexpr int PS = RS * TY;
  static constexpr int TILE = PS * TZ;
  static constexpr int W = KMAX <= 5 ? 8 : 5;       // tile code = sigma * W
  static constexpr int FW = W == 8 ? 12 : 2 * W;    // accumulator field width (FW sigma = shift)
  static constexpr int NT = 128;
  static constexpr int G = PACK4 ? NB / 2 : NB;
  static constexpr int NCNT = M * KMAX * KMAX;
};

template <class C>
__host__ __device__ constexpr int poff(int b, int v) {
  const ShellVec d = shell_vec(C::KIND, v);
  const int bx = basis_comp(C::KIND, b, 0), by = basis_comp(C::KIND, b, 1),
            bz = basis_comp(C::KIND, b, 2);
  const int bp = basis_of_parity(C::KIND, (bx + d.x) & 1, (by + d.y) & 1, (bz + d.z) & 1);
  return floordiv2(bx + d.x) + floordiv2(by + d.y) * C::RS + floordiv2(bz + d.z) * C::PS +
         (bp - b) * C::XW;
}

// bit position FW sigma of the field of the species with tile code c = W sigma
template <class C>
__device__ __forceinline__ uint32_t field_shift(uint32_t c) {
  if constexpr (C::W == 8) return c + (c >> 1);
  else return 2u * c;
}

template <class C, int B, int Mm, int... I>
__device__ __forceinline__ unsigned long long half_shell(const uint8_t* base,
                                                         std::integer_sequence<int, I...>) {
  return (0ull + ... + (1ull << field_shift<C>(base[poff<C>(B, pos_vec(C::KIND, Mm, I))])));
}

template <class C, int B, int... Ms>
__device__ __forceinline__ void all_shells(const uint8_t* base, unsigned long long* acc,
                                           std::integer_sequence<int, Ms...>) {
  ((acc[Ms] = half_shell<C, B, Ms>(base, std::make_integer_sequence<int, shell_z(C::KIND, Ms) / 2>{})),
   ...);
}

__device__ __forceinline__ int pwrap(int v, int n) {
  if (v < 0) v += n;
  if (v >= n) v -= n;
  if (v < 0 || v >= n) v = ((v % n) + n) % n;  // lattices thinner than the halo
  return v;
}

template <class C>
__global__ void __launch_bounds__(C::NT) k_pair_count_tiled(const __grid_constant__ Geom g,
                                                            const uint8_t* __restrict__ occ,
                                                            unsigned long long* __restrict__ hcnt) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* s_cnt = reinterpret_cast<uint32_t*>(smem);
  uint8_t* tiles = smem + round_up(4 * C::NCNT, 16);  // two box buffers of C::TILE bytes
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = C::NT / 32;
  for (int i = tid; i < C::NCNT; i += C::NT) s_cnt[i] = 0;

  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const int nbx = (nx + C::BXC - 1) / C::BXC;
  const int nby = (ny + C::BYC - 1) / C::BYC;
  const int nbz = (nz + C::BZC - 1) / C::BZC;
  const int n_boxes = nbx * nby * nbz;
  const int xl = tid % C::BXC;  // this thread's x column inside the box
  const int rg = tid / C::BXC;  // 0 or 1: row parity
  const size_t px = static_cast<size_t>(g.px);

  // stage box `box` into buffer `buf`: x in [x0, x0 + ex), y in [y0 - 2, y0 + 10),
  // z in [z0 - 2, z0 + 10); 8-bit storage without an x seam goes through
  // cp.async (completes later), everything else is copied synchronously
  auto stage = [&](int box, uint8_t* tile) {
    const int x0 = (box % nbx) * C::BXC;
    const int y0 = ((box / nbx) % nby) * C::BYC;
    const int z0 = (box / (nbx * nby)) * C::BZC;
    const int ex = min(C::TX, nx - x0 + C::HX);
    constexpr int n_sub = C::TY * C::TZ * C::G;
    if (x0 + ex <= nx) {
      const int n8 = (ex + 7) >> 3;
      const int rpi = 32 / n8;
      const int my_r = lane / n8, my_c = lane - (lane / n8) * n8;
      const uint8_t* src0 = occ + x0 + 8 * my_c;
      for (int base = warp * rpi; base < n_sub; base += NW * rpi) {
        const int sub = base + my_r;
        if (my_r < rpi && sub < n_sub) {
          const int grp = sub % C::G;
          const int t = sub / C::G;
          const int ty = t % C::TY, tz = t / C::TY;
          const int gy = pwrap(y0 - C::HYZ + ty, ny), gz = pwrap(z0 - C::HYZ + tz, nz);
          const uint8_t* src = src0 + ((static_cast<size_t>(grp) * nz + gz) * ny + gy) * px;
          uint8_t* row = tile + tz * C::PS + ty * C::RS + 8 * my_c;
          if constexpr (!C::PACK4) {
            const uint32_t dst = static_cast<uint32_t>(__cvta_generic_to_shared(row + grp * C::XW));
            asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst), "l"(src) : "memory");
          } else {
            const uint2 v = *reinterpret_cast<const uint2*>(src);
            *reinterpret_cast<uint2*>(row + 2 * grp * C::XW) =
                make_uint2((v.x & 0x0F0F0F0Fu) * C::W, (v.y & 0x0F0F0F0Fu) * C::W);
            *reinterpret_cast<uint2*>(row + (2 * grp + 1) * C::XW) =
                make_uint2(((v.x >> 4) & 0x0F0F0F0Fu) * C::W, ((v.y >> 4) & 0x0F0F0F0Fu) * C::W);
          }
        }
      }
    } else {
      for (int sub = warp; sub < n_sub; sub += NW) {
        const int grp = sub % C::G;
        const int t = sub / C::G;
        const int ty = t % C::TY, tz = t / C::TY;
        const int gy = pwrap(y0 - C::HYZ + ty, ny), gz = pwrap(z0 - C::HYZ + tz, nz);
        const uint8_t* src = occ + ((static_cast<size_t>(grp) * nz + gz) * ny + gy) * px;
        uint8_t* row = tile + tz * C::PS + ty * C::RS;
        for (int tx = lane; tx < ex; tx += 32) {
          const uint8_t v = src[pwrap(x0 + tx, nx)];
          if constexpr (!C::PACK4) {
            row[grp * C::XW + tx] = v;
          } else {
            row[2 * grp * C::XW + tx] = static_cast<uint8_t>((v & 15) * C::W);
            row[(2 * grp + 1) * C::XW + tx] = static_cast<uint8_t>((v >> 4) * C::W);
          }
        }
      }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
  };

  int buf = 0;
  if (static_cast<int>(blockIdx.x) < n_boxes) stage(blockIdx.x, tiles);
  for (int box = blockIdx.x; box < n_boxes; box += gridDim.x, buf ^= 1) {
    const int next = box + gridDim.x;
    if (next < n_boxes) {
      stage(next, tiles + (buf ^ 1) * C::TILE);  // prefetch while this box is counted
      asm volatile("cp.async.wait_group 1;\n" ::: "memory");
    } else {
      asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    }
    __syncthreads();
    const uint8_t* tile = tiles + buf * C::TILE;
    const int x0 = (box % nbx) * C::BXC;
    const int y0 = ((box / nbx) % nby) * C::BYC;
    const int z0 = (box / (nbx * nby)) * C::BZC;
    // ---- count
    unsigned long long R[C::KMAX][C::M];
    auto clear = [&]() {
#pragma unroll
      for (int p = 0; p < C::KMAX; ++p)
#pragma unroll
        for (int m = 0; m < C::M; ++m) R[p][m] = 0;
    };
    // warp-reduce every field (REDUX) and add it to the block's counters
    auto flush = [&]() {
#pragma unroll
      for (int p = 0; p < C::KMAX; ++p)
#pragma unroll
        for (int m = 0; m < C::M; ++m)
#pragma unroll
          for (int s = 0; s < C::KMAX; ++s) {
            const uint32_t c =
                static_cast<uint32_t>(R[p][m] >> (C::FW * s)) & ((1u << C::FW) - 1u);
            const uint32_t t = __reduce_add_sync(0xffffffffu, c);
            if ((tid & 31) == 0 && t) atomicAdd(&s_cnt[(m * C::KMAX + p) * C::KMAX + s], t);
          }
      clear();
    };
    clear();
    const bool x_in = x0 + xl < g.n[0];
    auto rows = [&](auto bconst) {
      constexpr int B = decltype(bconst)::value;
      if (!x_in) return;
      for (int r = rg; r < C::BYC * C::BZC; r += 2) {
        const int yl = r % C::BYC, zl = r / C::BYC;
        if (y0 + yl >= g.n[1] || z0 + zl >= g.n[2]) continue;
        const uint8_t* base =
            tile + (zl + C::HYZ) * C::PS + (yl + C::HYZ) * C::RS + B * C::XW + xl;
        unsigned long long acc[C::M];
        all_shells<C, B>(base, acc, std::make_integer_sequence<int, C::M>{});
        const uint32_t centre = *base;
#pragma unroll
        for (int p = 0; p < C::KMAX; ++p) {
          if (centre == static_cast<uint32_t>(p * C::W)) {  // one row: predicated adds
#pragma unroll
            for (int m = 0; m < C::M; ++m) R[p][m] += acc[m];
          }
        }
      }
    };
    // fields hold <= 32 rows x (z_m/2 <= 12) = 384 per basis pass: two passes
    // fit 10-bit fields, four fit 12-bit fields
    rows(std::integral_constant<int, 0>{});
    rows(std::integral_constant<int, 1>{});
    if constexpr (C::NB == 4) {
      if constexpr (C::FW < 12) flush();
      rows(std::integral_constant<int, 2>{});
      rows(std::integral_constant<int, 3>{});
    }
    flush();
    __syncthreads();  // the next prefetch reuses this buffer
  }
  __syncthreads();
  for (int i = tid; i < C::NCNT; i += C::NT)
    if (s_cnt[i]) atomicAdd(&hcnt[i], static_cast<unsigned long long>(s_cnt[i]));
}

template <class C>
bool p_supported(const Geom& g) {
  if (g.kind != C::KIND || g.pack4 != (C::PACK4 ? 1 : 0)) return false;
  // the kernel only reads the tile, so a small lattice whose halo holds
  // periodic copies of its own sites is counted correctly as well
  return g.K <= 6 && (g.K == 6) == (C::KMAX == 6);
}

template <class C>
cudaError_t p_launch(const Geom& g, const uint8_t* occ, unsigned long long* hcnt, int n_sm,
                     cudaStream_t st) {
  const size_t smem = round_up(4 * C::NCNT, 16) + 2 * C::TILE;
  cudaError_t e = cudaFuncSetAttribute(k_pair_count_tiled<C>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const int boxes = ((g.n[0] + C::BXC - 1) / C::BXC) * ((g.n[1] + C::BYC - 1) / C::BYC) *
                    ((g.n[2] + C::BZC - 1) / C::BZC);
  int grid = n_sm * 8;
  if (grid > boxes) grid = boxes;
  k_pair_count_tiled<C><<<grid, C::NT, smem, st>>>(g, occ, hcnt);
  return cudaGetLastError();
}

}  // namespace pairs
}  // namespace smcx
