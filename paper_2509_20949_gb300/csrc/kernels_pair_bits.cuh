// kernels_pair_bits.cuh -- bit-sliced directed shell pair counts
// (Warren-Cowley SRO, Sec. 3.2, Eq. 9, and the EPI energy, Sec. 3) for
// 8-bit storage.
//
// Output: rows of KMAX species per shell holding an upper-triangular U_m
// with U_m + U_m^T = N_m, the full-shell directed counts N_m[p'][p] = #{(i,
// d): d in S_m, sigma_i = p', sigma_{i+d} = p}, which is all the callers use
// (they form H + H^T of the tiled kernel's half-shell counts H, and N of a
// symmetric count is U + U^T as well).
//
// Counting by bit masks.  A warp turns 128 consecutive sites of a lattice
// row (a span) into one 32-bit mask per species and byte lane: lane i loads
// sites 128 s + 4 i .. + 3, and ballot j (byte j of every lane) is bit plane
// j of the span, bit i <-> site 128 s + 4 i + j.  The site one further in x
// is then plane j + 1 of the same bit, or, from plane 3, plane 0 of the next
// bit (a one-bit funnel shift across spans), so a half-shell neighbour's
// masks are plane re-indexing plus at most one shift.  Over the half shell
// S_m+ (the other half is the same bonds seen from the far end), for p < q
// < KMAX - 1, N_m[p][q] = N_m[q][p] = sum of popc((c_p & n_q) | (c_q & n_p))
// (centre masks c, neighbour masks n; c_p and c_q are disjoint) over
// planes, spans and vectors, stored as U[p][q]; U[p][p] = N_m[p][p] / 2 =
// sum of popc(c_p & n_p).  The last species' entries follow from the
// species counts: every site has z_m shell-m neighbours, so row p of N_m
// sums to c_p z_m -- a one-thread kernel fills them in.  A block owns boxes
// of whole x rows by BY x BZ rows (persistent grid); the masks of the box
// plus a halo of H rows in y and z (periodic) sit in shared memory.
#pragma once

#include <utility>

#include "device_util.cuh"
#include "kernels.h"
#include "kernels_pair.cuh"

namespace smcx {
namespace pbits {

using tiled::floordiv2;

template <int KIND_, int M_, int KMAX_>
struct BCfg {
  static constexpr int KIND = KIND_, M = M_, KMAX = KMAX_;
  static constexpr int NB = KIND == 0 ? 2 : 4;
  static constexpr int NQ = KMAX - 1;            // masks of species 0 .. KMAX - 2
  static constexpr int NQC = NQ <= 4 ? 1 : 2;    // 16-byte chunks of masks per span and plane
  static constexpr int W = KMAX <= 5 ? 8 : 5;    // storage code = sigma * W
  static constexpr int H = (KIND == 0 && M == 4) ? 2 : 1;  // halo rows; x offsets 0..H
  static constexpr int SW = 16 * NQC;            // words per span: 4 planes x NQC chunks
  static constexpr int NT = 256;
  static constexpr int NCNT = M * NQ * NQ;
};

// runtime box geometry.  Staged masks are plane-major: the 16-byte chunk
// (4 species masks) of plane j, chunk h, staged row r, span s is chunk
// ((j * NQC + h) * NROWS + r) * NS + s, so the threads of a warp, which take
// consecutive spans, read consecutive chunks (no bank conflicts).
struct BoxGeom {
  int BY, BZ, TY, TZ;  // box rows and rows with halo
  int NS, NSC;         // spans per staged row (ceil((nx + H) / 128)), centre spans
  int nby, nbz, n_boxes;  // boxes along y and z; box k = (y box k / nbz, z box k % nbz)
  int hstride;         // words between chunks h and h + 1 (NROWS * NS * 4)
  int pstride;         // words between planes (NQC * hstride)
  unsigned long long n_sites;
};

// half-shell neighbour V (shell table index) of a basis-B site: neighbour
// basis and conventional offsets (ox >= 0: the vector is lexicographically
// positive)
template <class C, int B, int V>
struct BNbr {
  static constexpr ShellVec v = shell_vec(C::KIND, V);
  static constexpr int bx = basis_comp(C::KIND, B, 0), by = basis_comp(C::KIND, B, 1),
                       bz = basis_comp(C::KIND, B, 2);
  static constexpr int bp = basis_of_parity(C::KIND, (bx + v.x) & 1, (by + v.y) & 1, (bz + v.z) & 1);
  static constexpr int ox = floordiv2(bx + v.x), oy = floordiv2(by + v.y), oz = floordiv2(bz + v.z);
  static_assert(ox >= 0 && ox <= C::H && oy >= -C::H && oy <= C::H && oz >= -C::H && oz <= C::H,
                "half-shell offset outside the staged halo");
};

__device__ __forceinline__ int pmod(int v, int n) {
  v %= n;
  return v < 0 ? v + n : v;
}

// masks of species 0 .. NQ-1 of plane j of the span at chunk index
// `rs` = row * NS + s (16-byte loads: the threads of a warp take consecutive
// spans, i.e. consecutive chunks)
template <class C>
__device__ __forceinline__ void load_masks(const uint32_t* s_mask, const BoxGeom& bg, int j, int rs,
                                           uint32_t (&m)[C::NQ]) {
#pragma unroll
  for (int h = 0; h < C::NQC; ++h) {
    const uint4 v = *reinterpret_cast<const uint4*>(s_mask + j * bg.pstride + h * bg.hstride + rs * 4);
    const uint32_t e[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
    for (int k = 0; k < 4; ++k)
      if (4 * h + k < C::NQ) m[4 * h + k] = e[k];
  }
}

// adds the pairs of vector V of one centre span: cm = centre masks (valid
// bits only), nrs = row * NS + s of the neighbour span
template <class C, int B, int V>
__device__ __forceinline__ void count_vec(const uint32_t (&cm)[4][C::NQ], const uint32_t* s_mask,
                                          const BoxGeom& bg, int nrs,
                                          uint32_t (&acc)[C::NQ][C::NQ]) {
  using N = BNbr<C, B, V>;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    uint32_t nm[C::NQ];
    const int jj = j + N::ox;
    if (jj < 4) {
      load_masks<C>(s_mask, bg, jj, nrs, nm);
    } else {
      uint32_t lo[C::NQ], hi[C::NQ];
      load_masks<C>(s_mask, bg, jj - 4, nrs, lo);
      load_masks<C>(s_mask, bg, jj - 4, nrs + 1, hi);
#pragma unroll
      for (int q = 0; q < C::NQ; ++q) nm[q] = __funnelshift_r(lo[q], hi[q], 1);
    }
    // a site has one species, so the centre masks of p and q are disjoint
    // and one popc of the union counts both orientations of the pair
#pragma unroll
    for (int p = 0; p < C::NQ; ++p) {
      acc[p][p] += __popc(cm[j][p] & nm[p]);
#pragma unroll
      for (int q = p + 1; q < C::NQ; ++q)
        acc[p][q] += __popc((cm[j][p] & nm[q]) | (cm[j][q] & nm[p]));
    }
  }
}

template <class C, int B, int Mm, int... K>
__device__ __forceinline__ void count_shell(const uint32_t (&cm)[4][C::NQ], const uint32_t* s_mask,
                                            const BoxGeom& bg, int tz, int ty, int s,
                                            uint32_t (&acc)[C::NQ][C::NQ],
                                            std::integer_sequence<int, K...>) {
  (count_vec<C, B, pairs::pos_vec(C::KIND, Mm, K)>(
       cm, s_mask, bg,
       ((BNbr<C, B, pairs::pos_vec(C::KIND, Mm, K)>::bp * bg.TZ +
         tz + BNbr<C, B, pairs::pos_vec(C::KIND, Mm, K)>::oz) * bg.TY +
        ty + BNbr<C, B, pairs::pos_vec(C::KIND, Mm, K)>::oy) * bg.NS + s,
       acc),
   ...);
}

template <class C>
__global__ void __launch_bounds__(C::NT) k_pair_count_bits(const __grid_constant__ Geom g,
                                                           const BoxGeom bg,
                                                           const uint8_t* __restrict__ occ,
                                                           unsigned long long* __restrict__ hcnt) {
  extern __shared__ __align__(16) uint32_t s_mask[];
  __shared__ uint32_t s_cnt[C::NCNT + C::NQ];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  constexpr int NW = C::NT / 32;
  for (int i = tid; i < C::NCNT + C::NQ; i += C::NT) s_cnt[i] = 0;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const size_t px = static_cast<size_t>(g.px);
  uint32_t scnt[C::NQ];  // species counts of this thread's centre spans
#pragma unroll
  for (int p = 0; p < C::NQ; ++p) scnt[p] = 0;

  // a block takes a contiguous run of boxes, z fastest within a column of
  // boxes, so that consecutive boxes share 2H staged rows in z
  const int k0 = static_cast<int>(static_cast<long long>(blockIdx.x) * bg.n_boxes / gridDim.x);
  const int k1 = static_cast<int>(static_cast<long long>(blockIdx.x + 1) * bg.n_boxes / gridDim.x);
  for (int box = k0; box < k1; ++box) {
    const int y0 = (box / bg.nbz) * bg.BY, z0 = (box % bg.nbz) * bg.BZ;
    // the previous box of this block is the one below in z: its staged rows
    // tz in [BZ, BZ + 2H) are this box's rows [0, 2H)
    const bool carry = box > k0 && box % bg.nbz != 0 && bg.BZ >= 2 * C::H;
    __syncthreads();  // the previous box's counting has finished reading the masks
    if (carry) {
      const int n_cp = 4 * C::NQC * C::NB * 2 * C::H * bg.TY * bg.NS;
      for (int i = tid; i < n_cp; i += C::NT) {
        int u = i;
        const int sp = u % bg.NS;
        u /= bg.NS;
        const int ty = u % bg.TY;
        u /= bg.TY;
        const int t = u % (2 * C::H);
        u /= 2 * C::H;
        const int b = u % C::NB;
        const int plane = u / C::NB;  // j * NQC + h
        const int src = ((b * bg.TZ + bg.BZ + t) * bg.TY + ty) * bg.NS + sp;
        const int dst = ((b * bg.TZ + t) * bg.TY + ty) * bg.NS + sp;
        uint4* base = reinterpret_cast<uint4*>(s_mask + plane * bg.hstride);
        base[dst] = base[src];
      }
      __syncthreads();  // the carried rows are read before the new rows overwrite them
    }
    // ---- masks of the box's rows plus halo (only the rows not carried): a
    // warp per staged row, spans of 128 sites (4 per lane), up to 8 spans'
    // loads in flight before their ballots
    const int tz0 = carry ? 2 * C::H : 0, nzs = bg.TZ - tz0;
    const int n_rows = C::NB * nzs * bg.TY;
    for (int rs = warp; rs < n_rows; rs += NW) {
      const int ty = rs % bg.TY, t = rs / bg.TY;
      const int tz = tz0 + t % nzs, b = t / nzs;
      const int r = (b * bg.TZ + tz) * bg.TY + ty;  // staged row index
      const int gy = pmod(y0 - C::H + ty, ny), gz = pmod(z0 - C::H + tz, nz);
      // 8-bit storage: basis b's row holds codes sigma * W; 4-bit storage:
      // row group b / 2 holds sigma of bases b & ~1 (low nibble) and b | 1
      const int grp = g.pack4 ? b >> 1 : b;
      const uint32_t sh = g.pack4 ? 4u * (b & 1) : 0u, fm = g.pack4 ? 0x0Fu : 0xFFu;
      const uint32_t mul = g.pack4 ? 1u : static_cast<uint32_t>(C::W);
      const uint8_t* row = occ + ((static_cast<size_t>(grp) * nz + gz) * ny + gy) * px;
      for (int s0 = 0; s0 < bg.NS; s0 += 8) {
        uint32_t wv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int x = 128 * (s0 + k) + 4 * lane;
          wv[k] = 0;
          if (s0 + k >= bg.NS) continue;
          if (x + 4 <= nx) {
            wv[k] = *reinterpret_cast<const uint32_t*>(row + x);  // rows are 16-byte aligned
          } else {  // periodic wrap of the row's end (rows shorter than a span wrap more)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              int xx = x + e;
              if (xx >= nx) xx -= nx;
              if (xx >= nx) xx %= nx;
              wv[k] |= static_cast<uint32_t>(row[xx]) << (8 * e);
            }
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          if (s0 + k >= bg.NS) break;
          uint32_t bal[4][C::NQ];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint32_t c = (wv[k] >> (8 * j + sh)) & fm;
#pragma unroll
            for (int q = 0; q < C::NQ; ++q)
              bal[j][q] = __ballot_sync(0xffffffffu, c == static_cast<uint32_t>(q) * mul);
          }
          if (lane == 0) {  // the ballots are warp-uniform: one lane stores the chunks
            uint32_t* dst = s_mask + (r * bg.NS + s0 + k) * 4;
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
              for (int h = 0; h < C::NQC; ++h) {
                uint32_t v[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) v[e] = 4 * h + e < C::NQ ? bal[j][4 * h + e] : 0u;
                *reinterpret_cast<uint4*>(dst + j * bg.pstride + h * bg.hstride) =
                    make_uint4(v[0], v[1], v[2], v[3]);
              }
          }
        }
      }
    }
    __syncthreads();
    // ---- pairs of every centre span of the box, shell by shell
    const int n_items = bg.BZ * bg.BY * bg.NSC;
    auto shell = [&](auto mconst) {
      constexpr int Mm = decltype(mconst)::value;
      uint32_t acc[C::NQ][C::NQ];
#pragma unroll
      for (int p = 0; p < C::NQ; ++p)
#pragma unroll
        for (int q = p; q < C::NQ; ++q) acc[p][q] = 0;
      auto basis = [&](auto bconst) {
        constexpr int B = decltype(bconst)::value;
        for (int it = tid; it < n_items; it += C::NT) {
          const int s = it % bg.NSC;
          const int t = it / bg.NSC;
          const int yl = t % bg.BY, zl = t / bg.BY;
          if (y0 + yl >= ny || z0 + zl >= nz) continue;
          const int tz = zl + C::H, ty = yl + C::H;
          const int crs = ((B * bg.TZ + tz) * bg.TY + ty) * bg.NS + s;
          const int rem = nx - 128 * s;  // sites of this span inside the row
          uint32_t cm[4][C::NQ];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const int nbits = min(32, max(0, (rem - j + 3) >> 2));
            const uint32_t valid = nbits == 32 ? 0xffffffffu : ((1u << nbits) - 1u);
            load_masks<C>(s_mask, bg, j, crs, cm[j]);
#pragma unroll
            for (int q = 0; q < C::NQ; ++q) cm[j][q] &= valid;
          }
          if constexpr (Mm == 0) {
#pragma unroll
            for (int p = 0; p < C::NQ; ++p)
              scnt[p] += __popc(cm[0][p]) + __popc(cm[1][p]) + __popc(cm[2][p]) + __popc(cm[3][p]);
          }
          count_shell<C, B, Mm>(cm, s_mask, bg, tz, ty, s, acc,
                                std::make_integer_sequence<int, shell_z(C::KIND, Mm) / 2>{});
        }
      };
      basis(std::integral_constant<int, 0>{});
      basis(std::integral_constant<int, 1>{});
      if constexpr (C::NB == 4) {
        basis(std::integral_constant<int, 2>{});
        basis(std::integral_constant<int, 3>{});
      }
#pragma unroll
      for (int p = 0; p < C::NQ; ++p)
#pragma unroll
        for (int q = p; q < C::NQ; ++q) {
          const uint32_t v = __reduce_add_sync(0xffffffffu, acc[p][q]);
          if (lane == 0 && v) atomicAdd(&s_cnt[(Mm * C::NQ + p) * C::NQ + q], v);
        }
    };
    shell(std::integral_constant<int, 0>{});
    if constexpr (C::M > 1) shell(std::integral_constant<int, 1>{});
    if constexpr (C::M > 2) shell(std::integral_constant<int, 2>{});
    if constexpr (C::M > 3) shell(std::integral_constant<int, 3>{});
  }
#pragma unroll
  for (int p = 0; p < C::NQ; ++p) {
    const uint32_t v = __reduce_add_sync(0xffffffffu, scnt[p]);
    if (lane == 0 && v) atomicAdd(&s_cnt[C::NCNT + p], v);
  }
  __syncthreads();
  constexpr int KM = C::KMAX - 1;
  for (int i = tid; i < C::NCNT; i += C::NT) {
    const int q = i % C::NQ, p = (i / C::NQ) % C::NQ, m = i / (C::NQ * C::NQ);
    if (s_cnt[i]) atomicAdd(&hcnt[(m * C::KMAX + p) * C::KMAX + q], static_cast<unsigned long long>(s_cnt[i]));
  }
  // species counts parked in H_0[p][KMAX - 1] until the finishing kernel
  for (int p = tid; p < C::NQ; p += C::NT)
    if (s_cnt[C::NCNT + p])
      atomicAdd(&hcnt[p * C::KMAX + KM], static_cast<unsigned long long>(s_cnt[C::NCNT + p]));
}

// The last species' row and column of every U_m from the species counts
// (one thread; see the header comment).  With N = U + U^T, row p of N sums
// to c_p z_m (z_m = the full shell): N_m[p][KMAX-1] = c_p z_m - sum_{q <
// KMAX-1} N_m[p][q], and N_m[KMAX-1][KMAX-1] (even) from the last row.
template <class C>
__global__ void k_pair_bits_finish(unsigned long long* __restrict__ h, unsigned long long n_sites) {
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  constexpr int KM = C::KMAX - 1;
  unsigned long long c[C::KMAX];
  unsigned long long rest = n_sites;
  for (int p = 0; p < KM; ++p) {
    c[p] = h[p * C::KMAX + KM];
    rest -= c[p];
  }
  c[KM] = rest;
  for (int m = 0; m < C::M; ++m) {
    const unsigned long long z = static_cast<unsigned long long>(shell_z(C::KIND, m));
    unsigned long long* um = h + m * C::KMAX * C::KMAX;
    unsigned long long last = 0;
    for (int p = 0; p < KM; ++p) {
      unsigned long long row = 0;  // sum over q < KM of N[p][q]
      for (int q = 0; q < KM; ++q)
        row += q == p ? 2 * um[p * C::KMAX + p] : um[min(p, q) * C::KMAX + max(p, q)];
      um[p * C::KMAX + KM] = c[p] * z - row;
      last += um[p * C::KMAX + KM];
    }
    um[KM * C::KMAX + KM] = (c[KM] * z - last) / 2;
  }
}

// box rows so that the staged masks fit `budget` bytes of shared memory;
// false if even 1 x 1 rows do not
template <class C>
bool box_for(const Geom& g, size_t budget, BoxGeom* bg, size_t* smem) {
  // a span past the last centre span only when the neighbours of the row's
  // last sites (x + H) do not fall into its wrapped tail; one padding chunk
  // after the masks keeps the next-span read of the last span in bounds
  // (its bits only reach invalid centres).  Box shapes, widest in y first
  // (with the z rows carried from box to box, a box costs (BY + 2H) / BY
  // staged rows per counted row).
  const int nsc = (g.n[0] + 127) / 128;
  const int ns = (g.n[0] + C::H + 127) / 128;
  constexpr int kShapes[][2] = {{16, 4}, {8, 8}, {8, 4}, {4, 4}, {4, 2}, {2, 2}, {2, 1}, {1, 1}};
  for (const auto& sh : kShapes) {
    const int by = sh[0], bz = sh[1];
    const int ty = by + 2 * C::H, tz = bz + 2 * C::H;
    const size_t bytes = (static_cast<size_t>(C::NB) * tz * ty * ns * C::SW + 4) * 4;
    const int hstride = C::NB * tz * ty * ns * 4;
    if (bytes <= budget) {
      bg->BY = by;
      bg->BZ = bz;
      bg->TY = ty;
      bg->TZ = tz;
      bg->NS = ns;
      bg->NSC = nsc;
      bg->nby = (g.n[1] + by - 1) / by;
      bg->nbz = (g.n[2] + bz - 1) / bz;
      bg->n_boxes = bg->nby * bg->nbz;
      bg->n_sites = static_cast<unsigned long long>(C::NB) * g.n[0] * g.n[1] * g.n[2];
      bg->hstride = hstride;
      bg->pstride = C::NQC * hstride;
      *smem = bytes;
      return true;
    }
  }
  return false;
}

template <class C>
bool b_supported(const Geom& g) {
  if (g.kind != C::KIND || g.K > 6 || (g.K == 6) != (C::KMAX == 6)) return false;
  BoxGeom bg;
  size_t smem;
  return box_for<C>(g, 227 * 1024, &bg, &smem);
}

template <class C>
cudaError_t b_launch(const Geom& g, const uint8_t* occ, unsigned long long* hcnt, int n_sm,
                     cudaStream_t st) {
  BoxGeom bg;
  size_t smem = 0;
  // two blocks per SM when the masks allow it
  if (!box_for<C>(g, 110 * 1024, &bg, &smem) && !box_for<C>(g, 227 * 1024, &bg, &smem))
    return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(k_pair_count_bits<C>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  int per_sm = 0;
  e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_pair_count_bits<C>, C::NT, smem);
  if (e != cudaSuccess) return e;
  int grid = n_sm * (per_sm < 1 ? 1 : per_sm);
  if (grid > bg.n_boxes) grid = bg.n_boxes;
  k_pair_count_bits<C><<<grid, C::NT, smem, st>>>(g, bg, occ, hcnt);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  k_pair_bits_finish<C><<<1, 32, 0, st>>>(hcnt, bg.n_sites);
  return cudaGetLastError();
}

}  // namespace pbits
}  // namespace smcx
