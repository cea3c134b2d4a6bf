// kernels_cell.cuh -- the cell sweep phase: one thread runs the trials of one
// active link cell (Sec. 2.2) reading and writing the device storage
// directly (through L1/L2; lattices of batched jobs are L2-resident).
//
// Used where shared-memory tiles do not fit: small and medium lattices, and
// the batched form, in which one launch runs one colour phase of every job
// of a batch (blocks map to jobs through a block table).  Works on any
// lattice with at least 4 conventional cells per dimension (then no two
// shell vectors reach the same site, so the swapped pair's mutual bond is
// the only term to remove from the raw neighbour counts).
//
// Neighbour addressing: for the anchor's conventional cell the wrapped
// coordinates of offsets -3..3 along each axis are tabulated once (as byte
// offsets of the device storage), every neighbour address is the sum of
// three table entries and a basis-row offset, all indices compile-time; the
// partner's tables are selected from the anchor's by its shift.  The energy
// change and the Metropolis test are those of the tiled kernel (one-hot
// SWAR counts, difference rows, threshold tables).
#pragma once

#include <utility>

#include "device_util.cuh"
#include "kernels.h"
#include "kernels_tiled.cuh"

namespace smcx {
namespace cell {

using tiled::floordiv2;
using tiled::round_up;

template <int KIND_, int M_, int KMAX_>
struct CCfg {
  static constexpr int KIND = KIND_, M = M_, KMAX = KMAX_;
  static constexpr int NB = KIND == 0 ? 2 : 4;
  static constexpr int W = KMAX <= 5 ? 6 : 5;
  static constexpr int Z1 = shell_z(KIND, 0);
  static constexpr int DOFF_C = tiled_doff_c(M, KMAX);
  static constexpr int ROWB = tiled_row_bytes(M, KMAX);
  static constexpr int RSTEP = ROWB / W;
  static constexpr int DBYTES = KMAX * KMAX * ROWB;
  static constexpr int NT = 128;
  static constexpr int D_OFF = 4 * kTabWords;                         // shared layout
  static constexpr int PT_OFF = round_up(D_OFF + DBYTES, 16);
  static constexpr int SMEM = PT_OFF + 4 * NB * Z1;
};

// partner of a basis-b anchor in first-shell direction dir: conventional
// shift (dx, dy, dz) in {-1,0,1} and basis, packed (dx+1)|(dy+1)<<2|(dz+1)<<4|bj<<6
template <class C, int E>
struct CPartner {
  static constexpr int b = E / C::Z1, dir = E % C::Z1;
  static constexpr ShellVec v = shell_vec(C::KIND, dir);
  static constexpr int bx = basis_comp(C::KIND, b, 0), by = basis_comp(C::KIND, b, 1),
                       bz = basis_comp(C::KIND, b, 2);
  static constexpr int bj = basis_of_parity(C::KIND, (bx + v.x) & 1, (by + v.y) & 1, (bz + v.z) & 1);
  static constexpr int value = (floordiv2(bx + v.x) + 1) | ((floordiv2(by + v.y) + 1) << 2) |
                               ((floordiv2(bz + v.z) + 1) << 4) | (bj << 6);
};

template <class C, int... E>
__device__ __forceinline__ void fill_cpartner(int* t, std::integer_sequence<int, E...>) {
  ((t[E] = CPartner<C, E>::value), ...);
}

// neighbour V of a basis-B site: conventional offsets (index into the
// coordinate tables, 3 = the site's own cell) and the neighbour's basis
template <class C, int B, int V>
struct CNbr {
  static constexpr ShellVec v = shell_vec(C::KIND, V);
  static constexpr int bx = basis_comp(C::KIND, B, 0), by = basis_comp(C::KIND, B, 1),
                       bz = basis_comp(C::KIND, B, 2);
  static constexpr int ix = floordiv2(bx + v.x) + 3, iy = floordiv2(by + v.y) + 3,
                       iz = floordiv2(bz + v.z) + 3;
  static constexpr int bp = basis_of_parity(C::KIND, (bx + v.x) & 1, (by + v.y) & 1, (bz + v.z) & 1);
};

// FCC partner side: offsets of neighbour V from a site of basis 0 (index
// into tables of offsets -3..3), whether each component of V is odd (then a
// basis with that component 1 moves one cell further), and V's parity class
template <class C, int V>
struct CNbr0 {
  static constexpr ShellVec v = shell_vec(C::KIND, V);
  static constexpr int ix = floordiv2(v.x) + 3, iy = floordiv2(v.y) + 3, iz = floordiv2(v.z) + 3;
  static constexpr bool ox = (v.x & 1) != 0, oy = (v.y & 1) != 0, oz = (v.z & 1) != 0;
  static constexpr int cls = basis_of_parity(C::KIND, v.x & 1, v.y & 1, v.z & 1);
};

struct Coords {
  uint32_t x[7], y[7], z[7];  // byte offsets of coordinates -3..3 (x, y*px, z*ny*px)
};

template <class C, int B, int S, int LO, int HI>
__device__ __forceinline__ uint32_t csum_i(const uint8_t* occ, const Coords& T, const uint32_t* bofs) {
  if constexpr (HI - LO == 1) {
    using N = CNbr<C, B, S + LO>;
    return 1u << occ[T.x[N::ix] + T.y[N::iy] + T.z[N::iz] + bofs[N::bp]];
  } else {
    constexpr int MID = (LO + HI) / 2;
    return csum_i<C, B, S, LO, MID>(occ, T, bofs) + csum_i<C, B, S, MID, HI>(occ, T, bofs);
  }
}

// FCC partner: T holds the partner's own tables, To the tables shifted by one
// cell along the axes where the partner's basis component is 1
template <class C, int S, int LO, int HI>
__device__ __forceinline__ uint32_t csum_j_fcc(const uint8_t* occ, const Coords& T,
                                               const Coords& To, const uint32_t* cls_ofs) {
  if constexpr (HI - LO == 1) {
    using N = CNbr0<C, S + LO>;
    const uint32_t ax = N::ox ? To.x[N::ix] : T.x[N::ix];
    const uint32_t ay = N::oy ? To.y[N::iy] : T.y[N::iy];
    const uint32_t az = N::oz ? To.z[N::iz] : T.z[N::iz];
    return 1u << occ[ax + ay + az + cls_ofs[N::cls]];
  } else {
    constexpr int MID = (LO + HI) / 2;
    return csum_j_fcc<C, S, LO, MID>(occ, T, To, cls_ofs) + csum_j_fcc<C, S, MID, HI>(occ, T, To, cls_ofs);
  }
}

template <class C, int B, int... Ms>
__device__ __forceinline__ void cacc_i(const uint8_t* occ, const Coords& T, const uint32_t* bofs,
                                       uint32_t* acc, std::integer_sequence<int, Ms...>) {
  ((acc[Ms] = csum_i<C, B, shell_start(C::KIND, Ms), 0, shell_z(C::KIND, Ms)>(occ, T, bofs)), ...);
}

template <class C, int... Ms>
__device__ __forceinline__ void cacc_j_fcc(const uint8_t* occ, const Coords& T, const Coords& To,
                                           const uint32_t* cls_ofs, uint32_t* acc,
                                           std::integer_sequence<int, Ms...>) {
  ((acc[Ms] = csum_j_fcc<C, shell_start(C::KIND, Ms), 0, shell_z(C::KIND, Ms)>(occ, T, To, cls_ofs)),
   ...);
}

__device__ __forceinline__ uint32_t sel3(int k, uint32_t a, uint32_t b, uint32_t c) {
  return k == 0 ? a : (k == 1 ? b : c);
}

// Trials of one link cell.  g: geometry; occ: device storage (8-bit codes);
// t: global sweep index; shift: the sweep's origin; cell (cx, cy, cz).
template <class C>
__device__ __forceinline__ void run_cell(const Geom& g, uint8_t* __restrict__ occ, uint32_t t,
                                         const int* shift, int cx, int cy, int cz, int mode,
                                         int sbin, const uint32_t* s_tab, const uint8_t* s_d,
                                         const int* s_pt, uint32_t* n_att, uint32_t* n_unl,
                                         uint32_t* n_acc, int64_t* sum_de) {
  const int c[3] = {cx, cy, cz};
  int lo[3], hi[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    lo[d] = link_bound(g, d, c[d]);
    hi[d] = link_bound(g, d, c[d] + 1);
  }
  const uint32_t cid = (static_cast<uint32_t>(cz) * g.m[1] + cy) * g.m[0] + cx;
  const int nx = g.n[0], ny = g.n[1], nz = g.n[2];
  const uint32_t px = static_cast<uint32_t>(g.px);
  const uint32_t zstr = px * static_cast<uint32_t>(ny);
  const uint32_t gstr = zstr * static_cast<uint32_t>(nz);
  uint32_t bofs[4];
#pragma unroll
  for (int b = 0; b < 4; ++b) bofs[b] = static_cast<uint32_t>(b) * gstr;
  const int lx = hi[0] - lo[0], ly = hi[1] - lo[1], lz = hi[2] - lo[2];
  *n_att += static_cast<uint32_t>(lx * ly * lz * C::NB);

  auto wrap = [](int v, int n) {
    v += v < 0 ? n : 0;
    v -= v >= n ? n : 0;
    return v;
  };

  for (int zr = 0; zr < lz; ++zr)
    for (int yr = 0; yr < ly; ++yr)
      for (int xr = 0; xr < lx; ++xr) {
        const int gx = wrap(lo[0] + xr + shift[0], nx);
        const int gy = wrap(lo[1] + yr + shift[1], ny);
        const int gz = wrap(lo[2] + zr + shift[2], nz);
        Coords T;
#pragma unroll
        for (int k = 0; k < 7; ++k) {
          T.x[k] = static_cast<uint32_t>(wrap(gx + k - 3, nx));
          T.y[k] = static_cast<uint32_t>(wrap(gy + k - 3, ny)) * px;
          T.z[k] = static_cast<uint32_t>(wrap(gz + k - 3, nz)) * zstr;
        }
        const uint32_t cc = static_cast<uint32_t>((zr * ly + yr) * lx + xr);

        auto attempt = [&](auto bconst, uint32_t wa, uint32_t wb) {
          constexpr int B = decltype(bconst)::value;
          const uint32_t dir = __umulhi(wa, static_cast<uint32_t>(C::Z1));
          const int pt = s_pt[B * C::Z1 + dir];
          const int sx = pt & 3, sy = (pt >> 2) & 3, sz = (pt >> 4) & 3, bj = pt >> 6;
          const uint32_t ai = T.x[3] + T.y[3] + T.z[3] + bofs[B];
          // the partner's tables: offsets -3..3 around its own cell (index
          // k + shift), entries beyond the anchor's range are never used
          // (partner-side indices stay in 1..5)
          Coords J;
#pragma unroll
          for (int k = 1; k < 6; ++k) {
            J.x[k] = sel3(sx, T.x[k - 1], T.x[k], T.x[k + 1]);
            J.y[k] = sel3(sy, T.y[k - 1], T.y[k], T.y[k + 1]);
            J.z[k] = sel3(sz, T.z[k - 1], T.z[k], T.z[k + 1]);
          }
          J.x[0] = J.x[6] = J.y[0] = J.y[6] = J.z[0] = J.z[6] = 0;
          const uint32_t aj = J.x[3] + J.y[3] + J.z[3] + bofs[bj];
          const uint32_t p = occ[ai], q = occ[aj];
          uint32_t acc_i[C::M], acc_j[C::M];
          cacc_i<C, B>(occ, T, bofs, acc_i, std::make_integer_sequence<int, C::M>{});
          if constexpr (C::KIND == 0) {
            cacc_i<C, 1 - B>(occ, J, bofs, acc_j, std::make_integer_sequence<int, C::M>{});
          } else {
            // partner basis bj: components of beta_bj shift odd offsets by one
            const bool kx = bj == 2 || bj == 3, ky = bj == 1 || bj == 3, kz = bj == 1 || bj == 2;
            Coords Jo;
#pragma unroll
            for (int k = 1; k < 5; ++k) {
              Jo.x[k] = kx ? J.x[k + 1] : J.x[k];
              Jo.y[k] = ky ? J.y[k + 1] : J.y[k];
              Jo.z[k] = kz ? J.z[k + 1] : J.z[k];
            }
            Jo.x[0] = Jo.x[5] = Jo.x[6] = Jo.y[0] = Jo.y[5] = Jo.y[6] = 0;
            Jo.z[0] = Jo.z[5] = Jo.z[6] = 0;
            uint32_t cls_ofs[4];
#pragma unroll
            for (int cl = 0; cl < 4; ++cl) cls_ofs[cl] = bofs[bj ^ cl];
            cacc_j_fcc<C>(occ, J, Jo, cls_ofs, acc_j, std::make_integer_sequence<int, C::M>{});
          }
          const bool unlike = p != q;
          *n_unl += unlike;
          const uint8_t* row = s_d + (p * C::KMAX + q) * C::RSTEP;
          constexpr int ND = C::M * (C::KMAX - 1);
          int32_t dr[(ND + 3) / 4 * 4];
#pragma unroll
          for (int v = 0; v < (ND + 3) / 4; ++v) {
            const int4 d4 = reinterpret_cast<const int4*>(row)[v];
            dr[4 * v] = d4.x;
            dr[4 * v + 1] = d4.y;
            dr[4 * v + 2] = d4.z;
            dr[4 * v + 3] = d4.w;
          }
          long long de = -*reinterpret_cast<const long long*>(row + C::DOFF_C);
#pragma unroll
          for (int m = 0; m < C::M; ++m) {
            if constexpr (C::KMAX <= 5) {
              const uint32_t F = 0x20820820u + acc_i[m] - acc_j[m];
#pragma unroll
              for (int s = 1; s < C::KMAX; ++s)
                de += static_cast<long long>(static_cast<int>((F >> (6 * s)) & 63u)) *
                      static_cast<long long>(dr[m * (C::KMAX - 1) + s - 1]);
            } else {
#pragma unroll
              for (int s = 1; s < C::KMAX; ++s)
                de += static_cast<long long>(static_cast<int>((acc_i[m] >> (5 * s)) & 31u) -
                                             static_cast<int>((acc_j[m] >> (5 * s)) & 31u)) *
                      static_cast<long long>(dr[m * (C::KMAX - 1) + s - 1]);
            }
          }
          const uint64_t idx = static_cast<uint64_t>(de) >> sbin;
          const uint32_t i2 = idx >> 18 < 511u ? static_cast<uint32_t>(idx >> 18) : 511u;
          const uint32_t thr = compose_threshold(s_tab[idx & 511u], s_tab[512 + ((idx >> 9) & 511u)],
                                                 s_tab[1024 + i2]);
          const bool ok = unlike && (de <= 0 || mode == kModeAcceptAll ||
                                     (mode == kModeNormal && idx < (1ull << 27) && wb < thr));
          if (ok) {
            occ[ai] = static_cast<uint8_t>(q);
            occ[aj] = static_cast<uint8_t>(p);
            ++*n_acc;
            *sum_de += de;
          }
        };

        const U4 w0 = philox4x32_10_rk(cc * (C::NB / 2), cid, t, 0u, g.rk);
        attempt(std::integral_constant<int, 0>{}, w0.x, w0.y);
        attempt(std::integral_constant<int, 1>{}, w0.z, w0.w);
        if constexpr (C::NB == 4) {
          const U4 w1 = philox4x32_10_rk(cc * 2 + 1, cid, t, 0u, g.rk);
          attempt(std::integral_constant<int, 2>{}, w1.x, w1.y);
          attempt(std::integral_constant<int, 3>{}, w1.z, w1.w);
        }
      }
}

// the active cell with index `ci` of colour `colour` (cells of one colour in
// the order x fastest); false when the colour has no cell
__device__ __forceinline__ bool colour_cell(const Geom& g, int colour, uint32_t ci, int* c) {
  uint32_t A[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int bit = (colour >> d) & 1;
    if (g.m[d] == 1 && bit) return false;
    A[d] = g.m[d] == 1 ? 1u : static_cast<uint32_t>(g.m[d] / 2);
  }
  const uint32_t ax = ci % A[0], ay = (ci / A[0]) % A[1], az = ci / (A[0] * A[1]);
  if (az >= A[2]) return false;
  const uint32_t a[3] = {ax, ay, az};
#pragma unroll
  for (int d = 0; d < 3; ++d)
    c[d] = g.m[d] == 1 ? 0 : static_cast<int>(2 * a[d] + ((colour >> d) & 1));
  return true;
}

__device__ __forceinline__ void sweep_shift(const Geom& g, uint32_t t, bool no_shift, int* s) {
  if (no_shift) {
    s[0] = s[1] = s[2] = 0;
    return;
  }
  const U4 w = philox4x32_10_rk(0u, 0u, t, 1u, g.rk);
  s[0] = static_cast<int>(__umulhi(w.x, static_cast<uint32_t>(g.n[0])));
  s[1] = static_cast<int>(__umulhi(w.y, static_cast<uint32_t>(g.n[1])));
  s[2] = static_cast<int>(__umulhi(w.z, static_cast<uint32_t>(g.n[2])));
}

template <class C>
__device__ __forceinline__ void load_tables(uint8_t* smem, const uint32_t* tab, const uint8_t* dtab) {
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);
  for (int w = threadIdx.x; w < kTabWords; w += blockDim.x) s_tab[w] = tab[w];
  for (int w = threadIdx.x; w < C::DBYTES / 4; w += blockDim.x)
    reinterpret_cast<uint32_t*>(smem + C::D_OFF)[w] = reinterpret_cast<const uint32_t*>(dtab)[w];
  if (threadIdx.x == 0)
    fill_cpartner<C>(reinterpret_cast<int*>(smem + C::PT_OFF),
                     std::make_integer_sequence<int, C::NB * C::Z1>{});
}

// one colour phase of one lattice (plain path)
template <class C>
__global__ void __launch_bounds__(C::NT, 4) k_sweep_cells_single(const __grid_constant__ Geom g,
                                                              const PhaseArgs a,
                                                              const __grid_constant__ Tables tab,
                                                              uint8_t* __restrict__ occ,
                                                              const uint8_t* __restrict__ dtab,
                                                              unsigned long long* __restrict__ stats,
                                                              uint32_t n_cells) {
  __shared__ __align__(16) uint8_t smem[C::SMEM];
  load_tables<C>(smem, tab.w, dtab);
  __syncthreads();
  uint32_t n_att = 0, n_unl = 0, n_acc = 0;
  int64_t sum_de = 0;
  const uint32_t ci = blockIdx.x * C::NT + threadIdx.x;
  int c[3];
  if (ci < n_cells && colour_cell(g, a.colour, ci, c))
    run_cell<C>(g, occ, a.t, a.shift, c[0], c[1], c[2], a.mode, a.s,
                reinterpret_cast<const uint32_t*>(smem), smem + C::D_OFF,
                reinterpret_cast<const int*>(smem + C::PT_OFF), &n_att, &n_unl, &n_acc, &sum_de);
  warp_reduce_add_stats(stats, n_att, n_unl, n_acc, sum_de);
}

// one job of a batch, as the batched kernel reads it
struct JobDev {
  Geom g;
  uint8_t* occ;                 // device storage (8-bit codes)
  const uint8_t* dtab;          // difference rows
  const uint32_t* tab;          // Metropolis threshold tables (3 x 512)
  unsigned long long* stats;    // [0..3] this chunk, [4..7] since the job started
  uint32_t t0;                  // global sweep index of the chunk's first sweep
  uint32_t sweeps;              // sweeps the job runs in this chunk
  int mode, sbin;               // acceptance mode and bin shift of its temperature
  int no_shift;                 // SMCX_NO_SHIFT
  int pad_;
};

// One colour phase of sweep s of the chunk for every job of one kernel
// variant: blocks[i] = (job, first cell index) of block i.
template <class C>
__global__ void __launch_bounds__(C::NT, 4) k_sweep_cells_batch(const JobDev* __restrict__ jobs,
                                                             const uint2* __restrict__ blocks,
                                                             uint32_t n_blocks, uint32_t s,
                                                             int colour) {
  __shared__ __align__(16) uint8_t smem[C::SMEM];
  __shared__ Geom sg;
  if (blockIdx.x >= n_blocks) return;
  const uint2 bk = blocks[blockIdx.x];
  const JobDev* J = jobs + bk.x;
  if (threadIdx.x == 0) sg = J->g;
  load_tables<C>(smem, J->tab, J->dtab);
  __syncthreads();
  uint32_t n_att = 0, n_unl = 0, n_acc = 0;
  int64_t sum_de = 0;
  if (s < J->sweeps) {
    const uint32_t t = J->t0 + s;
    int shift[3];
    sweep_shift(sg, t, J->no_shift != 0, shift);
    int c[3];
    if (colour_cell(sg, colour, bk.y + threadIdx.x, c))
      run_cell<C>(sg, J->occ, t, shift, c[0], c[1], c[2], J->mode, J->sbin,
                  reinterpret_cast<const uint32_t*>(smem), smem + C::D_OFF,
                  reinterpret_cast<const int*>(smem + C::PT_OFF), &n_att, &n_unl, &n_acc, &sum_de);
  }
  warp_reduce_add_stats(J->stats, n_att, n_unl, n_acc, sum_de);
}

}  // namespace cell
}  // namespace smcx
