// kernels_cell.cuh -- the cell sweep phase: one thread runs the trials of one
// active link cell (Sec. 2.2) reading and writing the device storage
// directly (through L1/L2; lattices of batched jobs are L2-resident).
//
// Used for small and medium lattices (where it is also faster than the
// shared-memory tiles: they stay in L2) and for batches of many jobs, whose
// work items (32 cells of one job and colour phase, one per lane) are run
// either by one launch per colour phase or by one persistent launch per
// chunk of sweeps following a plan (k_sweep_cells_phase /
// k_sweep_cells_queue).  Works on any lattice with at least 4 conventional
// cells per dimension (then no two shell vectors reach the same site, so
// the swapped pair's mutual bond is the only term to remove from the raw
// neighbour counts).
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

// INLINE_KEYS: the Philox key schedule is computed in registers (the batched
// kernel, whose geometry sits in shared memory) instead of read from g.rk
template <int KIND_, int M_, int KMAX_, bool INLINE_KEYS_ = false>
struct CCfg {
  static constexpr int KIND = KIND_, M = M_, KMAX = KMAX_;
  static constexpr bool INLINE_KEYS = INLINE_KEYS_;
  static constexpr int NB = KIND == 0 ? 2 : 4;
  static constexpr int W = KMAX <= 5 ? 8 : 5;
  static constexpr int Z1 = shell_z(KIND, 0);
  static constexpr int DOFF_C = tiled_doff_c(M, KMAX);
  static constexpr int ROWB = tiled_row_bytes(M, KMAX);
  static constexpr int RSTEP = ROWB / W;
  static constexpr int DBYTES = KMAX * KMAX * ROWB;
  static constexpr int NT = 128;
  // resident blocks per SM the register budget allows: FCC with 3-4 shells
  // and BCC with 4 shells spill at 128 registers, so they get 170
  static constexpr int MINB = ((KIND == 1 && M >= 3) || (KIND == 0 && M >= 4)) ? 3 : 4;
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
    return onehot(occ[T.x[N::ix] + T.y[N::iy] + T.z[N::iz] + bofs[N::bp]]);
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
    return onehot(occ[ax + ay + az + cls_ofs[N::cls]]);
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
  const uint32_t key0 = g.seed_lo, key1 = g.seed_hi;
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
          // like pairs run the same branch-free path (their result is
          // discarded): for these L1-cached loads an early exit costs more
          // in divergence than it saves
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
          long long de;
          if constexpr (C::KMAX <= 5) {
            de = delta_e_dp4a<C::M, C::DOFF_C>(acc_i, acc_j, row);
          } else {
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
            de = -*reinterpret_cast<const long long*>(row + C::DOFF_C);
#pragma unroll
            for (int m = 0; m < C::M; ++m)
#pragma unroll
              for (int s = 1; s < C::KMAX; ++s)
                de += static_cast<long long>(static_cast<int>((acc_i[m] >> (5 * s)) & 31u) -
                                             static_cast<int>((acc_j[m] >> (5 * s)) & 31u)) *
                      static_cast<long long>(dr[m * (C::KMAX - 1) + s - 1]);
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

        auto draw = [&](uint32_t c0) {
          if constexpr (C::INLINE_KEYS) return philox4x32_10(c0, cid, t, 0u, key0, key1);
          else return philox4x32_10_rk(c0, cid, t, 0u, g.rk);
        };
        const U4 w0 = draw(cc * (C::NB / 2));
        attempt(std::integral_constant<int, 0>{}, w0.x, w0.y);
        attempt(std::integral_constant<int, 1>{}, w0.z, w0.w);
        if constexpr (C::NB == 4) {
          const U4 w1 = draw(cc * 2 + 1);
          attempt(std::integral_constant<int, 2>{}, w1.x, w1.y);
          attempt(std::integral_constant<int, 3>{}, w1.z, w1.w);
        }
      }
}

// the active cell with index `ci` of colour `colour` (cells of one colour in
// the order x fastest); false when the colour has no cell
__device__ __forceinline__ bool colour_cell(const Geom& g, int colour, int az0, int naz, uint32_t ci,
                                            int* c) {
  uint32_t A[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int bit = (colour >> d) & 1;
    if (g.m[d] == 1 && bit) return false;
    A[d] = g.m[d] == 1 ? 1u : static_cast<uint32_t>(g.m[d] / 2);
  }
  const uint32_t ax = ci % A[0], ay = (ci / A[0]) % A[1], az = ci / (A[0] * A[1]) + az0;
  if (az >= A[2] || az >= static_cast<uint32_t>(az0 + naz)) return false;
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
__global__ void __launch_bounds__(C::NT, C::MINB) k_sweep_cells_single(const __grid_constant__ Geom g,
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
  if (ci < n_cells && colour_cell(g, a.colour, a.az0, a.naz, ci, c))
    run_cell<C>(g, occ, a.t, a.shift, c[0], c[1], c[2], a.mode, a.s,
                reinterpret_cast<const uint32_t*>(smem), smem + C::D_OFF,
                reinterpret_cast<const int*>(smem + C::PT_OFF), &n_att, &n_unl, &n_acc, &sum_de);
  warp_reduce_add_stats(stats, n_att, n_unl, n_acc, sum_de);
}

// ---- batched form: one persistent launch runs a chunk of sweeps of every job

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
  int variant;                  // cell_variant(g)
  uint32_t items;               // work items of one colour phase
  uint32_t ex, ey;              // items along x and y of the active-cell grid
  uint32_t A[3];                // active cells of a colour along each axis
};

// The chunk's work.  Within a colour phase the items of the active jobs
// follow one another in `order` (the phase-synchronous schedule runs item k
// of every phase on warp k).  An item is 32 active cells of one job, one per
// lane of a warp: with tx < 0 the next 32 cells of the colour in x-fastest
// order, else a box of 2^tx x 2^ty x 2^(5-tx-ty) cells of the colour's
// active-cell grid.  The persistent schedule follows a plan: warp w of the
// grid owns segments seg[wfirst[w] .. wfirst[w+1]) -- a segment is a range
// of consecutive items (x = job slot, y = first item, z = items) -- and runs
// them for every colour phase of the chunk in turn, the same items in every
// phase.
struct QueueArgs {
  const JobDev* jobs;
  const uint32_t* order;        // slots of the active jobs
  const uint32_t* first;        // first item of order[a] within a phase; first[n_active] = n_items
  uint32_t n_active;
  uint32_t n_items;
  const uint4* seg;             // persistent plan: segments
  const uint32_t* wfirst;       // first segment of each warp; wfirst[n_warps] = segments
  uint32_t n_warps;             // warps of the plan (the persistent grid's)
  uint32_t n_ph;                // colour phases of the chunk (8 x its sweeps)
  unsigned long long* ctr;      // [1] status, [2 + slot] items finished per job
  unsigned long long* qstats;   // [0] items that waited, [1] polls, [2] ns waited
  int tx, ty;
};

constexpr unsigned long long kQueueTimeout = 1;        // status: a wait gave up
constexpr unsigned long long kWaitLimitNs = 2000000000ull;  // 2 s per wait
constexpr uint32_t kWaitMaxPolls = 1u << 24;                // and at most this many polls
constexpr int kQueueWarps = 4;  // warps per block of either batched schedule

__device__ __forceinline__ unsigned long long globaltimer_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

__device__ __forceinline__ unsigned long long ld_relaxed(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

// Bounded wait until *p >= need (relaxed polls with exponential back-off,
// 32 ns to 4 us, so that waiting warps do not crowd the L2 slice of the
// counter; the caller fences after a success).  False when the status word
// is set by another warp, after kWaitLimitNs, or after kWaitMaxPolls polls.
// A wait that polled adds itself, its polls and its duration to qstats.
static __device__ __noinline__ bool wait_at_least(const unsigned long long* p,
                                                  unsigned long long need,
                                                  const unsigned long long* status,
                                                  unsigned long long* qstats) {
  if (ld_relaxed(p) >= need) return true;
  const unsigned long long t0 = globaltimer_ns();
  uint32_t sleep_ns = 32;
  bool ok = false;
  uint32_t it = 1;
  for (; it <= kWaitMaxPolls; ++it) {
    __nanosleep(sleep_ns);
    if (sleep_ns < 4096) sleep_ns <<= 1;
    if (ld_relaxed(p) >= need) {
      ok = true;
      break;
    }
    if ((it & 15u) == 0) {
      if (ld_relaxed(status) != 0) break;
      if (globaltimer_ns() - t0 > kWaitLimitNs) break;
    }
  }
  atomicAdd(qstats, 1ull);
  atomicAdd(qstats + 1, static_cast<unsigned long long>(it));
  atomicAdd(qstats + 2, globaltimer_ns() - t0);
  return ok;
}

template <int KIND, int M, int KMAX>
__device__ __forceinline__ void run_queued(const Geom& g, uint8_t* occ, int mode, int sbin,
                                           uint32_t t, const int* shift, const int* c,
                                           const uint32_t* s_tab, const uint8_t* s_d,
                                           const int* s_pt, uint32_t* n_att, uint32_t* n_unl,
                                           uint32_t* n_acc, int64_t* sum_de) {
  using C = CCfg<KIND, M, KMAX, true>;
  run_cell<C>(g, occ, t, shift, c[0], c[1], c[2], mode, sbin, s_tab, s_d,
              s_pt + (KIND ? 2 * shell_z(0, 0) : 0), n_att, n_unl, n_acc, sum_de);
}

// Shared state of a block of either batched schedule: the partner tables of
// both lattice kinds and each warp's copy of its current job's geometry
// (its tables sit in the warp's slice of the dynamic shared memory).
struct QueueShared {
  int pt[2 * shell_z(0, 0) + 4 * shell_z(1, 0)];
  Geom g[kQueueWarps];
};

__device__ __forceinline__ void queue_block_init(QueueShared& sh) {
  constexpr int kPtB = 2 * shell_z(0, 0), kPtF = 4 * shell_z(1, 0);
  if (threadIdx.x == 0) {
    fill_cpartner<CCfg<0, 2, 5>>(sh.pt, std::make_integer_sequence<int, kPtB>{});
    fill_cpartner<CCfg<1, 2, 5>>(sh.pt + kPtB, std::make_integer_sequence<int, kPtF>{});
  }
  __syncthreads();
}

// job slot of item k of a phase and the item's index within the job
__device__ __forceinline__ uint32_t queue_job(const QueueArgs& q, uint32_t k, uint32_t* li) {
  uint32_t lo = 0, hi = q.n_active;  // first[lo] <= k < first[hi]
  while (hi - lo > 1) {
    const uint32_t mid = (lo + hi) >> 1;
    if (__ldg(q.first + mid) <= k) lo = mid;
    else hi = mid;
  }
  *li = k - __ldg(q.first + lo);
  return __ldg(q.order + lo);
}

// the job's geometry into the warp's shared slot, unless the warp's previous
// item was of the same job (warp-uniform).  The job's threshold and
// difference tables are read where they are, in global memory, through L1:
// a per-warp shared copy (12 KB) would leave the SM's L1 too small for the
// lattices of the jobs it runs.
__device__ __forceinline__ void queue_load_job(const JobDev* J, uint32_t slot, uint32_t* cur,
                                               Geom* g, int lane) {
  if (slot == *cur) return;
  const uint32_t* gsrc = reinterpret_cast<const uint32_t*>(&J->g);
  uint32_t* gdst = reinterpret_cast<uint32_t*>(g);
  for (int w = lane; w < static_cast<int>(sizeof(Geom) / 4); w += 32) gdst[w] = __ldg(gsrc + w);
  *cur = slot;
  __syncwarp();
}

// The 32 cells of item li of colour phase ph (sweep ph / 8 of the chunk) of
// job J, one per lane, then the warp's statistics into the job's counters.
__device__ __forceinline__ void queue_run_item(const QueueArgs& q, const JobDev* J, uint32_t ph,
                                               uint32_t li, int lane, const Geom& g,
                                               const int* s_pt) {
  const uint32_t* const s_tab =
      reinterpret_cast<const uint32_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->tab)));
  const uint8_t* const s_d =
      reinterpret_cast<const uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->dtab)));
  const int colour = static_cast<int>(ph & 7u);
  const uint32_t A0 = __ldg(&J->A[0]), A1 = __ldg(&J->A[1]);
  uint32_t a[3];
  if (q.tx < 0) {
    const uint32_t ci = li * 32u + static_cast<uint32_t>(lane);
    a[0] = ci % A0;
    a[1] = (ci / A0) % A1;
    a[2] = ci / (A0 * A1);
  } else {
    const int tz = 5 - q.tx - q.ty;
    const uint32_t ex = __ldg(&J->ex), ey = __ldg(&J->ey);
    const uint32_t ix = li % ex, r = li / ex;
    const uint32_t iy = r % ey, iz = r / ey;
    a[0] = (ix << q.tx) + (lane & ((1u << q.tx) - 1u));
    a[1] = (iy << q.ty) + ((lane >> q.tx) & ((1u << q.ty) - 1u));
    a[2] = (iz << tz) + (static_cast<uint32_t>(lane) >> (q.tx + q.ty));
  }
  bool active = true;
  int c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const int bit = (colour >> d) & 1;
    active = active && a[d] < __ldg(&J->A[d]) && !(g.m[d] == 1 && bit);
    c[d] = g.m[d] == 1 ? 0 : static_cast<int>(2 * a[d]) + bit;
  }
  uint32_t n_att = 0, n_unl = 0, n_acc = 0;
  int64_t sum_de = 0;
  if (active) {
    const uint32_t t = __ldg(&J->t0) + (ph >> 3);
    const int mode = __ldg(&J->mode), sbin = __ldg(&J->sbin);
    uint8_t* const occ =
        reinterpret_cast<uint8_t*>(__ldg(reinterpret_cast<const unsigned long long*>(&J->occ)));
    int shift[3];
    sweep_shift(g, t, __ldg(&J->no_shift) != 0, shift);
#define SMCX_RUNQ(KI, MM, KM)                                                                 \
  run_queued<KI, MM, KM>(g, occ, mode, sbin, t, shift, c, s_tab, s_d, s_pt, &n_att, &n_unl, \
                         &n_acc, &sum_de)
    switch (__ldg(&J->variant)) {
      case 0: SMCX_RUNQ(0, 2, 5); break;
      case 1: SMCX_RUNQ(0, 2, 6); break;
      case 2: SMCX_RUNQ(0, 3, 5); break;
      case 3: SMCX_RUNQ(0, 3, 6); break;
      case 4: SMCX_RUNQ(0, 4, 5); break;
      case 5: SMCX_RUNQ(0, 4, 6); break;
      case 6: SMCX_RUNQ(1, 2, 5); break;
      case 7: SMCX_RUNQ(1, 2, 6); break;
      case 8: SMCX_RUNQ(1, 3, 5); break;
      case 9: SMCX_RUNQ(1, 3, 6); break;
      case 10: SMCX_RUNQ(1, 4, 5); break;
      default: SMCX_RUNQ(1, 4, 6); break;
    }
#undef SMCX_RUNQ
  }
  unsigned long long* const stats = reinterpret_cast<unsigned long long*>(
      __ldg(reinterpret_cast<const unsigned long long*>(&J->stats)));
  warp_reduce_add_stats(stats, n_att, n_unl, n_acc, sum_de);
}

// Persistent schedule: every colour phase of a chunk of sweeps of every job
// of a batch in one launch.  Each warp runs its segments of the plan phase
// by phase, in plan order (a segment's items are the same in every phase,
// so a warp keeps coming back to the same part of the same lattice and
// finds it in its SM's L1).  Before a segment of phase ph, the warp waits
// (bounded) until all items of the job's phase ph - 1 have finished,
// wherever they run.  The launch is cooperative, so every warp of the plan
// is resident; a warp waits only for items of an earlier phase, which every
// other warp reaches before any item of a later one, so by induction over
// the phases every wait ends.  A finished segment is released (warp
// barrier, fence, counter increment); the waiting lane polls the count with
// relaxed loads and fences once it has seen it (acquire), then the warp
// barrier passes that on to the other lanes.
template <int MINB>
__global__ void __launch_bounds__(32 * kQueueWarps, MINB)
    k_sweep_cells_queue(const __grid_constant__ QueueArgs q) {
  __shared__ QueueShared sh;
  queue_block_init(sh);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t gw = blockIdx.x * kQueueWarps + warp;
  if (gw >= q.n_warps) return;
  unsigned long long* const status = q.ctr + 1;
  unsigned long long* const done = q.ctr + 2;
  const uint32_t s0 = __ldg(q.wfirst + gw), s1 = __ldg(q.wfirst + gw + 1);
  uint32_t cur = 0xFFFFFFFFu;
  for (uint32_t ph = 0; ph < q.n_ph; ++ph) {
    for (uint32_t s = s0; s < s1; ++s) {
      const uint4 sg = __ldg(q.seg + s);
      const JobDev* J = q.jobs + sg.x;
      if ((ph >> 3) >= __ldg(&J->sweeps)) continue;  // the job stops earlier; nobody waits for it
      int stop = 0;
      if (lane == 0) {
        stop = ld_relaxed(status) != 0;
        if (!stop && ph != 0) {
          if (wait_at_least(done + sg.x, static_cast<unsigned long long>(ph) * __ldg(&J->items),
                            status, q.qstats))
            __threadfence();
          else {
            atomicExch(status, kQueueTimeout);
            stop = 1;
          }
        }
      }
      stop = __shfl_sync(0xffffffffu, stop, 0);
      if (stop) return;
      queue_load_job(J, sg.x, &cur, &sh.g[warp], lane);
      __syncwarp();
      for (uint32_t li = sg.y; li < sg.y + sg.z; ++li)
        queue_run_item(q, J, ph, li, lane, sh.g[warp], sh.pt);
      __syncwarp();
      if (lane == 0) {
        __threadfence();
        atomicAdd(done + sg.x, static_cast<unsigned long long>(sg.z));
      }
    }
  }
}

// Phase-synchronous schedule: colour phase ph of every job of a batch in
// one launch (kernel boundaries order the phases); warp w of block b runs
// item 4b + w of the phase.
template <int MINB>
__global__ void __launch_bounds__(32 * kQueueWarps, MINB)
    k_sweep_cells_phase(const __grid_constant__ QueueArgs q, uint32_t ph) {
  __shared__ QueueShared sh;
  queue_block_init(sh);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t k = blockIdx.x * kQueueWarps + warp;
  if (k >= q.n_items) return;
  uint32_t li;
  const uint32_t slot = queue_job(q, k, &li);
  const JobDev* J = q.jobs + slot;
  if ((ph >> 3) >= __ldg(&J->sweeps)) return;
  uint32_t cur = 0xFFFFFFFFu;
  queue_load_job(J, slot, &cur, &sh.g[warp], lane);
  queue_run_item(q, J, ph, li, lane, sh.g[warp], sh.pt);
}

}  // namespace cell
}  // namespace smcx
