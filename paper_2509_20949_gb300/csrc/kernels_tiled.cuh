// kernels_tiled.cuh -- the shared-memory tiled sweep phase.
//
// One colour phase of the checkerboard (Sec. 2.2): every active link cell
// runs its trials sequentially (raster order), cells of one colour run
// concurrently because they never touch one another's interaction zones.
// A block owns BX x BY x BZ active cells of the phase; it stages their
// cells plus a two-conventional-cell halo (the local interaction zone of
// every trial, Sec. 2.2) from HBM into shared memory -- one bulk (TMA) copy
// per tile sub-row, completed on an mbarrier, where the sub-row's 16-byte
// aligned span fits the tile row; 8-byte cp.async copies otherwise; byte
// loads for tiles across the periodic x seam -- and runs the trials on the
// shared tile.  An accepted swap is stored to HBM at once (8-bit storage,
// 32-bit offsets that follow the loop counters); tiles across a periodic
// seam and packed storage instead store the part of the tile their trials
// can have changed back to HBM at the end.
//
// Energy change of a trial (EPI model, Sec. 3): with p = sigma_i, q = sigma_j,
//   dE = sum_m sum_s dx_{m,s} (V_m(q,s) - V_m(p,s)) - (V_1(p,p)+V_1(q,q)-2V_1(p,q)),
// where dx_{m,s} = (# shell-m neighbours of i of species s) - (same for j):
// the neighbour species are counted with one-hot SWAR adds (each shared
// memory byte holds sigma*W, the bit position of species sigma in the count
// word), the i-j bond, counted once from each side, is removed by the last
// term.  Because sum_s dx_{m,s} = 0 one species' column folds into the
// others.  K <= 5 (W = 8): byte s counts species s, species 4 shifts out, and
// the two count words meet in four byte dot products per shell
// (delta_e_dp4a); K = 6 (W = 5): 5-bit fields, species 0 folded.
//
// Shared tile layout: rows (z, y) of pitch RS holding NB sub-rows (one per
// basis site b) of pitch XW; byte x of sub-row b is site (x, y, z, b).  With
// warps of 16 cells along x and 2 along y (cells 2L conventional cells
// apart) RS is congruent to 16 modulo 32 bytes, so the 32 lanes hit 32
// distinct banks for every anchor-side neighbour load; warps of 32 cells
// along x take the pitches described at Cfg::RS.  Shared offsets of every neighbour are
// compile-time constants (the anchor's basis is unrolled); the partner's
// basis is fixed for BCC and taken from four class bases for FCC.
#pragma once

#include <utility>

#include "device_util.cuh"
#include "kernels.h"

namespace smcx {
namespace tiled {

__host__ __device__ constexpr int floordiv2(int v) { return v >= 0 ? v / 2 : -((1 - v) / 2); }
__host__ __device__ constexpr int round_up(int v, int a) { return (v + a - 1) / a * a; }

// parity mask (bit c = component c odd) of basis site b
__host__ __device__ constexpr int basis_mask(int kind, int b) {
  return basis_comp(kind, b, 0) | (basis_comp(kind, b, 1) << 1) | (basis_comp(kind, b, 2) << 2);
}
__host__ __device__ constexpr int basis_from_mask(int kind, int mask) {
  return basis_of_parity(kind, mask & 1, (mask >> 1) & 1, (mask >> 2) & 1);
}

__host__ __device__ constexpr int shell_reach_c(int kind, int M) {
  int r = 0;
  for (int i = 0; i < shell_start(kind, M); ++i) {
    const ShellVec v = shell_vec(kind, i);
    const int ax = v.x < 0 ? -v.x : v.x, ay = v.y < 0 ? -v.y : v.y, az = v.z < 0 ? -v.z : v.z;
    r = ax > r ? ax : r;
    r = ay > r ? ay : r;
    r = az > r ? az : r;
  }
  return r;
}

template <int KIND_, int M_, int KMAX_, bool PACK4_, int BX_, int BY_, int BZ_, bool RAGGED_>
struct Cfg {
  static constexpr int KIND = KIND_, M = M_, KMAX = KMAX_, BX = BX_, BY = BY_, BZ = BZ_;
  static constexpr bool PACK4 = PACK4_, RAGGED = RAGGED_;
  static constexpr int NB = KIND == 0 ? 2 : 4;
  static constexpr int HR = shell_reach_c(KIND, M);
  static constexpr int L = (1 + HR) / 2 + 1;   // link-cell edge (conventional cells)
  static constexpr int H = 2;                  // halo: reads reach 1 + h_R <= 4 half units
  // cells of edge L+1 in a ragged dimension (none when every edge is L)
  static constexpr int SLACK = RAGGED ? 2 * L - 1 : 0;
  static constexpr int EXT_X = (2 * BX - 1) * L + SLACK + 2 * H;
  static constexpr int EXT_Y = (2 * BY - 1) * L + SLACK + 2 * H;
  static constexpr int EXT_Z = (2 * BZ - 1) * L + SLACK + 2 * H;
  static constexpr int XW = round_up(EXT_X + 14, 8);  // 8-byte copy alignment slack
  static constexpr int RS0 = NB * XW;
  // Row and plane pitches.  Warps of 16 x 2 cells: RS = 16 mod 32 bytes puts
  // the two y lanes of a warp 16 banks apart.  Warps of 32 cells along x
  // (BX = 32) cover all 32 banks with their anchors whatever the pitches,
  // which are then chosen for the partner side: RS = 64 mod 128 and PS = 0
  // mod 128, so a partner one row or plane away moves a lane by 0 or 16
  // banks (at most two-way conflicts; a partner one byte away in x stays in
  // its own or the next lane's word).
  static constexpr bool WIDE = BX == 32;
  static constexpr int BANK = BX >= 16 ? 16 : BX;     // lane spacing of the y lanes in banks
  static constexpr int RS_W = round_up(RS0, 64) % 128 == 0 ? round_up(RS0, 64) + 64
                                                           : round_up(RS0, 64);
  static constexpr int RS = WIDE ? RS_W : RS0 + (((BANK - RS0 % 32) % 32) + 32) % 32;
  static constexpr int PS = WIDE ? round_up(RS * EXT_Y, 128) : RS * EXT_Y;
  static constexpr int W = KMAX <= 5 ? 8 : 5;
  static constexpr int NT = BX * BY * BZ;
  // resident blocks per SM the register budget must allow (shared memory
  // admits about as many)
  static constexpr int MINB = NT >= 256 ? 3 : (NT >= 128 ? 4 : 6);
  static constexpr int Z1 = shell_z(KIND, 0);
  static constexpr int NV = shell_start(KIND, M);
  // difference rows: int32 D'[m][s-1] then the int64 constant C at DOFF_C;
  // row (sigma_p, sigma_q) starts at byte (code_p * KMAX + code_q) * RSTEP,
  // i.e. at (sigma_p * KMAX + sigma_q) * ROWB, so codes index it directly
  static constexpr int DOFF_C = tiled_doff_c(M, KMAX);
  static constexpr int ROWB = tiled_row_bytes(M, KMAX);
  static constexpr int RSTEP = ROWB / W;
  static constexpr int DBYTES = KMAX * KMAX * ROWB;
  static constexpr int G = PACK4 ? NB / 2 : NB;                   // device row groups
  static constexpr int MBAR_OFF = round_up(4 * kTabWords + DBYTES + 8 * NB * Z1, 8);
  static constexpr int TILE_OFF = round_up(MBAR_OFF + 8, 16);  // bytes before the tile
  // sub-rows can be bulk-copied (16-byte aligned destinations) when every
  // pitch is a multiple of 16 bytes
  static constexpr bool BULK = XW % 16 == 0 && RS % 16 == 0 && PS % 16 == 0;
  static_assert(WIDE ? (RS % 128 == 64 && PS % 128 == 0) : RS % 32 == BANK % 32, "bank padding");
  static_assert(RS % 8 == 0 && XW % 8 == 0, "8-byte alignment of the tile rows");
};

// shared-memory offset of neighbour d of a site of basis b: the neighbour's
// conventional cell is floor((beta_b + d)/2) away, its basis the parity of
// beta_b + d.
template <class C>
__host__ __device__ constexpr int nbr_offset(int b, int dx, int dy, int dz) {
  const int bx = basis_comp(C::KIND, b, 0), by = basis_comp(C::KIND, b, 1),
            bz = basis_comp(C::KIND, b, 2);
  const int cx = floordiv2(bx + dx), cy = floordiv2(by + dy), cz = floordiv2(bz + dz);
  const int bp = basis_of_parity(C::KIND, (bx + dx) & 1, (by + dy) & 1, (bz + dz) & 1);
  return cx + cy * C::RS + cz * C::PS + (bp - b) * C::XW;
}

template <class C, int B, int V>
struct NbrOff {
  static constexpr ShellVec v = shell_vec(C::KIND, V);
  static constexpr int value = nbr_offset<C>(B, v.x, v.y, v.z);
};

// FCC partner-side decomposition: offset(b, d) = off0(d) + corr(b, class(d)),
// class(d) = basis index of d's parity.
template <class C, int V>
struct Off0 {
  static constexpr ShellVec v = shell_vec(C::KIND, V);
  static constexpr int cls = basis_of_parity(C::KIND, v.x & 1, v.y & 1, v.z & 1);
  static constexpr int value = nbr_offset<C>(0, v.x, v.y, v.z);
};

template <class C>
__host__ __device__ constexpr int corr_of(int b, int cls) {
  // any vector of class cls gives the same correction; use the parity vector itself
  return nbr_offset<C>(b, basis_comp(C::KIND, cls, 0), basis_comp(C::KIND, cls, 1),
                       basis_comp(C::KIND, cls, 2)) -
         nbr_offset<C>(0, basis_comp(C::KIND, cls, 0), basis_comp(C::KIND, cls, 1),
                       basis_comp(C::KIND, cls, 2));
}

// one-hot SWAR count of the species codes at base + offsets of shell vectors
// [S + LO, S + HI), summed as a balanced tree (independent adds)
template <class C, int B, int S, int LO, int HI>
__device__ __forceinline__ uint32_t count_i(const uint8_t* base) {
  if constexpr (HI - LO == 1) {
    return onehot(base[NbrOff<C, B, S + LO>::value]);
  } else {
    constexpr int MID = (LO + HI) / 2;
    return count_i<C, B, S, LO, MID>(base) + count_i<C, B, S, MID, HI>(base);
  }
}

template <class C, int S, int LO, int HI>
__device__ __forceinline__ uint32_t count_j_fcc(const uint8_t* const* cls_base) {
  if constexpr (HI - LO == 1) {
    return onehot(cls_base[Off0<C, S + LO>::cls][Off0<C, S + LO>::value]);
  } else {
    constexpr int MID = (LO + HI) / 2;
    return count_j_fcc<C, S, LO, MID>(cls_base) + count_j_fcc<C, S, MID, HI>(cls_base);
  }
}

template <class C, int B, int... Ms>
__device__ __forceinline__ void count_all_i(const uint8_t* base, uint32_t* acc,
                                            std::integer_sequence<int, Ms...>) {
  ((acc[Ms] = count_i<C, B, shell_start(C::KIND, Ms), 0, shell_z(C::KIND, Ms)>(base)), ...);
}

template <class C, int... Ms>
__device__ __forceinline__ void count_all_j_fcc(const uint8_t* const* cls_base, uint32_t* acc,
                                                std::integer_sequence<int, Ms...>) {
  ((acc[Ms] = count_j_fcc<C, shell_start(C::KIND, Ms), 0, shell_z(C::KIND, Ms)>(cls_base)), ...);
}

// partner table entry e = b * Z1 + dir: (shared offset of the partner of a
// basis-b anchor in first-shell direction dir) * 4 + the partner's basis
template <class C, int E>
struct PartnerEntry {
  static constexpr int b = E / C::Z1, dir = E % C::Z1;
  static constexpr ShellVec v = shell_vec(C::KIND, dir);
  static constexpr int bj = basis_of_parity(C::KIND, (basis_comp(C::KIND, b, 0) + v.x) & 1,
                                            (basis_comp(C::KIND, b, 1) + v.y) & 1,
                                            (basis_comp(C::KIND, b, 2) + v.z) & 1);
  static constexpr int value = nbr_offset<C>(b, v.x, v.y, v.z) * 4 + bj;
};

template <class C, int... E>
__device__ __forceinline__ void fill_partner_table(int* s_part, std::integer_sequence<int, E...>) {
  ((s_part[E] = PartnerEntry<C, E>::value), ...);
}

// conventional-cell shift (dx, dy, dz) and basis of the partner of a basis-b
// anchor in first-shell direction dir
template <class C, int... E>
__device__ __forceinline__ void partner_shift_impl(int e, int* dx, int* dy, int* dz, int* bj,
                                                   std::integer_sequence<int, E...>) {
  ((e == E ? (*dx = floordiv2(basis_comp(C::KIND, PartnerEntry<C, E>::b, 0) + PartnerEntry<C, E>::v.x),
              *dy = floordiv2(basis_comp(C::KIND, PartnerEntry<C, E>::b, 1) + PartnerEntry<C, E>::v.y),
              *dz = floordiv2(basis_comp(C::KIND, PartnerEntry<C, E>::b, 2) + PartnerEntry<C, E>::v.z),
              *bj = PartnerEntry<C, E>::bj, 0)
           : 0),
   ...);
}

template <class C>
__device__ __forceinline__ void partner_shift(int b, int dir, int* dx, int* dy, int* dz, int* bj) {
  partner_shift_impl<C>(b * C::Z1 + dir, dx, dy, dz, bj,
                        std::make_integer_sequence<int, C::NB * C::Z1>{});
}

// sigma of each byte of a word of codes sigma * W: W = 8 a shift; W = 5
// (sigma <= 5) per 16-bit lane (code * 52) >> 8, exact for codes <= 25
template <int W>
__device__ __forceinline__ uint32_t codes_to_sigma(uint32_t w) {
  if constexpr (W == 8) {
    return (w >> 3) & 0x1F1F1F1Fu;
  } else {
    const uint32_t even = (((w & 0x00FF00FFu) * 52u) >> 8) & 0x00FF00FFu;
    const uint32_t odd = ((((w >> 8) & 0x00FF00FFu) * 52u) >> 8) & 0x00FF00FFu;
    return even | (odd << 8);
  }
}
template <int W>
__device__ __forceinline__ uint32_t code_to_sigma(uint32_t c) {
  if constexpr (W == 8) return c >> 3;
  else return (c * 52u) >> 8;
}

// ---- bulk copies (TMA) completed on an mbarrier --------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(bar), "r"(count) : "memory");
  // make the initialised barrier visible to the bulk-copy (async) proxy
  asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
  asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
}
// arrival of the barrier's single expected arrival, announcing `bytes` of
// copies that complete on it
__device__ __forceinline__ void mbar_arrive_expect(uint32_t bar, uint32_t bytes) {
  asm volatile("{\n .reg .b64 st;\n mbarrier.arrive.expect_tx.shared::cta.b64 st, [%0], %1;\n}\n"
               ::"r"(bar), "r"(bytes) : "memory");
}
// global -> shared bulk copy: both addresses 16-byte aligned, bytes a
// multiple of 16
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n"
      ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, uint32_t parity) {
  uint32_t done;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(done) : "r"(bar), "r"(parity) : "memory");
  return done != 0;
}
__device__ __forceinline__ unsigned long long tiled_globaltimer() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// waits for phase `parity` of the barrier, giving up after about a second
// (%globaltimer) or 2^24 polls; returns whether it completed
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, uint32_t parity) {
  const unsigned long long t0 = tiled_globaltimer();
  for (uint32_t i = 0; i < (1u << 24); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if ((i & 63u) == 63u && tiled_globaltimer() - t0 > 1000000000ull) break;
  }
  return false;
}

template <class C>
__global__ void __launch_bounds__(C::NT, C::MINB) k_sweep_tiled(const __grid_constant__ Geom g,
                                                       const PhaseArgs a,
                                                       const __grid_constant__ Tables tab,
                                                       uint8_t* __restrict__ occ,
                                                       const uint32_t* __restrict__ dtab,
                                                       unsigned long long* __restrict__ stats) {
  extern __shared__ __align__(16) uint8_t smem[];
  uint32_t* s_tab = reinterpret_cast<uint32_t*>(smem);                      // 1536 words
  uint8_t* s_d = smem + 4 * kTabWords;                                      // DBYTES
  int* s_part = reinterpret_cast<int*>(s_d + C::DBYTES);                    // NB * Z1
  int* s_gpart = s_part + C::NB * C::Z1;                                    // NB * Z1
  uint64_t* s_bar = reinterpret_cast<uint64_t*>(smem + C::MBAR_OFF);        // staging barrier
  uint8_t* tile = smem + C::TILE_OFF;

  const int tid = threadIdx.x;
  const int lane = tid & 31, warp = tid >> 5;
  constexpr int NW = C::NT / 32;
  const int bit[3] = {a.colour & 1, (a.colour >> 1) & 1, (a.colour >> 2) & 1};
  const int bidx[3] = {static_cast<int>(blockIdx.x), static_cast<int>(blockIdx.y),
                       static_cast<int>(blockIdx.z)};
  constexpr int Bsz[3] = {C::BX, C::BY, C::BZ};

  int lo[3], ext[3], g0[3], a_first[3], a_last[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    a_first[d] = bidx[d] * Bsz[d] + (d == 2 ? a.az0 : 0);
    a_last[d] = min(a_first[d] + Bsz[d], d == 2 ? a.az0 + a.naz : g.m[d] / 2) - 1;
    const int c0 = 2 * a_first[d] + bit[d], c1 = 2 * a_last[d] + bit[d];
    lo[d] = link_bound(g, d, c0) - C::H;
    ext[d] = link_bound(g, d, c1 + 1) + C::H - lo[d];
    int v = lo[d] + a.shift[d];
    v += v < 0 ? g.n[d] : 0;
    v -= v >= g.n[d] ? g.n[d] : 0;
    g0[d] = v;
  }
  const bool wrap_x = g0[0] + ext[0] > g.n[0];
  const bool wrap_any = wrap_x || g0[1] + ext[1] > g.n[1] || g0[2] + ext[2] > g.n[2];
  // device storage: rows of px bytes, the z step and the basis-row step
  const long long zstr = static_cast<long long>(g.n[1]) * g.px;
  const long long gstr = zstr * g.n[2];
  // accepted swaps are stored at once with 32-bit offsets (8-bit storage, no
  // wrap, fewer than 2^31 bytes of storage); otherwise the tile is written
  // back at the end
  const bool direct = !C::PACK4 && !wrap_any && gstr * C::NB < (1ll << 31);
  // staging: bulk copies of the 16-byte aligned span of each sub-row when
  // it fits the tile row, else 8-byte copies; the tile's x origin `off` is
  // the global x of its first site modulo the copy alignment
  const bool bulk = C::BULK && a.staging == 0 && !wrap_x && (g0[0] & 15) + ext[0] <= C::XW;
  const int off = bulk ? (g0[0] & 15) : (g0[0] & 7);

  // ---- tables ------------------------------------------------------------
  for (int w = tid; w < kTabWords; w += C::NT) s_tab[w] = tab.w[w];
  for (int w = tid; w < C::DBYTES / 4; w += C::NT)
    reinterpret_cast<uint32_t*>(s_d)[w] = dtab[w];
  if (tid == 0) fill_partner_table<C>(s_part, std::make_integer_sequence<int, C::NB * C::Z1>{});
  // storage offset of the partner from its anchor (8-bit storage, no wrap)
  if (tid < C::NB * C::Z1) {
    const int b = tid / C::Z1, dir = tid % C::Z1;
    int dx = 0, dy = 0, dz = 0, bj = 0;
    partner_shift<C>(b, dir, &dx, &dy, &dz, &bj);
    s_gpart[tid] = static_cast<int>(dx + dy * static_cast<long long>(g.px) + dz * zstr +
                                    (bj - b) * gstr);
  }

  // ---- stage the tile ----------------------------------------------------
  // sub-row index sub = (tz * ext_y + ty) * G + grp; tz = sub / (G ext_y) by a
  // 16-bit reciprocal (exact: sub < 2^16 / 64, ext_y < 64)
  const int n_sub = ext[1] * ext[2] * C::G;
  const int ext_y = ext[1];
  const uint32_t inv_ey = (65536u + ext_y - 1) / ext_y;
  auto sub_row = [=](int sub, int* grp, int* ty, int* tz) {
    *grp = sub % C::G;
    const int t = sub / C::G;
    *tz = static_cast<int>((static_cast<uint32_t>(t) * inv_ey) >> 16);
    *ty = t - *tz * ext_y;
  };
  const int g0y = g0[1], g0z = g0[2];
  const int ny = g.n[1], nz = g.n[2];
  const size_t px = static_cast<size_t>(g.px);
  auto grow = [=](int grp, int ty, int tz) -> size_t {
    int gy = g0y + ty;
    gy -= gy >= ny ? ny : 0;
    int gz = g0z + tz;
    gz -= gz >= nz ? nz : 0;
    return ((static_cast<size_t>(grp) * nz + gz) * ny + gy) * px;
  };
  if (bulk) {
    // one bulk copy per sub-row (packed storage: the packed row lands in
    // the odd basis's sub-row and is unpacked in place below)
    const uint32_t bar = smem_u32(s_bar);
    const uint32_t bytes = static_cast<uint32_t>(round_up(off + ext[0], 16));
    if (tid == 0) {
      mbar_init(bar, 1);
      mbar_arrive_expect(bar, bytes * static_cast<uint32_t>(n_sub));
    }
    __syncthreads();
    const uint8_t* src0 = occ + (g0[0] - off);
    const uint32_t tbase = smem_u32(tile);
    for (int sub = tid; sub < n_sub; sub += C::NT) {
      int grp, ty, tz;
      sub_row(sub, &grp, &ty, &tz);
      const int slot = C::PACK4 ? 2 * grp + 1 : grp;
      bulk_g2s(tbase + tz * C::PS + ty * C::RS + slot * C::XW, src0 + grow(grp, ty, tz), bytes,
               bar);
    }
    bool done = mbar_wait_bounded(bar, 0);
    if (!done) {
      // report it, and do not leave while copies into this block's shared
      // memory may still be in flight
      atomicOr(stats + kStatWait, 1ull);
      done = mbar_wait_bounded(bar, 0);
    }
    if (__syncthreads_or(!done)) return;  // the whole block leaves together
    if constexpr (C::PACK4) {
      // unpack 16 packed bytes (two sites each) per step: low nibbles to
      // the even basis's sub-row, high nibbles in place
      const int nc = static_cast<int>(bytes >> 4);  // 16-byte chunks per sub-row (<= 32)
      const int rpi = 32 / nc;
      const int my_r = lane / nc, my_c = lane - (lane / nc) * nc;
      for (int base = warp * rpi; base < n_sub; base += NW * rpi) {
        const int sub = base + my_r;
        if (my_r >= rpi || sub >= n_sub) continue;
        int grp, ty, tz;
        sub_row(sub, &grp, &ty, &tz);
        uint8_t* row = tile + tz * C::PS + ty * C::RS + 16 * my_c;
        const uint4 v = *reinterpret_cast<const uint4*>(row + (2 * grp + 1) * C::XW);
        const uint4 lo4 = make_uint4((v.x & 0x0F0F0F0Fu) * C::W, (v.y & 0x0F0F0F0Fu) * C::W,
                                     (v.z & 0x0F0F0F0Fu) * C::W, (v.w & 0x0F0F0F0Fu) * C::W);
        const uint4 hi4 = make_uint4(((v.x >> 4) & 0x0F0F0F0Fu) * C::W,
                                     ((v.y >> 4) & 0x0F0F0F0Fu) * C::W,
                                     ((v.z >> 4) & 0x0F0F0F0Fu) * C::W,
                                     ((v.w >> 4) & 0x0F0F0F0Fu) * C::W);
        *reinterpret_cast<uint4*>(row + (2 * grp) * C::XW) = lo4;
        *reinterpret_cast<uint4*>(row + (2 * grp + 1) * C::XW) = hi4;
      }
    }
  } else if (!wrap_x) {
    const int n8 = (off + ext[0] + 7) >> 3;  // 8-byte chunks per sub-row (<= 32)
    const int rpi = 32 / n8;                 // sub-rows per warp pass
    const int my_r = lane / n8, my_c = lane - (lane / n8) * n8;
    const uint8_t* src0 = occ + (g0[0] - off) + 8 * my_c;
    if constexpr (!C::PACK4) {
      // asynchronous 8-byte global -> shared copies, all in flight at once
      const uint32_t sbase = static_cast<uint32_t>(__cvta_generic_to_shared(tile)) + 8 * my_c;
      for (int base = warp * rpi; base < n_sub; base += NW * rpi) {
        const int sub = base + my_r;
        if (my_r < rpi && sub < n_sub) {
          int grp, ty, tz;
          sub_row(sub, &grp, &ty, &tz);
          const uint32_t dst = sbase + tz * C::PS + ty * C::RS + grp * C::XW;
          asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(dst),
                       "l"(src0 + grow(grp, ty, tz))
                       : "memory");
        }
      }
      asm volatile("cp.async.wait_all;\n" ::: "memory");
    } else {
      for (int base = warp * rpi; base < n_sub; base += NW * rpi) {
        const int sub = base + my_r;
        if (my_r < rpi && sub < n_sub) {
          int grp, ty, tz;
          sub_row(sub, &grp, &ty, &tz);
          const uint2 v = *reinterpret_cast<const uint2*>(src0 + grow(grp, ty, tz));
          uint8_t* row = tile + tz * C::PS + ty * C::RS + 8 * my_c;
          const uint2 lo4 = make_uint2((v.x & 0x0F0F0F0Fu) * C::W, (v.y & 0x0F0F0F0Fu) * C::W);
          const uint2 hi4 = make_uint2(((v.x >> 4) & 0x0F0F0F0Fu) * C::W,
                                       ((v.y >> 4) & 0x0F0F0F0Fu) * C::W);
          *reinterpret_cast<uint2*>(row + (2 * grp) * C::XW) = lo4;
          *reinterpret_cast<uint2*>(row + (2 * grp + 1) * C::XW) = hi4;
        }
      }
    }
  } else {
    // the tile's x range crosses the periodic seam: byte copies, one warp per
    // sub-row
    for (int sub = warp; sub < n_sub; sub += NW) {
      int grp, ty, tz;
      sub_row(sub, &grp, &ty, &tz);
      const uint8_t* src = occ + grow(grp, ty, tz);
      uint8_t* row = tile + tz * C::PS + ty * C::RS + off;
      for (int tx = lane; tx < ext[0]; tx += 32) {
        int gx = g0[0] + tx;
        gx -= gx >= g.n[0] ? g.n[0] : 0;
        const uint8_t v = src[gx];
        if constexpr (!C::PACK4) {
          row[grp * C::XW + tx] = v;
        } else {
          row[(2 * grp) * C::XW + tx] = static_cast<uint8_t>((v & 15) * C::W);
          row[(2 * grp + 1) * C::XW + tx] = static_cast<uint8_t>((v >> 4) * C::W);
        }
      }
    }
  }
  __syncthreads();

  // ---- trials ------------------------------------------------------------
  uint32_t n_att = 0, n_unl = 0, n_acc = 0;
  int64_t sum_de = 0;
  const int la[3] = {tid % C::BX, (tid / C::BX) % C::BY, tid / (C::BX * C::BY)};
  const int ac[3] = {a_first[0] + la[0], a_first[1] + la[1], a_first[2] + la[2]};
  if (ac[0] <= a_last[0] && ac[1] <= a_last[1] && ac[2] <= a_last[2]) {
    int o[3], l[3], c[3];
#pragma unroll
    for (int d = 0; d < 3; ++d) {
      c[d] = 2 * ac[d] + bit[d];
      const int b0 = link_bound(g, d, c[d]);
      o[d] = b0 - lo[d];
      l[d] = link_bound(g, d, c[d] + 1) - b0;
    }
    const uint32_t cid = (static_cast<uint32_t>(c[2]) * g.m[1] + c[1]) * g.m[0] + c[0];
    n_att = static_cast<uint32_t>(l[0] * l[1] * l[2] * C::NB);

    // storage offset of this cell's first site (direct stores only)
    const uint32_t gcell = direct ? static_cast<uint32_t>(
        (static_cast<long long>(g0[2] + o[2]) * g.n[1] + (g0[1] + o[1])) * g.px + (g0[0] + o[0]))
        : 0u;

    auto attempt = [&](auto bconst, int ai, uint32_t gi, uint32_t wa, uint32_t wb) {
      constexpr int B = decltype(bconst)::value;
      const uint32_t dir = __umulhi(wa, static_cast<uint32_t>(C::Z1));
      const int pt = s_part[B * C::Z1 + dir];
      const int aj = ai + (pt >> 2);
      const uint32_t p = tile[ai], q = tile[aj];
      // a like pair is a no-op trial (Sec. 2.1): its lanes issue none of the
      // neighbourhood loads below, which also thins the partner-side bank
      // conflicts of the lanes that do
      if (p == q) return;
      ++n_unl;
      uint32_t acc_i[C::M], acc_j[C::M];
      count_all_i<C, B>(tile + ai, acc_i, std::make_integer_sequence<int, C::M>{});
      if constexpr (C::KIND == 0) {
        count_all_i<C, 1 - B>(tile + aj, acc_j, std::make_integer_sequence<int, C::M>{});
      } else {
        const int bj = pt & 3;
        const uint8_t* cls_base[4];
#pragma unroll
        for (int cl = 0; cl < 4; ++cl) {
          const int c01 = (bj & 1) ? corr_of<C>(1, cl) : corr_of<C>(0, cl);
          const int c23 = (bj & 1) ? corr_of<C>(3, cl) : corr_of<C>(2, cl);
          cls_base[cl] = tile + aj + ((bj & 2) ? c23 : c01);
        }
        count_all_j_fcc<C>(cls_base, acc_j, std::make_integer_sequence<int, C::M>{});
      }
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
      // Metropolis (Sec. 2.1, Eq. 3) without branches: the table lookups are
      // clamped in range and only matter when dE > 0 in normal mode
      const uint64_t idx = static_cast<uint64_t>(de) >> a.s;
      const uint32_t i2 = idx >> 18 < 511u ? static_cast<uint32_t>(idx >> 18) : 511u;
      const uint32_t thr = compose_threshold(s_tab[idx & 511u], s_tab[512 + ((idx >> 9) & 511u)],
                                             s_tab[1024 + i2]);
      const bool ok = de <= 0 || a.mode == kModeAcceptAll ||
                      (a.mode == kModeNormal && idx < (1ull << 27) && wb < thr);
      if (ok) {
        tile[ai] = static_cast<uint8_t>(q);
        tile[aj] = static_cast<uint8_t>(p);
        if (direct) {
          occ[gi] = static_cast<uint8_t>(q);
          occ[gi + s_gpart[B * C::Z1 + dir]] = static_cast<uint8_t>(p);
        }
        ++n_acc;
        sum_de += de;
      }
    };

    for (int zr = 0; zr < l[2]; ++zr)
      for (int yr = 0; yr < l[1]; ++yr) {
        const int rb = off + (o[2] + zr) * C::PS + (o[1] + yr) * C::RS + o[0];
        const uint32_t grb = gcell + static_cast<uint32_t>(zr * zstr + yr * g.px);
        const uint32_t cc0 = static_cast<uint32_t>((zr * l[1] + yr) * l[0]);
        for (int xr = 0; xr < l[0]; ++xr) {
          const uint32_t cc = cc0 + xr;
          const int ai = rb + xr;
          const uint32_t gi = grb + xr;
          const uint32_t gs = static_cast<uint32_t>(gstr);
          const U4 w0 = philox4x32_10_rk(cc * (C::NB / 2), cid, a.t, 0u, g.rk);
          attempt(std::integral_constant<int, 0>{}, ai, gi, w0.x, w0.y);
          attempt(std::integral_constant<int, 1>{}, ai + C::XW, gi + gs, w0.z, w0.w);
          if constexpr (C::NB == 4) {
            const U4 w1 = philox4x32_10_rk(cc * 2 + 1, cid, a.t, 0u, g.rk);
            attempt(std::integral_constant<int, 2>{}, ai + 2 * C::XW, gi + 2 * gs, w1.x, w1.y);
            attempt(std::integral_constant<int, 3>{}, ai + 3 * C::XW, gi + 3 * gs, w1.z, w1.w);
          }
        }
      }
  }

  // ---- write back --------------------------------------------------------
  // Tiles whose accepted swaps changed only the tile (packed storage, tiles
  // across a periodic seam).  The sites a block's trials can have changed
  // lie within one conventional cell of its link cells (a partner is one
  // half unit from its anchor): tile indices [1, ext - 1) along every axis,
  // the cells starting H = 2 in.  No other link cell of this colour writes
  // there (the edge rule that keeps their interaction zones apart, Sec.
  // 2.2), so the region is stored whole; its sites that no trial changed get
  // back the value they already hold.
  if (!direct) {
    __syncthreads();
    const int wy = ext[1] - 2;
    const int n_wsub = wy * (ext[2] - 2) * C::G;
    const uint32_t inv_wy = (65536u + wy - 1) / wy;  // exact as inv_ey above
    auto wsub_row = [=](int sub, int* grp, int* ty, int* tz) {
      *grp = sub % C::G;
      const int t = sub / C::G;
      const int z = static_cast<int>((static_cast<uint32_t>(t) * inv_wy) >> 16);
      *tz = z + 1;
      *ty = t - z * wy + 1;
    };
    // the stored value of byte t of the sub-row of group grp
    auto stored = [&](const uint8_t* row, int grp, int t) -> uint32_t {
      if constexpr (!C::PACK4) {
        return row[grp * C::XW + t];
      } else {
        return code_to_sigma<C::W>(row[(2 * grp) * C::XW + t]) |
               (code_to_sigma<C::W>(row[(2 * grp + 1) * C::XW + t]) << 4);
      }
    };
    const int a0 = off + 1, a1 = off + ext[0] - 1;  // shared bytes [a0, a1) of a sub-row
    if (!wrap_x) {
      // whole 8-byte chunks f0 .. f1-1 of the staging grid (shared offset 8c
      // <-> global g0x - off + 8c, both 8-byte aligned), spread over every
      // thread; then the partial chunks at the two ends, byte by byte
      // (a short tile row may hold one whole chunk or none: nf = 1 divides
      // exactly without the reciprocal, nf = 0 leaves only the two ends)
      const int f0 = (a0 + 7) >> 3, f1 = max(a1 >> 3, f0), nf = f1 - f0;
      const uint32_t inv_nf =
          nf > 1 ? static_cast<uint32_t>((0x100000000ull + nf - 1) / nf) : 0u;  // exact: jb nf < 2^32
      uint8_t* const gx0 = occ + (g0[0] - off);
      for (int jb = tid; jb < n_wsub * nf; jb += C::NT) {
        const int sub = nf == 1 ? jb : static_cast<int>(__umulhi(static_cast<uint32_t>(jb), inv_nf));
        const int c = f0 + jb - sub * nf;
        int grp, ty, tz;
        wsub_row(sub, &grp, &ty, &tz);
        const uint8_t* row = tile + tz * C::PS + ty * C::RS + 8 * c;
        uint2 v;
        if constexpr (!C::PACK4) {
          v = *reinterpret_cast<const uint2*>(row + grp * C::XW);
        } else {
          const uint2 lo4 = *reinterpret_cast<const uint2*>(row + (2 * grp) * C::XW);
          const uint2 hi4 = *reinterpret_cast<const uint2*>(row + (2 * grp + 1) * C::XW);
          v = make_uint2(codes_to_sigma<C::W>(lo4.x) | (codes_to_sigma<C::W>(hi4.x) << 4),
                         codes_to_sigma<C::W>(lo4.y) | (codes_to_sigma<C::W>(hi4.y) << 4));
        }
        *reinterpret_cast<uint2*>(gx0 + grow(grp, ty, tz) + 8 * c) = v;
      }
      for (int jb = tid; jb < 2 * n_wsub; jb += C::NT) {
        const int sub = jb >> 1;
        // the ends [a0, 8 f0) and [8 f1, a1), clipped to [a0, a1), at most 7
        // bytes each
        const int t0 = (jb & 1) ? max(8 * f1, a0) : a0, t1 = (jb & 1) ? a1 : min(8 * f0, a1);
        int grp, ty, tz;
        wsub_row(sub, &grp, &ty, &tz);
        const uint8_t* row = tile + tz * C::PS + ty * C::RS;
        uint8_t* dst = gx0 + grow(grp, ty, tz);
#pragma unroll
        for (int k = 0; k < 7; ++k)
          if (t0 + k < t1) dst[t0 + k] = static_cast<uint8_t>(stored(row, grp, t0 + k));
      }
    } else {
      // the tile's x range crosses the periodic seam: byte stores, one warp
      // per sub-row
      for (int sub = warp; sub < n_wsub; sub += NW) {
        int grp, ty, tz;
        wsub_row(sub, &grp, &ty, &tz);
        uint8_t* dst = occ + grow(grp, ty, tz);
        const uint8_t* row = tile + tz * C::PS + ty * C::RS;
        for (int t = a0 + lane; t < a1; t += 32) {
          int gx = g0[0] + (t - off);
          gx -= gx >= g.n[0] ? g.n[0] : 0;
          dst[gx] = static_cast<uint8_t>(stored(row, grp, t));
        }
      }
    }
  }
  warp_reduce_add_stats(stats, n_att, n_unl, n_acc, sum_de);
}

template <class C>
size_t smem_bytes(int ext_z) {
  return static_cast<size_t>(C::TILE_OFF) + static_cast<size_t>(C::PS) * ext_z;
}

// cells of colour bit `bit` along one dimension: the largest tile extent of
// any block whose first cell index is a_base + k bsz (for the dynamic
// shared-memory size)
inline int max_extent(int n, int m, int bsz, int halo, int a_base = 0) {
  const int A = m / 2;
  int best = 0;
  for (int bit = 0; bit < 2; ++bit)
    for (int a0 = a_base; a0 < A; a0 += bsz) {
      const int a1 = (a0 + bsz < A ? a0 + bsz : A) - 1;
      const int c0 = 2 * a0 + bit, c1 = 2 * a1 + bit;
      const int lo = static_cast<int>((static_cast<long long>(c0) * n) / m) - halo;
      const int hi = static_cast<int>((static_cast<long long>(c1 + 1) * n) / m) + halo;
      best = hi - lo > best ? hi - lo : best;
    }
  return best;
}

template <class C>
bool supported(const Geom& g) {
  if (g.kind != C::KIND || g.M != C::M || g.L != C::L || g.pack4 != (C::PACK4 ? 1 : 0)) return false;
  if (g.K > C::KMAX || code_width(g.K) != (g.pack4 ? code_width(g.K) : C::W)) return false;
  if (C::KMAX == 6 && g.K != 6) return false;
  const int Bsz[3] = {C::BX, C::BY, C::BZ};
  const int EXT[3] = {C::EXT_X, C::EXT_Y, C::EXT_Z};
  for (int d = 0; d < 3; ++d) {
    if (g.m[d] < 4) return false;
    if (g.m[d] / 2 < Bsz[d] + 1) return false;  // a tile never wraps onto itself
    if (max_extent(g.n[d], g.m[d], Bsz[d], C::H) > EXT[d]) return false;
  }
  return smem_bytes<C>(max_extent(g.n[2], g.m[2], C::BZ, C::H)) <= 227 * 1024;
}

template <class C>
cudaError_t launch_cfg(const Geom& g, const PhaseArgs& a, const Tables& tab, uint8_t* occ,
                       const TiledEpi& epi, unsigned long long* stats, cudaStream_t st) {
  const int ext_z = max_extent(g.n[2], g.m[2], C::BZ, C::H, a.az0);
  const size_t smem = smem_bytes<C>(ext_z);
  if (a.naz <= 0 || a.az0 < 0 || a.az0 + a.naz > g.m[2] / 2) return cudaErrorInvalidValue;
  if (smem > 227 * 1024) return cudaErrorNotSupported;
  cudaError_t e = cudaFuncSetAttribute(k_sweep_tiled<C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  const dim3 grid((g.m[0] / 2 + C::BX - 1) / C::BX, (g.m[1] / 2 + C::BY - 1) / C::BY,
                  (a.naz + C::BZ - 1) / C::BZ);
  k_sweep_tiled<C><<<grid, C::NT, smem, st>>>(g, a, tab, occ, epi.d_table, stats);
  return cudaGetLastError();
}

}  // namespace tiled
}  // namespace smcx
