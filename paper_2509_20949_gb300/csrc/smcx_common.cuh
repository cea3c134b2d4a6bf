// smcx_common.cuh -- definitions shared by the library's host code and kernels.
//
// Geometry (half-unit shell vectors of BCC/FCC, basis vectors), the
// Philox4x32-10 generator and the launch-parameter structs.  The oracle under
// oracle/ has its own independent versions of all of these.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace smcx {

constexpr int kMaxShells = 4;
constexpr int kMaxShellVecs = 64;  // BCC shells 1-4: 50 vectors, FCC: 54
constexpr int kTabWords = 3 * 512; // Metropolis threshold tables T_0, T_1, T_2

enum AcceptMode : int { kModeNormal = 0, kModeAcceptAll = 1, kModeZeroT = 2 };

// ---------------------------------------------------------------------------
// Neighbour shells in half units h = a/2, shells in ascending distance, the
// vectors of one shell sorted lexicographically on (dx, dy, dz).
// BCC: |d|^2 = 3 (8), 4 (6), 8 (12), 11 (24).  FCC: 2 (12), 4 (6), 6 (24), 8 (12).
// ---------------------------------------------------------------------------
struct ShellVec { int8_t x, y, z; };

// Tables are function-local so that host code and device code (after
// unrolling, with constant indices) can both use them.
__host__ __device__ constexpr int shell_z(int kind, int m) {
  constexpr int bcc[4] = {8, 6, 12, 24};
  constexpr int fcc[4] = {12, 6, 24, 12};
  return kind == 0 ? bcc[m] : fcc[m];
}

__host__ __device__ constexpr ShellVec shell_vec(int kind, int idx) {
  constexpr ShellVec bcc[50] = {
      // shell 1: (+-1,+-1,+-1)
      {-1, -1, -1}, {-1, -1, 1}, {-1, 1, -1}, {-1, 1, 1}, {1, -1, -1}, {1, -1, 1}, {1, 1, -1}, {1, 1, 1},
      // shell 2: permutations of (+-2,0,0)
      {-2, 0, 0}, {0, -2, 0}, {0, 0, -2}, {0, 0, 2}, {0, 2, 0}, {2, 0, 0},
      // shell 3: permutations of (+-2,+-2,0)
      {-2, -2, 0}, {-2, 0, -2}, {-2, 0, 2}, {-2, 2, 0}, {0, -2, -2}, {0, -2, 2},
      {0, 2, -2}, {0, 2, 2}, {2, -2, 0}, {2, 0, -2}, {2, 0, 2}, {2, 2, 0},
      // shell 4: permutations of (+-3,+-1,+-1)
      {-3, -1, -1}, {-3, -1, 1}, {-3, 1, -1}, {-3, 1, 1},
      {-1, -3, -1}, {-1, -3, 1}, {-1, -1, -3}, {-1, -1, 3}, {-1, 1, -3}, {-1, 1, 3}, {-1, 3, -1}, {-1, 3, 1},
      {1, -3, -1}, {1, -3, 1}, {1, -1, -3}, {1, -1, 3}, {1, 1, -3}, {1, 1, 3}, {1, 3, -1}, {1, 3, 1},
      {3, -1, -1}, {3, -1, 1}, {3, 1, -1}, {3, 1, 1},
  };
  constexpr ShellVec fcc[54] = {
      // shell 1: permutations of (+-1,+-1,0)
      {-1, -1, 0}, {-1, 0, -1}, {-1, 0, 1}, {-1, 1, 0}, {0, -1, -1}, {0, -1, 1},
      {0, 1, -1}, {0, 1, 1}, {1, -1, 0}, {1, 0, -1}, {1, 0, 1}, {1, 1, 0},
      // shell 2: permutations of (+-2,0,0)
      {-2, 0, 0}, {0, -2, 0}, {0, 0, -2}, {0, 0, 2}, {0, 2, 0}, {2, 0, 0},
      // shell 3: permutations of (+-2,+-1,+-1)
      {-2, -1, -1}, {-2, -1, 1}, {-2, 1, -1}, {-2, 1, 1},
      {-1, -2, -1}, {-1, -2, 1}, {-1, -1, -2}, {-1, -1, 2}, {-1, 1, -2}, {-1, 1, 2}, {-1, 2, -1}, {-1, 2, 1},
      {1, -2, -1}, {1, -2, 1}, {1, -1, -2}, {1, -1, 2}, {1, 1, -2}, {1, 1, 2}, {1, 2, -1}, {1, 2, 1},
      {2, -1, -1}, {2, -1, 1}, {2, 1, -1}, {2, 1, 1},
      // shell 4: permutations of (+-2,+-2,0)
      {-2, -2, 0}, {-2, 0, -2}, {-2, 0, 2}, {-2, 2, 0}, {0, -2, -2}, {0, -2, 2},
      {0, 2, -2}, {0, 2, 2}, {2, -2, 0}, {2, 0, -2}, {2, 0, 2}, {2, 2, 0},
  };
  return kind == 0 ? bcc[idx] : fcc[idx];
}

__host__ __device__ constexpr int basis_count(int kind) { return kind == 0 ? 2 : 4; }

// basis vector component c of basis site b (half units)
__host__ __device__ constexpr int basis_comp(int kind, int b, int c) {
  return kind == 0 ? b : (b == 0 ? 0 : (c == b - 1 ? 0 : 1));
}

// basis index of a parity vector (px, py, pz); -1 when not a lattice site
__host__ __device__ constexpr int basis_of_parity(int kind, int px, int py, int pz) {
  if (kind == 0) return (px == py && py == pz) ? px : -1;
  if (((px + py + pz) & 1) != 0) return -1;
  if (px == 0 && py == 0 && pz == 0) return 0;
  return px == 0 ? 1 : (py == 0 ? 2 : 3);
}

__host__ __device__ constexpr int shell_start(int kind, int m) {
  int s = 0;
  for (int i = 0; i < m; ++i) s += shell_z(kind, i);
  return s;
}


// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC11): per round two 32x32
// multiplications by fixed odd constants; the high halves are xor-ed with
// the untouched counter words and the round key; the key advances by two Weyl
// increments between rounds.
// ---------------------------------------------------------------------------
struct U4 { uint32_t x, y, z, w; };

__host__ __device__ __forceinline__ uint32_t mulhi32(uint32_t a, uint32_t b) {
#ifdef __CUDA_ARCH__
  return __umulhi(a, b);
#else
  return static_cast<uint32_t>((static_cast<uint64_t>(a) * b) >> 32);
#endif
}

__host__ __device__ __forceinline__ U4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2,
                                                     uint32_t c3, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a_lo = 0xD2511F53u * c0, a_hi = mulhi32(0xD2511F53u, c0);
    const uint32_t b_lo = 0xCD9E8D57u * c2, b_hi = mulhi32(0xCD9E8D57u, c2);
    const uint32_t n0 = b_hi ^ c1 ^ k0;
    const uint32_t n2 = a_hi ^ c3 ^ k1;
    c0 = n0;
    c1 = b_lo;
    c2 = n2;
    c3 = a_lo;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  return U4{c0, c1, c2, c3};
}

// Metropolis threshold: exp(-beta dE) scaled by 2^32, from three 512-entry
// tables indexed by the bin index idx = dE >> s (dE > 0, idx < 2^27).
__host__ __device__ __forceinline__ uint32_t compose_threshold(uint32_t t0, uint32_t t1,
                                                              uint32_t t2) {
  return mulhi32(mulhi32(t0, t1), t2);
}

// ---------------------------------------------------------------------------
// Launch parameters.
// ---------------------------------------------------------------------------
// Device storage of the occupancy (internal; the C ABI exchanges the
// canonical layout).  Rows of px bytes (n_x rounded up to 16) ordered
// [group][z][y]:
//   8-bit: group = basis site b, byte x holds the code sigma * W of site
//          (x, y, z, b) -- W is the bit position step of the one-hot species
//          counters of the tiled and cell sweeps (8 for K <= 5: species s
//          counted in byte s, species 4 shifted out; 5 for K = 6; 1 above);
//   4-bit: group = basis pair b/2, byte x holds sigma of b even in the low
//          and of b odd in the high nibble (both sites of one conventional
//          cell, so no two link cells ever write one byte).
struct Geom {
  int kind, nb;
  int n[3];
  int m[3];       // link cells per dimension (even, or 1)
  int L;          // nominal cell edge (conventional cells)
  int K, M;       // species, shells in use
  int z1;         // first-shell coordination
  int pack4;      // occupancy stored two sites per byte
  int px;         // device row pitch in bytes (multiple of 16)
  int W;          // code multiplier of 8-bit storage
  uint32_t seed_lo, seed_hi;
  uint32_t rk[10][2];  // Philox round keys of the seed (host-precomputed)
  // link-cell bounds floor(c n_d / m_d) = c q_d + floor(c r_d / m_d) with
  // n_d = q_d m_d + r_d; the last term is umulhi(c r_d, bmag_d) with
  // bmag_d = ceil(2^32 / m_d), exact while c r_d < m_d^2 < 2^32 / m_d
  // (m_d <= 1600; bmag_d = 0 selects a 64-bit division)
  uint32_t bq[3], br[3], bmag[3];
};

__host__ __device__ __forceinline__ int link_bound(const Geom& g, int d, int c) {
  if (g.bmag[d])
    return static_cast<int>(static_cast<uint32_t>(c) * g.bq[d] +
                            mulhi32(static_cast<uint32_t>(c) * g.br[d], g.bmag[d]));
  return static_cast<int>((static_cast<long long>(c) * g.n[d]) / g.m[d]);
}

// Philox4x32-10 with the ten round keys precomputed (same generator as
// philox4x32_10; the key schedule is a pure function of the seed).
__host__ __device__ __forceinline__ U4 philox4x32_10_rk(uint32_t c0, uint32_t c1, uint32_t c2,
                                                        uint32_t c3, const uint32_t (*rk)[2]) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    const uint32_t a_lo = 0xD2511F53u * c0, a_hi = mulhi32(0xD2511F53u, c0);
    const uint32_t b_lo = 0xCD9E8D57u * c2, b_hi = mulhi32(0xCD9E8D57u, c2);
    const uint32_t n0 = b_hi ^ c1 ^ rk[r][0];
    const uint32_t n2 = a_hi ^ c3 ^ rk[r][1];
    c0 = n0;
    c1 = b_lo;
    c2 = n2;
    c3 = a_lo;
  }
  return U4{c0, c1, c2, c3};
}

__host__ __device__ inline int code_width(int K) { return K <= 5 ? 8 : (K == 6 ? 5 : 1); }

__host__ __device__ inline size_t dev_row(const Geom& g, int grp, int z, int y) {
  return ((static_cast<size_t>(grp) * g.n[2] + z) * g.n[1] + y) * static_cast<size_t>(g.px);
}

struct PhaseArgs {
  uint32_t t;      // global sweep index
  int shift[3];    // link-cell origin of this sweep
  int colour;      // 0..7
  int mode, s;     // acceptance mode, bin shift
  // active link cells of this colour along z: indices a in [az0, az0 + naz)
  // of the cells c_z = 2 a + (colour >> 2 & 1) (all of them unless a run is
  // restricted to a range of z planes of cells)
  int az0, naz;
  int staging;     // tiled kernel: 0 = bulk copies where they fit, 1 = 8-byte copies only
};

struct Tables {
  uint32_t w[kTabWords];
};

// Device-side statistics block inside the workspace: [0..3] this call,
// [4..7] since the running energy was last (re)started, [8] upload
// validation flag, [9] set when a device wait of a sweep kernel gave up
// (sticky until the host reads it).
constexpr int kStatCall = 0;
constexpr int kStatCum = 4;
constexpr int kStatStatus = 8;
constexpr int kStatWait = 9;

// Shell vectors of one lattice kind for device lookups (generic kernels).
struct ShellParam {
  int8_t v[kMaxShellVecs][3];
  int start[kMaxShells + 1];
};

// Local-energy model (the nonlinear short-range model of Sec. 3): per-site
// energies eps(i) = sum_m sum_s T_m[s_i][s][c_{i,m,s}] of the shell-resolved
// species counts, at most 3 shells and 8 species.  A trial recomputes eps on
// every distinct site of U = {i, j} u shells(i) u shells(j); u[dir] lists
// those sites as displacements from i (half units) for partner direction dir,
// which are distinct sites when every n_d >= 4.
constexpr int kLocalMaxShells = 3;
constexpr int kLocalMaxK = 8;
constexpr int kLocalMaxV = 42;                // FCC shells 1-3: 12 + 6 + 24
constexpr int kLocalMaxU = 2 + 2 * kLocalMaxV;
constexpr int kLocalMaxZ1 = 12;
constexpr int kLocalMaxZT = 25;               // 1 + the largest z_m in use
constexpr int64_t kLocalMaxAbsT = int64_t(1) << 48;
// u[dir][0] = 0 (the site i) and u[dir][1] = the partner j; for the others,
// shells_i / shells_j: bit m set when i / j is in shell m+1 of that site.
// The items list, per direction, every (site e of U, shell m+1) in which
// exactly one of i, j lies, sorted by shell: item_m = m | (j's shell) << 2.
// Every direction has the same items per shell (the directions are images of
// one another under the point group), so item x scans the same shell for
// every direction.
constexpr int kLocalMaxItems = 2 * kLocalMaxU;
struct LocalParam {
  int M, K, zt, total;
  int start[kLocalMaxShells + 1];
  int n_u[kLocalMaxZ1];
  int n_items;
  int8_t v[kLocalMaxV][3];
  int8_t u[kLocalMaxZ1][kLocalMaxU][3];
  uint8_t shells_i[kLocalMaxZ1][kLocalMaxU];
  uint8_t shells_j[kLocalMaxZ1][kLocalMaxU];
  // not copied to shared memory by the sweep kernel (read once per block)
  uint8_t item_e[kLocalMaxZ1][kLocalMaxItems];
  uint8_t item_m[kLocalMaxZ1][kLocalMaxItems];
};

}  // namespace smcx
