// kernels.h -- host-side launchers of the library's CUDA kernels.
#pragma once

#include "smcx_common.cuh"

namespace smcx {

cudaError_t launch_sweep_generic(const Geom& g, const PhaseArgs& a, const ShellParam& sp,
                                 const Tables& tab, uint8_t* occ, const int64_t* V,
                                 unsigned long long* stats, cudaStream_t st);

cudaError_t launch_pair_count_generic(const Geom& g, const ShellParam& sp, int n_shells,
                                      const uint8_t* occ, unsigned long long* counts,
                                      uint32_t n_cells, int n_sm, cudaStream_t st);

// (skip: device flag; the conversion does nothing when it is non-zero)
cudaError_t launch_canon_to_dev(const Geom& g, const uint8_t* canon, uint8_t* occ,
                                uint32_t n_cells, int n_sm, cudaStream_t st,
                                const unsigned int* skip = nullptr);
cudaError_t launch_dev_to_canon(const Geom& g, const uint8_t* occ, uint8_t* canon,
                                uint32_t n_cells, int n_sm, cudaStream_t st);
cudaError_t launch_validate(const uint8_t* canon, uint64_t n, uint32_t K, unsigned int* flag,
                            int n_sm, cudaStream_t st);

cudaError_t launch_philox_fill(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3, uint64_t key,
                               uint32_t n, uint32_t* out, cudaStream_t st);

// ---- tiled sweep (shared-memory tiles + halos) ---------------------------
// Per-(p, q) rows of the energy-difference table used by the tiled kernel.
struct TiledEpi {
  int kmax;        // 5 or 6 (species classes compiled)
  const uint32_t* d_table;
};

// Returns cudaErrorNotSupported (without launching) when no compiled tile
// shape fits the lattice; the caller then uses the generic kernel.
cudaError_t launch_sweep_tiled(const Geom& g, const PhaseArgs& a, const Tables& tab, uint8_t* occ,
                               const TiledEpi& epi, unsigned long long* stats, int shape,
                               cudaStream_t st);
bool tiled_supported(const Geom& g, int shape);
int tiled_shape_count(int kind);
void tiled_shape_cells(int kind, int shape, int cells[3]);

// Layout of the difference rows of the tiled and cell kernels, shared by
// the host table builder and the kernels: row (sigma_p, sigma_q) at byte
// (sigma_p * kmax + sigma_q) * tiled_row_bytes, the int64 constant C at
// tiled_doff_c.  K <= 5 (kmax 5, storage codes 8 sigma): per shell m one
// 16-byte word group, word t holding byte t of D'_{m,s} for s = 0..3
// (delta_e_dp4a).  K = 6 (kmax 6, codes 5 sigma): int32 D'[m][s - 1].
__host__ __device__ constexpr int tiled_code_width(int kmax) { return kmax <= 5 ? 8 : 5; }
__host__ __device__ constexpr int tiled_doff_c(int M, int kmax) {
  return (4 * M * (kmax - 1) + 7) / 8 * 8;
}
// rows are 16-byte aligned (vector loads): rstep * W must be a multiple of
// 16.  With W = 8 the row is an odd number of 16-byte words, so the rows of
// the (p, q) pairs that the lanes of a warp pick at random start at eight
// different bank offsets (fewer conflicts in their 16-byte loads).
__host__ __device__ constexpr int tiled_row_bytes(int M, int kmax) {
  const int W = tiled_code_width(kmax);
  if (W == 8) {
    const int words = (tiled_doff_c(M, kmax) + 8 + 15) / 16;
    return 16 * (words % 2 ? words : words + 1);
  }
  const int rstep = ((tiled_doff_c(M, kmax) + 8 + W - 1) / W + 15) / 16 * 16;
  return rstep * W;
}

}  // namespace smcx

namespace smcx {
// bit-sliced half-shell pair counts of 8-bit lattices (see pair_bits.cu)
cudaError_t launch_pair_count_bits(const Geom& g, int n_shells, const uint8_t* occ,
                                   unsigned long long* h, int n_sm, cudaStream_t st,
                                   bool check_only, bool* ok);
// tiled half-shell pair counts (see pair_tiled.cu); rows of K_MAX = K <= 5 ? 5 : 6
cudaError_t launch_pair_count_tiled(const Geom& g, int n_shells, const uint8_t* occ,
                                    unsigned long long* h, int n_sm, cudaStream_t st,
                                    bool check_only);
}  // namespace smcx

namespace smcx {
// cell sweep phase (kernels_cell.cuh): any 8-bit lattice with K <= 6,
// 2 <= M <= 4 and every n_d >= 4; dtab = the tiled kernel's difference rows
bool cell_supported(const Geom& g);
int cell_variant(const Geom& g);
cudaError_t launch_sweep_cells(const Geom& g, const PhaseArgs& a, const Tables& tab, uint8_t* occ,
                               const uint8_t* dtab, unsigned long long* stats, cudaStream_t st);
// batched sweep (kernels_cell.cuh), args = cell::QueueArgs, one kernel pair
// per register budget (3 or 4 resident blocks of 128 threads per SM):
// launch_sweep_queue_N = the persistent schedule (a chunk of sweeps in one
// launch; grid = n_sm x resident blocks per SM), launch_sweep_phase_N = one
// colour phase ph of every job; sweep_queue_blocks_N() = resident blocks per
// SM (0 on error)
cudaError_t launch_sweep_queue_3(const void* args, int grid, cudaStream_t st);
cudaError_t launch_sweep_queue_4(const void* args, int grid, cudaStream_t st);
cudaError_t launch_sweep_phase_3(const void* args, uint32_t ph, cudaStream_t st);
cudaError_t launch_sweep_phase_4(const void* args, uint32_t ph, cudaStream_t st);
int sweep_queue_blocks_3();
int sweep_queue_blocks_4();
}  // namespace smcx

namespace smcx {
// analyses (analysis.cu): species counts per bin of a cylinder along a
// lattice axis (counts [n_bins][K], zeroed by the caller; n_bins * K <= 8192)
cudaError_t launch_profile(const Geom& g, const uint8_t* occ, int axis, const int* origin_h,
                           unsigned long long r2max, uint32_t length, uint32_t n_bins,
                           unsigned long long* counts, int n_sm, cudaStream_t st);
// clusters of the sites with species in `mask` (first-shell connectivity):
// lab, cnt = n_sites uint32 each (device scratch); afterwards lab[0..*n_out)
// holds the cluster sizes (any order); *n_out and *err zeroed by the caller,
// *err != 0 when a capped loop gave up
cudaError_t launch_clusters(const Geom& g, const uint8_t* occ, uint32_t mask, uint32_t* lab,
                            uint32_t* cnt, unsigned long long* n_out, unsigned int* err,
                            uint32_t n_sites, int n_sm, cudaStream_t st);
// occupancy ^= theirs ^ before over `bytes` bytes (a multiple of 16; all
// three 16-byte aligned): the boundary-plane merge of a z decomposition
cudaError_t launch_merge_planes(uint8_t* occ, const uint8_t* theirs, const uint8_t* before,
                                size_t bytes, int n_sm, cudaStream_t st);

// local-energy model: one colour phase over cells z index az0 .. az0 + naz
// (a.naz > 0), and the total energy as n_blocks int64 partial sums.  lp and T
// are device copies (T: [M][K][K][zt] int64, n_T entries).
// (t32: every table entry fits int32, and the kernel keeps the table in
// shared memory as int32)
cudaError_t launch_sweep_local(const Geom& g, const PhaseArgs& a, const Tables& tab,
                               uint8_t* occ, const LocalParam* lp, const int64_t* T, int n_T,
                               bool t32, int n_items, unsigned long long* stats, cudaStream_t st);
cudaError_t launch_local_energy(const Geom& g, const LocalParam* lp, const int64_t* T, int n_T,
                                const uint8_t* occ, long long* partial, int n_blocks,
                                cudaStream_t st);

}  // namespace smcx
