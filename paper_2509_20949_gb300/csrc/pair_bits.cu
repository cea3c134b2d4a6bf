// pair_bits.cu -- instantiations of the bit-sliced pair-count kernel.
#include "kernels_pair_bits.cuh"

namespace smcx {

template <int KIND, int M, int KMAX>
static cudaError_t pb_run(const Geom& g, const uint8_t* occ, unsigned long long* h, int n_sm,
                          cudaStream_t st, bool check_only, bool* ok) {
  using C = pbits::BCfg<KIND, M, KMAX>;
  *ok = pbits::b_supported<C>(g);
  if (check_only || !*ok) return cudaSuccess;
  return pbits::b_launch<C>(g, occ, h, n_sm, st);
}

template <int KIND, int M>
static cudaError_t pb_k(const Geom& g, const uint8_t* occ, unsigned long long* h, int n_sm,
                        cudaStream_t st, bool check_only, bool* ok) {
  return g.K == 6 ? pb_run<KIND, M, 6>(g, occ, h, n_sm, st, check_only, ok)
                  : pb_run<KIND, M, 5>(g, occ, h, n_sm, st, check_only, ok);
}

// Half-shell counts H[m][p'][p] of a lattice in 8- or 4-bit storage (rows of
// K_MAX = 5 or 6 species) into h (zeroed by the caller), by bit masks; *ok =
// false (nothing launched) when the lattice is not supported.
cudaError_t launch_pair_count_bits(const Geom& g, int n_shells, const uint8_t* occ,
                                   unsigned long long* h, int n_sm, cudaStream_t st,
                                   bool check_only, bool* ok) {
  *ok = false;
  if (g.K > 6) return cudaSuccess;
  const int M = n_shells < 2 ? 2 : n_shells;
  if (g.kind == 0) {
    if (M == 2) return pb_k<0, 2>(g, occ, h, n_sm, st, check_only, ok);
    if (M == 3) return pb_k<0, 3>(g, occ, h, n_sm, st, check_only, ok);
    return pb_k<0, 4>(g, occ, h, n_sm, st, check_only, ok);
  }
  if (M == 2) return pb_k<1, 2>(g, occ, h, n_sm, st, check_only, ok);
  if (M == 3) return pb_k<1, 3>(g, occ, h, n_sm, st, check_only, ok);
  return pb_k<1, 4>(g, occ, h, n_sm, st, check_only, ok);
}

}  // namespace smcx
