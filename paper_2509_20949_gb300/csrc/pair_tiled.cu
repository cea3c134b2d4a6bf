// pair_tiled.cu -- instantiations of the tiled pair-count kernel.
#include "kernels_pair.cuh"

namespace smcx {

template <int KIND, int M, int KMAX, bool P>
static cudaError_t pc_run(const Geom& g, const uint8_t* occ, unsigned long long* h, int n_sm,
                          cudaStream_t st, bool check_only, bool* ok) {
  using C = pairs::PCfg<KIND, M, KMAX, P>;
  *ok = pairs::p_supported<C>(g);
  if (check_only || !*ok) return cudaSuccess;
  return pairs::p_launch<C>(g, occ, h, n_sm, st);
}

template <int KIND, int M>
static cudaError_t pc_k(const Geom& g, const uint8_t* occ, unsigned long long* h, int n_sm,
                        cudaStream_t st, bool check_only, bool* ok) {
  const bool k6 = g.K == 6;
  if (g.pack4)
    return k6 ? pc_run<KIND, M, 6, true>(g, occ, h, n_sm, st, check_only, ok)
              : pc_run<KIND, M, 5, true>(g, occ, h, n_sm, st, check_only, ok);
  return k6 ? pc_run<KIND, M, 6, false>(g, occ, h, n_sm, st, check_only, ok)
            : pc_run<KIND, M, 5, false>(g, occ, h, n_sm, st, check_only, ok);
}

// Half-shell counts H[m][p'][p] (m < n_shells, laid out with K_MAX = 5 or 6
// species per row) into h (zeroed by the caller); the directed counts are
// H + H^T.  The bit-sliced kernel (pair_bits.cu) takes 8- and 4-bit lattices
// whose masks fit shared memory, the byte-tile kernel here the rest.
// cudaErrorNotSupported when the lattice needs the generic kernel.
cudaError_t launch_pair_count_tiled(const Geom& g, int n_shells, const uint8_t* occ,
                                    unsigned long long* h, int n_sm, cudaStream_t st,
                                    bool check_only) {
  bool ok = false;
  cudaError_t e = cudaSuccess;
  if (g.K > 6) return cudaErrorNotSupported;
  e = launch_pair_count_bits(g, n_shells, occ, h, n_sm, st, check_only, &ok);
  if (ok || e != cudaSuccess) return e;
  const int M = n_shells < 2 ? 2 : n_shells;
  if (g.kind == 0) {
    if (M == 2) e = pc_k<0, 2>(g, occ, h, n_sm, st, check_only, &ok);
    else if (M == 3) e = pc_k<0, 3>(g, occ, h, n_sm, st, check_only, &ok);
    else e = pc_k<0, 4>(g, occ, h, n_sm, st, check_only, &ok);
  } else {
    if (M == 2) e = pc_k<1, 2>(g, occ, h, n_sm, st, check_only, &ok);
    else if (M == 3) e = pc_k<1, 3>(g, occ, h, n_sm, st, check_only, &ok);
    else e = pc_k<1, 4>(g, occ, h, n_sm, st, check_only, &ok);
  }
  if (!ok) return cudaErrorNotSupported;
  return e;
}

}  // namespace smcx
