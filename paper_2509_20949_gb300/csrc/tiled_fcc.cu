// tiled_fcc.cu -- instantiations of the tiled sweep phase for FCC lattices.
#include "kernels_tiled.cuh"

namespace smcx {
namespace tiled {

// tile shapes (active cells per block along x, y, z)
constexpr int kFccShapes[2][3] = {{16, 2, 2}, {16, 2, 4}};

template <int M, int KMAX, bool P, int S>
using FccCfg = Cfg<1, M, KMAX, P, kFccShapes[S][0], kFccShapes[S][1], kFccShapes[S][2]>;

template <int M, int KMAX, bool P, int S>
static cudaError_t run(const Geom& g, const PhaseArgs& a, const Tables& tab, uint8_t* occ,
                       const TiledEpi& epi, unsigned long long* stats, cudaStream_t st,
                       bool check_only, bool* ok) {
  using C = FccCfg<M, KMAX, P, S>;
  *ok = supported<C>(g);
  if (check_only || !*ok) return cudaSuccess;
  return launch_cfg<C>(g, a, tab, occ, epi, stats, st);
}

template <int M, int KMAX, bool P>
static cudaError_t by_shape(int shape, const Geom& g, const PhaseArgs& a, const Tables& tab,
                            uint8_t* occ, const TiledEpi& epi, unsigned long long* stats,
                            cudaStream_t st, bool check_only, bool* ok) {
  switch (shape) {
    case 0: return run<M, KMAX, P, 0>(g, a, tab, occ, epi, stats, st, check_only, ok);
    case 1: return run<M, KMAX, P, 1>(g, a, tab, occ, epi, stats, st, check_only, ok);
    default: *ok = false; return cudaSuccess;
  }
}

cudaError_t dispatch_fcc(int shape, const Geom& g, const PhaseArgs& a, const Tables& tab,
                         uint8_t* occ, const TiledEpi& epi, unsigned long long* stats,
                         cudaStream_t st, bool check_only, bool* ok) {
  *ok = false;
  const bool k6 = g.K == 6;
  if (g.K > 6) return cudaSuccess;
#define SMCX_FCC_CASE(MM)                                                                     \
  if (g.M == MM) {                                                                            \
    if (g.pack4)                                                                              \
      return k6 ? by_shape<MM, 6, true>(shape, g, a, tab, occ, epi, stats, st, check_only, ok) \
                : by_shape<MM, 5, true>(shape, g, a, tab, occ, epi, stats, st, check_only, ok); \
    return k6 ? by_shape<MM, 6, false>(shape, g, a, tab, occ, epi, stats, st, check_only, ok)  \
              : by_shape<MM, 5, false>(shape, g, a, tab, occ, epi, stats, st, check_only, ok); \
  }
  SMCX_FCC_CASE(2)
  SMCX_FCC_CASE(3)
  SMCX_FCC_CASE(4)
#undef SMCX_FCC_CASE
  return cudaSuccess;
}

void fcc_shape_cells(int shape, int cells[3]) {
  for (int d = 0; d < 3; ++d) cells[d] = kFccShapes[shape][d];
}

}  // namespace tiled
}  // namespace smcx
