// cell_inst.cu -- instantiations and launchers of the cell sweep phase.
#include "kernels_cell.cuh"

namespace smcx {
namespace cell {

template <int KIND, int M, int KMAX>
static cudaError_t single(const Geom& g, const PhaseArgs& a, const Tables& tab, uint8_t* occ,
                          const uint8_t* dtab, unsigned long long* stats, cudaStream_t st) {
  using C = CCfg<KIND, M, KMAX>;
  if (a.naz <= 0) return cudaErrorInvalidValue;
  uint32_t n = static_cast<uint32_t>(a.naz);
  for (int d = 0; d < 2; ++d) n *= g.m[d] == 1 ? 1u : static_cast<uint32_t>(g.m[d] / 2);
  k_sweep_cells_single<C><<<(n + C::NT - 1) / C::NT, C::NT, 0, st>>>(g, a, tab, occ, dtab, stats, n);
  return cudaGetLastError();
}

}  // namespace cell

// variant index = kind * 6 + (M - 2) * 2 + (K == 6)
bool cell_supported(const Geom& g) {
  if (g.pack4 || g.K > 6 || g.M < 2 || g.M > 4) return false;
  for (int d = 0; d < 3; ++d)
    if (g.n[d] < 4) return false;
  return true;
}

int cell_variant(const Geom& g) { return g.kind * 6 + (g.M - 2) * 2 + (g.K == 6 ? 1 : 0); }

#define SMCX_CELL_SWITCH(CALL)                                  \
  switch (variant) {                                            \
    case 0: return CALL(0, 2, 5);                               \
    case 1: return CALL(0, 2, 6);                               \
    case 2: return CALL(0, 3, 5);                               \
    case 3: return CALL(0, 3, 6);                               \
    case 4: return CALL(0, 4, 5);                               \
    case 5: return CALL(0, 4, 6);                               \
    case 6: return CALL(1, 2, 5);                               \
    case 7: return CALL(1, 2, 6);                               \
    case 8: return CALL(1, 3, 5);                               \
    case 9: return CALL(1, 3, 6);                               \
    case 10: return CALL(1, 4, 5);                              \
    case 11: return CALL(1, 4, 6);                              \
    default: return cudaErrorNotSupported;                      \
  }

cudaError_t launch_sweep_cells(const Geom& g, const PhaseArgs& a, const Tables& tab, uint8_t* occ,
                               const uint8_t* dtab, unsigned long long* stats, cudaStream_t st) {
  if (!cell_supported(g)) return cudaErrorNotSupported;
  const int variant = cell_variant(g);
#define SMCX_SINGLE(K, M, X) cell::single<K, M, X>(g, a, tab, occ, dtab, stats, st)
  SMCX_CELL_SWITCH(SMCX_SINGLE)
#undef SMCX_SINGLE
}


}  // namespace smcx
