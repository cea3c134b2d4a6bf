// tiled_dispatch.cu -- selection of the tiled sweep instantiation: the
// exact-extent (uniform edge) tiles first, the ragged ones otherwise.
#include "kernels.h"

namespace smcx {
namespace tiled {
#define SMCX_DECL(NAME)                                                                      \
  cudaError_t NAME(int shape, const Geom& g, const PhaseArgs& a, const Tables& tab,         \
                   uint8_t* occ, const TiledEpi& epi, unsigned long long* stats,             \
                   cudaStream_t st, bool check_only, bool* ok);
SMCX_DECL(dispatch_bcc_uniform)
SMCX_DECL(dispatch_bcc_ragged)
SMCX_DECL(dispatch_fcc_uniform)
SMCX_DECL(dispatch_fcc_ragged)
#undef SMCX_DECL

static cudaError_t dispatch(int shape, const Geom& g, const PhaseArgs& a, const Tables& tab,
                            uint8_t* occ, const TiledEpi& epi, unsigned long long* stats,
                            cudaStream_t st, bool check_only, bool* ok) {
  cudaError_t e;
  if (g.kind == 0) {
    e = dispatch_bcc_uniform(shape, g, a, tab, occ, epi, stats, st, check_only, ok);
    if (*ok) return e;
    return dispatch_bcc_ragged(shape, g, a, tab, occ, epi, stats, st, check_only, ok);
  }
  e = dispatch_fcc_uniform(shape, g, a, tab, occ, epi, stats, st, check_only, ok);
  if (*ok) return e;
  return dispatch_fcc_ragged(shape, g, a, tab, occ, epi, stats, st, check_only, ok);
}
}  // namespace tiled

static const int kShapeCells[2][3][3] = {{{16, 2, 8}, {16, 2, 4}, {32, 1, 8}},
                                         {{16, 2, 4}, {16, 2, 2}, {32, 1, 4}}};

int tiled_shape_count(int kind) {
  (void)kind;
  return 3;
}

void tiled_shape_cells(int kind, int shape, int cells[3]) {
  for (int d = 0; d < 3; ++d) cells[d] = kShapeCells[kind][shape][d];
}

bool tiled_supported(const Geom& g, int shape) {
  bool ok = false;
  const Tables* none = nullptr;
  PhaseArgs a{};
  TiledEpi e{};
  tiled::dispatch(shape, g, a, *none, nullptr, e, nullptr, nullptr, true, &ok);
  return ok;
}

cudaError_t launch_sweep_tiled(const Geom& g, const PhaseArgs& a, const Tables& tab, uint8_t* occ,
                               const TiledEpi& epi, unsigned long long* stats, int shape,
                               cudaStream_t st) {
  bool ok = false;
  const cudaError_t e = tiled::dispatch(shape, g, a, tab, occ, epi, stats, st, false, &ok);
  if (!ok) return cudaErrorNotSupported;
  return e;
}

}  // namespace smcx
