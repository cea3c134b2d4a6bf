// tiled_dispatch.cu -- selection of the tiled sweep instantiation.
#include "kernels.h"

namespace smcx {
namespace tiled {
cudaError_t dispatch_bcc(int shape, const Geom& g, const PhaseArgs& a, const Tables& tab,
                         uint8_t* occ, const TiledEpi& epi, unsigned long long* stats,
                         cudaStream_t st, bool check_only, bool* ok);
cudaError_t dispatch_fcc(int shape, const Geom& g, const PhaseArgs& a, const Tables& tab,
                         uint8_t* occ, const TiledEpi& epi, unsigned long long* stats,
                         cudaStream_t st, bool check_only, bool* ok);
void bcc_shape_cells(int shape, int cells[3]);
void fcc_shape_cells(int shape, int cells[3]);
}  // namespace tiled

int tiled_row_words(int M, int kmax) { return (M * (kmax - 1) + 2 + 1) / 2 * 2; }

int tiled_shape_count(int kind) {
  (void)kind;
  return 2;
}

void tiled_shape_cells(int kind, int shape, int cells[3]) {
  if (kind == 0)
    tiled::bcc_shape_cells(shape, cells);
  else
    tiled::fcc_shape_cells(shape, cells);
}

bool tiled_supported(const Geom& g, int shape) {
  bool ok = false;
  Tables* none = nullptr;
  PhaseArgs a{};
  TiledEpi e{};
  if (g.kind == 0)
    tiled::dispatch_bcc(shape, g, a, *none, nullptr, e, nullptr, nullptr, true, &ok);
  else
    tiled::dispatch_fcc(shape, g, a, *none, nullptr, e, nullptr, nullptr, true, &ok);
  return ok;
}

cudaError_t launch_sweep_tiled(const Geom& g, const PhaseArgs& a, const Tables& tab, uint8_t* occ,
                               const TiledEpi& epi, unsigned long long* stats, int shape,
                               cudaStream_t st) {
  bool ok = false;
  const cudaError_t e =
      g.kind == 0 ? tiled::dispatch_bcc(shape, g, a, tab, occ, epi, stats, st, false, &ok)
                  : tiled::dispatch_fcc(shape, g, a, tab, occ, epi, stats, st, false, &ok);
  if (!ok) return cudaErrorNotSupported;
  return e;
}

}  // namespace smcx
