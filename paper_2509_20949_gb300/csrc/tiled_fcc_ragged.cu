// tiled_fcc_ragged.cu -- tiled sweep instantiations: FCC, ragged link-cell edges.
#define SMCX_KIND 1
#define SMCX_RAGGED 1
#define SMCX_DISPATCH dispatch_fcc_ragged
#include "tiled_inst.inc"
