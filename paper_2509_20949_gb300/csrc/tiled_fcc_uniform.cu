// tiled_fcc_uniform.cu -- tiled sweep instantiations: FCC, uniform link-cell edges.
#define SMCX_KIND 1
#define SMCX_RAGGED 0
#define SMCX_DISPATCH dispatch_fcc_uniform
#include "tiled_inst.inc"
