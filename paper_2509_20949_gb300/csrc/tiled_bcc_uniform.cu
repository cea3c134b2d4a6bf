// tiled_bcc_uniform.cu -- tiled sweep instantiations: BCC, uniform link-cell edges.
#define SMCX_KIND 0
#define SMCX_RAGGED 0
#define SMCX_DISPATCH dispatch_bcc_uniform
#include "tiled_inst.inc"
