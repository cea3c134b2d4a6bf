// tiled_bcc_ragged.cu -- tiled sweep instantiations: BCC, ragged link-cell edges.
#define SMCX_KIND 0
#define SMCX_RAGGED 1
#define SMCX_DISPATCH dispatch_bcc_ragged
#include "tiled_inst.inc"
