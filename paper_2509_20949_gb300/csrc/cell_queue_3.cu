// cell_queue_3.cu -- batched sweep kernels, 3 blocks of 128 threads per SM.
#define SMCX_QUEUE_MINB 3
#define SMCX_QUEUE_LAUNCHER launch_sweep_queue_3
#define SMCX_PHASE_LAUNCHER launch_sweep_phase_3
#define SMCX_QUEUE_BLOCKS sweep_queue_blocks_3
#include "cell_queue.inc"
