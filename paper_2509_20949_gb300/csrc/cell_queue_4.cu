// cell_queue_4.cu -- batched sweep kernels, 4 blocks of 128 threads per SM.
#define SMCX_QUEUE_MINB 4
#define SMCX_QUEUE_LAUNCHER launch_sweep_queue_4
#define SMCX_PHASE_LAUNCHER launch_sweep_phase_4
#define SMCX_QUEUE_BLOCKS sweep_queue_blocks_4
#include "cell_queue.inc"
