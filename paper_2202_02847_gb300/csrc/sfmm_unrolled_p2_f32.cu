// Unrolled translation kernels for order P = 2 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 2
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p2_f32
#include "sfmm_unrolled_inst.cuh"
