// Unrolled translation kernels for order P = 6 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 6
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p6_f32
#include "sfmm_unrolled_inst.cuh"
