// Unrolled translation kernels for order P = 1 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 1
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p1_f32
#include "sfmm_unrolled_inst.cuh"
