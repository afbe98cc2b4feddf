// Unrolled translation kernels for order P = 3 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 3
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p3_f32
#include "sfmm_unrolled_inst.cuh"
