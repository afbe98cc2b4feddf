// Unrolled translation kernels for order P = 10 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 10
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p10_f32
#include "sfmm_unrolled_inst.cuh"
