// Unrolled translation kernels for order P = 7 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 7
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p7_f32
#include "sfmm_unrolled_inst.cuh"
