// Unrolled translation kernels for order P = 8 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 8
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p8_f32
#include "sfmm_unrolled_inst.cuh"
