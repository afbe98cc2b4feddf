// Unrolled translation kernels for order P = 5 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 5
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p5_f32
#include "sfmm_unrolled_inst.cuh"
