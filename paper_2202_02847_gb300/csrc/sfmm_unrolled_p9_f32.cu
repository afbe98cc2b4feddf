// Unrolled translation kernels for order P = 9 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 9
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p9_f32
#include "sfmm_unrolled_inst.cuh"
