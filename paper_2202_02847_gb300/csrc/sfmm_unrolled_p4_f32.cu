// Unrolled translation kernels for order P = 4 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 4
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p4_f32
#include "sfmm_unrolled_inst.cuh"
