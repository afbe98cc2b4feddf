// Unrolled translation kernels for order P = 12 in float (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 12
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p12_f32
#include "sfmm_unrolled_inst.cuh"
