// Unrolled batch kernels for order P = 11 in float (see sfmm_unrolled.cuh; the
// lists kernels of this order compile in sfmm_unrolled_p11_f32_lists.cu).
#define SFMM_UNROLLED_P 11
#define SFMM_UNROLLED_T float
#define SFMM_UNROLLED_NS p11_f32
#define SFMM_UNROLLED_PART 1
#include "sfmm_unrolled_inst.cuh"
