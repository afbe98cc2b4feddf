// Unrolled batch kernels for order P = 11 in double (see sfmm_unrolled.cuh; the
// lists kernels of this order compile in sfmm_unrolled_p11_f64_lists.cu).
#define SFMM_UNROLLED_P 11
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p11_f64
#define SFMM_UNROLLED_PART 1
#include "sfmm_unrolled_inst.cuh"
