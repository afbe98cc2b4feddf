// Unrolled translation kernels for order P = 6 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 6
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p6_f64
#include "sfmm_unrolled_inst.cuh"
