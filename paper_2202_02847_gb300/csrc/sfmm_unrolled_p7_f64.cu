// Unrolled translation kernels for order P = 7 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 7
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p7_f64
#include "sfmm_unrolled_inst.cuh"
