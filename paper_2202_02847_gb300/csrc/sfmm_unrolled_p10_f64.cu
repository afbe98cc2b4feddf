// Unrolled translation kernels for order P = 10 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 10
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p10_f64
#include "sfmm_unrolled_inst.cuh"
