// Unrolled translation kernels for order P = 3 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 3
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p3_f64
#include "sfmm_unrolled_inst.cuh"
