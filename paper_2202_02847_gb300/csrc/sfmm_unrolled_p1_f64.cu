// Unrolled translation kernels for order P = 1 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 1
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p1_f64
#include "sfmm_unrolled_inst.cuh"
