// Unrolled translation kernels for order P = 2 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 2
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p2_f64
#include "sfmm_unrolled_inst.cuh"
