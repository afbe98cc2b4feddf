// Unrolled translation kernels for order P = 8 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 8
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p8_f64
#include "sfmm_unrolled_inst.cuh"
