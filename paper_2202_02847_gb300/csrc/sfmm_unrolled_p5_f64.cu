// Unrolled translation kernels for order P = 5 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 5
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p5_f64
#include "sfmm_unrolled_inst.cuh"
