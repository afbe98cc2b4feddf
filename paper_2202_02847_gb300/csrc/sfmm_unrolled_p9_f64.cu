// Unrolled translation kernels for order P = 9 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 9
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p9_f64
#include "sfmm_unrolled_inst.cuh"
