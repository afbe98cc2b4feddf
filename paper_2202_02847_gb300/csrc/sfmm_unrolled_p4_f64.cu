// Unrolled translation kernels for order P = 4 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 4
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p4_f64
#include "sfmm_unrolled_inst.cuh"
