// Unrolled translation kernels for order P = 12 in double (see sfmm_unrolled.cuh).
#define SFMM_UNROLLED_P 12
#define SFMM_UNROLLED_T double
#define SFMM_UNROLLED_NS p12_f64
#include "sfmm_unrolled_inst.cuh"
