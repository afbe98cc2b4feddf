// Generic M2L kernels for float (see sfmm_generic.h).
#define SFMM_GENERIC_T float
#define SFMM_GENERIC_OP sfmm::OP_M2L
#include "sfmm_generic_inst.cuh"
