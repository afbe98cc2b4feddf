// Phased pass kernel for float (see sfmm_generic.h).
#define SFMM_GENERIC_T float
#define SFMM_GENERIC_PASS 1
#include "sfmm_generic_inst.cuh"
