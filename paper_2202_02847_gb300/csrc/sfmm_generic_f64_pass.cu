// Phased pass kernel for double (see sfmm_generic.h).
#define SFMM_GENERIC_T double
#define SFMM_GENERIC_PASS 1
#include "sfmm_generic_inst.cuh"
