// Generic M2M kernels for double (see sfmm_generic.h).
#define SFMM_GENERIC_T double
#define SFMM_GENERIC_OP sfmm::OP_M2M
#include "sfmm_generic_inst.cuh"
