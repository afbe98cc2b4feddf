// Launch interface of the fully unrolled kernels (one translation unit per
// compiled order, see sfmm_unrolled_inst.cuh).
#pragma once

#include <cuda_runtime.h>

namespace sfmm {
namespace unrolled {

struct Launch {
    int sm_count;
    size_t smem_optin;
    int *status;
    cudaStream_t stream;
};

// Orders with a compiled kernel set, and whether `P` is one of them.
bool compiled(int P);

// Copy the constant tables (NTAB reals each, layout of sfmm_unrolled.cuh) into
// every compiled unit on the current device.  Returns false on a CUDA error.
bool fill_constants(const double *t64, const float *t32);

// Set the shared-memory limit of every compiled kernel (current device).
void set_attributes(size_t smem_optin);

// Launch one batch / lists call; false if P is not compiled or the launch
// failed to be enqueued.
bool launch_batch(bool f64, int P, int op, const void *const *in, void *const *out,
                  const void *shift, long long count, int accumulate, const Launch &L);
bool launch_lists(bool f64, int P, int op, const void *const *src, const void *shift,
                  const long long *offsets, void *const *out, long long n_targets,
                  int accumulate, const Launch &L);

// size of the constant table in reals
int table_size();

}  // namespace unrolled
}  // namespace sfmm
