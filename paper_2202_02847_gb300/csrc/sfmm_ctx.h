// Internal definition of the handle behind sfmm_handle (not part of the ABI).
#pragma once

#include <cuda_runtime.h>

#include <cstddef>
#include <mutex>

#include <nvtx3/nvToolsExt.h>

#include "sfmm.h"
#include "sfmm_kernels.cuh"

// An NVTX range named after the API call, open for the call's duration (its
// launches and host work), so that a timeline tool shows every entry point;
// a no-op unless such a tool is attached.
struct SfmmRange {
    explicit SfmmRange(const char *name) { nvtxRangePushA(name); }
    ~SfmmRange() { nvtxRangePop(); }
    SfmmRange(const SfmmRange &) = delete;
    SfmmRange &operator=(const SfmmRange &) = delete;
};

struct sfmm_ctx {
    int Pmax = 0;
    sfmm_dtype dtype = SFMM_F64;
    int device = 0;
    int sm_count = 0;
    size_t smem_optin = 0;      // max dynamic shared memory per block
    void *d_tables = nullptr;   // one allocation holding every table
    int *d_status = nullptr;    // device status word (atomicOr by kernels)
    unsigned long long *d_work = nullptr;   // chunk counter of the group-lists launches (with the scratch)
    unsigned long long *d_pass = nullptr;   // per-phase chunk and barrier counters of the pass kernel
    sfmm::DevTables<double> t64{};
    sfmm::DevTables<float> t32{};
    // global scratch for orders whose rotated solid does not fit in shared
    // memory: one slot of x_elems(P_max) elements per lane of a resident warp
    void *d_scratch = nullptr;
    size_t scratch_bytes = 0;
    // launches that use the scratch are ordered through this event so that
    // calls on different streams never share it concurrently
    std::mutex scratch_mu;
    cudaEvent_t scratch_free = nullptr;
    // the unrolled kernels (fixed orders) have their constant tables on this device
    bool unrolled_ok = false;
    // launch policy per (op, p_in, p_out): sfmm_policy and warps per block (0 = auto)
    unsigned char policy[3][65][65] = {};
    unsigned char warps[3][65][65] = {};
};
