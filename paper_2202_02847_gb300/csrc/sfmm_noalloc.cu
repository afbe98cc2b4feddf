// sfmm_translate_batch_noalloc: batched translations that allocate nothing.
//
// Some callers cannot allocate device memory at the point where they
// translate: a plug-in running inside a fixed device-memory budget handed out
// by a host framework that owns every allocation, or a real-time loop where an
// allocation (and the implicit device synchronisation of cudaMalloc /
// cudaFree) is not allowed.  For them this
// entry point runs the global-scratch variant of the batch kernel with its
// scratch in a fixed device array compiled into the library instead of a
// buffer owned by the handle.  It calls no cudaMalloc, cudaFree or other
// allocating routine.
#include <cuda_runtime.h>

#include <mutex>

#include "sfmm.h"
#include "sfmm_ctx.h"
#include "sfmm_kernels.cuh"

using namespace sfmm;

namespace {

// Scratch of this entry point: the rotated solids of the resident warps, one
// slot of 32 * p_in(p_in+1) reals per warp.  A file-scope device array of a
// fixed 16 MiB: every GPU that loads the library holds it until the process
// exits.  Every call on a device shares it and it keeps the last call's
// contents; each lane writes its whole slot before reading it, so nothing has
// to start at zero.
constexpr size_t kNoallocScratchBytes = size_t(16) << 20;
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoallocScratchBytes];

// In host code g_noalloc_scratch is only a host-side stand-in; its device
// address is looked up once per device (with that device current) and cached.
// The same one-time set-up raises the shared-memory limit of this file's
// kernel instances (each translation unit is its own module, so the limits
// that sfmm_create sets do not reach them).  Neither step allocates.
constexpr int kMaxDevices = 64;
std::mutex g_mu;
void *g_scratch_addr[kMaxDevices] = {};

template <typename T>
bool raise_smem_limits(size_t smem) {
    return cudaFuncSetAttribute(batch_kernel<T, OP_M2M, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
           cudaFuncSetAttribute(batch_kernel<T, OP_M2L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess &&
           cudaFuncSetAttribute(batch_kernel<T, OP_L2L, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem) == cudaSuccess;
}

sfmm_status setup_device(int dev, size_t smem_optin, void **addr) {
    if (dev < 0 || dev >= kMaxDevices) return SFMM_ERR_UNSUPPORTED;
    std::lock_guard<std::mutex> lk(g_mu);
    if (g_scratch_addr[dev] == nullptr) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || p == nullptr)
            return SFMM_ERR_CUDA;
        if (!raise_smem_limits<double>(smem_optin) || !raise_smem_limits<float>(smem_optin))
            return SFMM_ERR_CUDA;
        g_scratch_addr[dev] = p;
    }
    *addr = g_scratch_addr[dev];
    return SFMM_OK;
}

template <typename T, int OP>
sfmm_status launch(const sfmm_ctx *h, const DevTables<T> &tb, const void *const *in,
                   void *const *out, const void *shift, int p_in, int p_out, long long count,
                   int accumulate, cudaStream_t stream, void *scratch) {
    const size_t per_warp = (size_t)row_elems(p_in, p_out) * WARP * sizeof(T);   // shared
    const size_t slot = (size_t)x_elems(p_in) * WARP * sizeof(T);                 // scratch
    const long long slots = (long long)(kNoallocScratchBytes / slot);
    if (slots < 1 || per_warp > h->smem_optin) return SFMM_ERR_UNSUPPORTED;
    long long w = (long long)(h->smem_optin / 2 / per_warp);
    if (w < 1) w = 1;
    if (w > 4) w = 4;
    if (w > slots) w = slots;
    long long blocks = slots / w;                                   // slot = warp index
    const long long need = (count + w * WARP - 1) / (w * WARP);
    if (blocks > need) blocks = need;
    auto kernel = batch_kernel<T, OP, true>;
    int nb = 0;
    const size_t smem = (size_t)w * per_warp;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, (int)(w * WARP), smem) == cudaSuccess && nb > 0 &&
        blocks > (long long)nb * h->sm_count)
        blocks = (long long)nb * h->sm_count;
    kernel<<<(unsigned)blocks, (unsigned)(w * WARP), smem, stream>>>(
        tb, reinterpret_cast<const T *const *>(in), reinterpret_cast<T *const *>(out),
        reinterpret_cast<const T *>(shift), p_in, p_out, count, accumulate,
        reinterpret_cast<T *>(scratch), h->d_status);
    return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
}

template <typename T>
sfmm_status dispatch(const sfmm_ctx *h, const DevTables<T> &tb, sfmm_op op, const void *const *in,
                     void *const *out, const void *shift, int p_in, int p_out, long long count,
                     int accumulate, cudaStream_t s, void *scratch) {
    if (op == SFMM_M2M)
        return launch<T, OP_M2M>(h, tb, in, out, shift, p_in, p_out, count, accumulate, s, scratch);
    if (op == SFMM_M2L)
        return launch<T, OP_M2L>(h, tb, in, out, shift, p_in, p_out, count, accumulate, s, scratch);
    return launch<T, OP_L2L>(h, tb, in, out, shift, p_in, p_out, count, accumulate, s, scratch);
}

}  // namespace

extern "C" sfmm_status sfmm_translate_batch_noalloc(sfmm_handle h, sfmm_op op,
                                                    const void *const *in, void *const *out,
                                                    const void *shift, int p_in, int p_out,
                                                    long long count, int accumulate,
                                                    sfmm_stream stream) {
    if (h == nullptr || count < 0) return SFMM_ERR_ARG;
    if (op != SFMM_M2M && op != SFMM_M2L && op != SFMM_L2L) return SFMM_ERR_ARG;
    if (p_in < 1 || p_out < 1 || p_in > h->Pmax || p_out > h->Pmax) return SFMM_ERR_ORDER;
    if (count == 0) return SFMM_OK;
    if (in == nullptr || out == nullptr || shift == nullptr) return SFMM_ERR_ARG;
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess) return SFMM_ERR_CUDA;
    if (dev != h->device) return SFMM_ERR_ARG;
    void *scratch = nullptr;
    const sfmm_status st = setup_device(dev, h->smem_optin, &scratch);
    if (st != SFMM_OK) return st;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    if (h->dtype == SFMM_F64)
        return dispatch<double>(h, h->t64, op, in, out, shift, p_in, p_out, count, accumulate, s, scratch);
    return dispatch<float>(h, h->t32, op, in, out, shift, p_in, p_out, count, accumulate, s, scratch);
}
