// Definitions of the generic launches, explicitly instantiated for one real
// type (SFMM_GENERIC_T) and either one op (SFMM_GENERIC_OP), the multi-class
// kernel (SFMM_GENERIC_MULTI) or the phased pass kernel (SFMM_GENERIC_PASS).  Included by one small translation
// unit per case, so the units compile in parallel.
#include <atomic>

#include "sfmm_generic.h"
#include "sfmm_wide.cuh"

#if !defined(SFMM_GENERIC_T) || \
    !(defined(SFMM_GENERIC_OP) || defined(SFMM_GENERIC_MULTI) || defined(SFMM_GENERIC_PASS))
#error "define SFMM_GENERIC_T and SFMM_GENERIC_OP, SFMM_GENERIC_MULTI or SFMM_GENERIC_PASS before including this file"
#endif

namespace sfmm {
namespace {

// Persistent grid: no more blocks than the device holds at once.
template <typename K>
long long resident_blocks(const sfmm_ctx *h, K kernel, const Geometry &g) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, g.warps * WARP, g.smem) != cudaSuccess || nb < 1)
        nb = 1;
    long long cap = (long long)nb * h->sm_count;
    return g.blocks < cap ? g.blocks : cap;
}

template <typename K>
void attr(K k, size_t smem) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

template <typename T, int OP>
void batch_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                  const T *const *I, T *const *O, const T *S, int p_in, int p_out,
                  long long count, int acc, T *scratch, int *status) {
    if (g.xg) {
        auto k = batch_kernel<T, OP, true>;
        k<<<(unsigned)resident_blocks(h, k, g), g.warps * WARP, g.smem, stream>>>(tb, I, O, S, p_in, p_out, count, acc, scratch, status);
    } else {
        auto k = batch_kernel<T, OP, false>;
        k<<<(unsigned)resident_blocks(h, k, g), g.warps * WARP, g.smem, stream>>>(tb, I, O, S, p_in, p_out, count, acc, scratch, status);
    }
}

template <typename T, int OP>
void lists_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                  const T *const *Sp, const T *S, const long long *offsets, T *const *O,
                  int p_in, int p_out, long long nt, int acc, T *scratch, int *status) {
    if (g.xg) {
        auto k = lists_kernel<T, OP, true>;
        k<<<(unsigned)resident_blocks(h, k, g), g.warps * WARP, g.smem, stream>>>(tb, Sp, S, offsets, O, p_in, p_out, nt, acc, scratch, status);
    } else {
        auto k = lists_kernel<T, OP, false>;
        k<<<(unsigned)resident_blocks(h, k, g), g.warps * WARP, g.smem, stream>>>(tb, Sp, S, offsets, O, p_in, p_out, nt, acc, scratch, status);
    }
}

template <typename T, int OP>
void glists_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                   const T *const *Sp, const T *S, const long long *offsets, T *const *O,
                   int p_in, int p_out, long long nt, int acc, int G, T *scratch,
                   unsigned long long *work, int *status) {
    auto k = glists_kernel<T, OP>;
    k<<<(unsigned)resident_blocks(h, k, g), g.warps * WARP, g.smem, stream>>>(tb, Sp, S, offsets, O, p_in, p_out, nt, acc, G, scratch, work, status);
}

template <typename T, int OP>
bool wide_launch(const sfmm_ctx *h, int wfix, cudaStream_t stream, const DevTables<T> &tb,
                 const T *const *I, T *const *O, const T *S, int p_in, int p_out, long long count,
                 int acc, int *status) {
    const int Q = p_in > p_out ? p_in : p_out;
    if (Q > wide::MAXQ) return false;
    const size_t per_warp = (size_t)wide::warp_units(Q) * sizeof(wide::Pk<T>);
    if (per_warp > h->smem_optin) return false;
    if (count == 0) return true;
    auto k = wide::wbatch_kernel<T, OP>;
    // block size and resident blocks per SM for (Q, wfix), from the occupancy
    // calculator once per process (the answer depends only on these and on the
    // kind of device, which is one per process here; a serving loop launches
    // this kernel once per chunk)
    static std::atomic<int> cache[wide::MAXQ + 1][9];
    int best_w = 0, best_nb = 0;
    const int key = wfix > 0 && wfix <= 8 ? wfix : 0;
    const int hit = cache[Q][key].load(std::memory_order_relaxed);
    if (hit > 0) {
        best_w = hit / 1024;
        best_nb = hit % 1024;
    } else {
        for (int w = 8; w >= 1; --w) {
            if ((size_t)w * per_warp > h->smem_optin || (wfix > 0 && w != wfix)) continue;
            int nb = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, w * WARP, (size_t)w * per_warp) != cudaSuccess)
                nb = 0;
            if (nb > 0 && w * nb > best_w * best_nb) {
                best_w = w;
                best_nb = nb;
            }
        }
        if (best_w >= 1) cache[Q][key].store(best_w * 1024 + best_nb, std::memory_order_relaxed);
    }
    if (best_w < 1) return false;
    const long long groups = (count + wide::Pk<T>::W - 1) / wide::Pk<T>::W;
    long long blocks = (groups + best_w - 1) / best_w;
    const long long cap = (long long)best_nb * h->sm_count;
    if (blocks > cap) blocks = cap;
    k<<<(unsigned)blocks, best_w * WARP, (size_t)best_w * per_warp, stream>>>(tb, I, O, S, p_in, p_out, count, acc,
                                                                             status);
    return true;
}

template <typename T>
void multi_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                  const MultiParams &mp, const T *const *src, const T *shift, const long long *offsets,
                  T *const *out, int acc, T *scratch, int *status) {
    auto k = multi_lists_kernel<T>;
    k<<<(unsigned)resident_blocks(h, k, g), g.warps * WARP, g.smem, stream>>>(tb, mp, src, shift, offsets, out, acc, scratch, status);
}

template <typename T>
long long pass_resident_blocks(const sfmm_ctx *h, const Geometry &g) {
    int nb = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, pass_kernel<T>, g.warps * WARP, g.smem) != cudaSuccess)
        return -1;
    return (long long)nb * h->sm_count;
}

template <typename T>
cudaError_t pass_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                        const PassParams &pp, T *scratch, unsigned long long *counters, int *status) {
    (void)h;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)g.blocks);
    cfg.blockDim = dim3((unsigned)(g.warps * WARP));
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, pass_kernel<T>, tb, pp, scratch, counters, status);
}

template <typename T, int OP>
void set_generic_attrs(size_t smem) {
    attr(batch_kernel<T, OP, false>, smem);
    attr(batch_kernel<T, OP, true>, smem);
    attr(lists_kernel<T, OP, false>, smem);
    attr(lists_kernel<T, OP, true>, smem);
    attr(glists_kernel<T, OP>, smem);
    attr(wide::wbatch_kernel<T, OP>, smem);
}

template <typename T>
void set_multi_attrs(size_t smem) {
    attr(multi_lists_kernel<T>, smem);
}

template <typename T>
void set_pass_attrs(size_t smem) {
    attr(pass_kernel<T>, smem);
}

#if defined(SFMM_GENERIC_OP)
using GT = SFMM_GENERIC_T;
constexpr int GOP = SFMM_GENERIC_OP;
template void batch_launch<GT, GOP>(const sfmm_ctx *, const Geometry &, cudaStream_t, const DevTables<GT> &,
                                    const GT *const *, GT *const *, const GT *, int, int, long long, int,
                                    GT *, int *);
template void lists_launch<GT, GOP>(const sfmm_ctx *, const Geometry &, cudaStream_t, const DevTables<GT> &,
                                    const GT *const *, const GT *, const long long *, GT *const *, int, int,
                                    long long, int, GT *, int *);
template void glists_launch<GT, GOP>(const sfmm_ctx *, const Geometry &, cudaStream_t, const DevTables<GT> &,
                                     const GT *const *, const GT *, const long long *, GT *const *, int, int,
                                     long long, int, int, GT *, unsigned long long *, int *);
template bool wide_launch<GT, GOP>(const sfmm_ctx *, int, cudaStream_t, const DevTables<GT> &,
                                   const GT *const *, GT *const *, const GT *, int, int, long long, int, int *);
template void set_generic_attrs<GT, GOP>(size_t);
#elif defined(SFMM_GENERIC_MULTI)
using GT = SFMM_GENERIC_T;
template void multi_launch<GT>(const sfmm_ctx *, const Geometry &, cudaStream_t, const DevTables<GT> &,
                               const MultiParams &, const GT *const *, const GT *, const long long *,
                               GT *const *, int, GT *, int *);
template void set_multi_attrs<GT>(size_t);
#else
using GT = SFMM_GENERIC_T;
template void set_pass_attrs<GT>(size_t);
template cudaError_t pass_launch<GT>(const sfmm_ctx *, const Geometry &, cudaStream_t, const DevTables<GT> &,
                                     const PassParams &, GT *, unsigned long long *, int *);
template long long pass_resident_blocks<GT>(const sfmm_ctx *, const Geometry &);
#endif

}  // namespace sfmm
