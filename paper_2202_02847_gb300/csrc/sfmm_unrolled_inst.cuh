// Instantiation of the unrolled kernels for one order (SFMM_UNROLLED_P) and
// one real type (SFMM_UNROLLED_T).  Included by one small translation unit per
// (order, type), so the units compile in parallel; the largest order's units
// are split further by SFMM_UNROLLED_PART (1: the batch kernels, 2: the lists
// kernels; 0, the default: both), each part a module with its own copy of the
// constant tables (fill for the batch part, fill_lists for the lists part).
#include "sfmm_unrolled.cuh"
#include "sfmm_unrolled_dispatch.h"

#if !defined(SFMM_UNROLLED_P) || !defined(SFMM_UNROLLED_T) || !defined(SFMM_UNROLLED_NS)
#error "define SFMM_UNROLLED_P, SFMM_UNROLLED_T and SFMM_UNROLLED_NS before including this file"
#endif
#ifndef SFMM_UNROLLED_PART
#define SFMM_UNROLLED_PART 0
#endif
#define SFMM_WITH_BATCH (SFMM_UNROLLED_PART != 2)
#define SFMM_WITH_LISTS (SFMM_UNROLLED_PART != 1)

namespace sfmm {
namespace unrolled {
namespace SFMM_UNROLLED_NS {

constexpr int P = SFMM_UNROLLED_P;
constexpr int S = P * (P + 1);

using Real = SFMM_UNROLLED_T;

// this module's copy of the constant tables
static bool fill_module(const double *t64, const float *t32) {
    if (std::is_same<Real, double>::value)
        return cudaMemcpyToSymbol(c_tab64, t64, sizeof(double) * NTAB) == cudaSuccess;
    return cudaMemcpyToSymbol(c_tab32, t32, sizeof(float) * NTAB) == cudaSuccess;
}

template <typename K>
void attr(K k, size_t smem) {
    cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

#if SFMM_WITH_BATCH
bool fill(const double *t64, const float *t32) { return fill_module(t64, t32); }
void set_attrs(size_t smem) {
    attr(ubatch_kernel<Real, P, OP_M2M>, smem);
    attr(ubatch_kernel<Real, P, OP_M2L>, smem);
    attr(ubatch_kernel<Real, P, OP_L2L>, smem);
}
#endif
#if SFMM_WITH_LISTS
#if SFMM_UNROLLED_PART == 2
bool fill_lists(const double *t64, const float *t32) { return fill_module(t64, t32); }
#else
bool fill_lists(const double *, const float *) { return true; }   // the batch part's module
#endif
// (a template, so that the FP32 units never name ulists_acc_kernel<float, P>)
template <typename R>
void set_attrs_acc(size_t smem) {
    if constexpr (sizeof(R) == 8 && P <= 10) attr(ulists_acc_kernel<R, P>, smem);
}
void set_attrs_lists(size_t smem) {
    attr(ulists_kernel<Real, P, OP_M2M, 8>, smem);
    attr(ulists_kernel<Real, P, OP_M2L, 32>, smem);
    attr(ulists_kernel<Real, P, OP_L2L, 8>, smem);
    set_attrs_acc<Real>(smem);
}
#endif

// warps per block and blocks for `chunks` warp-chunks of work: the block size
// that leaves the most warps resident per SM (FP64); in FP32 among blocks of 8
// or 4 warps first, whose warps spread evenly over the SM's four
// sub-partitions.  The work is dealt evenly over the warps, so a sub-partition
// that holds more warps than the others sets the pace: FP32 M2L lists at
// P = 10 ran 1.70 ms with two blocks of 7 warps per SM and 1.59 ms with three
// blocks of 4.
template <typename T, typename K>
bool geometry(K kernel, const Launch &L, long long chunks, int *warps, size_t *smem, long long *blocks) {
    const size_t per_warp = (size_t)S * XSTRIDE * sizeof(T);
    int wmax = (int)(L.smem_optin / per_warp);
    if (wmax < 1) return false;
    if (wmax > 8) wmax = 8;
    int best_w = 0, best_nb = 0;
    auto consider = [&](int w) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, w * 32, (size_t)w * per_warp) != cudaSuccess)
            nb = 0;
        if (nb > 0 && w * nb > best_w * best_nb) { best_w = w; best_nb = nb; }
    };
    if (sizeof(T) == 4) {
        if (wmax >= 8) consider(8);
        if (wmax >= 4) consider(4);
    }
    if (best_w < 1)
        for (int w = wmax; w >= 1; --w) consider(w);
    if (best_w < 1) { best_w = wmax; best_nb = 1; }
    // Small launches (no more warp-chunks than sub-partitions): blocks of at
    // most 4 warps, one warp per sub-partition.  The FP64 pipe of a
    // sub-partition is shared by its warps, so two warps of a small tree
    // level on one sub-partition take twice as long as on two.
    if (chunks <= 4LL * L.sm_count && best_w > 4) {
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, kernel, 4 * 32, (size_t)4 * per_warp) == cudaSuccess &&
            nb > 0) {
            best_w = 4;
            best_nb = nb;
        }
    }
    *warps = best_w;
    *smem = (size_t)best_w * per_warp;
    const long long b = (chunks + best_w - 1) / best_w;
    const long long cap = (long long)best_nb * L.sm_count;
    *blocks = b < cap ? b : cap;
    return *blocks >= 1;
}

#if SFMM_WITH_BATCH
template <typename T, int OP>
bool batch_t(const void *const *in, void *const *out, const void *shift, long long count,
             int accumulate, const Launch &L) {
    auto k = ubatch_kernel<T, P, OP>;
    int w;
    size_t smem;
    long long blocks;
    if (!geometry<T>(k, L, (count + 31) / 32, &w, &smem, &blocks)) return false;
    k<<<(unsigned)blocks, w * 32, smem, L.stream>>>(
        reinterpret_cast<const T *const *>(in), reinterpret_cast<T *const *>(out),
        reinterpret_cast<const T *>(shift), count, accumulate, L.status);
    return cudaGetLastError() == cudaSuccess;
}

#endif

#if SFMM_WITH_LISTS
// FP64 M2L lists with the lanes' running sums in tensor memory (orders up to
// 10, where a warp's sums take at most 220 columns): launched when the
// resident CTAs of an SM fit in its 512 columns, else false.
template <typename T>
bool lists_acc(const void *const *src, const void *shift, const long long *offsets,
               void *const *out, long long n_targets, int accumulate, const Launch &L) {
    if constexpr (sizeof(T) != 8 || P > 10) {
        return false;
    } else {
        auto k = ulists_acc_kernel<T, P>;
        int w;
        size_t smem;
        long long blocks;
        if (!geometry<T>(k, L, n_targets, &w, &smem, &blocks)) return false;
        smem += 16;                                  // the tensor-memory address slot
        if (smem > L.smem_optin) return false;
        int nb = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k, w * 32, smem) != cudaSuccess || nb < 1)
            return false;
        const int need = ((w + 3) / 4) * 2 * S;
        int tcols = 32;
        while (tcols < need) tcols <<= 1;
        if (tcols > 512 || nb * tcols > 512) return false;
        const long long cap = (long long)nb * L.sm_count;
        if (blocks > cap) blocks = cap;
        k<<<(unsigned)blocks, w * 32, smem, L.stream>>>(
            reinterpret_cast<const T *const *>(src), reinterpret_cast<const T *>(shift), offsets,
            reinterpret_cast<T *const *>(out), n_targets, accumulate, L.status, tcols);
        return cudaGetLastError() == cudaSuccess;
    }
}

template <typename T, int OP, int G>
bool lists_t(const void *const *src, const void *shift, const long long *offsets,
             void *const *out, long long n_targets, int accumulate, const Launch &L) {
    if constexpr (OP == OP_M2L && G == 32)
        if (lists_acc<T>(src, shift, offsets, out, n_targets, accumulate, L)) return true;
    auto k = ulists_kernel<T, P, OP, G>;
    int w;
    size_t smem;
    long long blocks;
    const long long chunks = (n_targets + (32 / G) - 1) / (32 / G);
    if (!geometry<T>(k, L, chunks, &w, &smem, &blocks)) return false;
    k<<<(unsigned)blocks, w * 32, smem, L.stream>>>(
        reinterpret_cast<const T *const *>(src), reinterpret_cast<const T *>(shift), offsets,
        reinterpret_cast<T *const *>(out), n_targets, accumulate, L.status);
    return cudaGetLastError() == cudaSuccess;
}

#endif

#if SFMM_WITH_BATCH
bool batch(int op, const void *const *in, void *const *out, const void *shift, long long count,
           int accumulate, const Launch &L) {
    if (op == OP_M2M) return batch_t<Real, OP_M2M>(in, out, shift, count, accumulate, L);
    if (op == OP_M2L) return batch_t<Real, OP_M2L>(in, out, shift, count, accumulate, L);
    return batch_t<Real, OP_L2L>(in, out, shift, count, accumulate, L);
}

#endif

#if SFMM_WITH_LISTS
bool lists(int op, const void *const *src, const void *shift, const long long *offsets,
           void *const *out, long long n_targets, int accumulate, const Launch &L) {
    if (op == OP_M2M) return lists_t<Real, OP_M2M, 8>(src, shift, offsets, out, n_targets, accumulate, L);
    if (op == OP_M2L) return lists_t<Real, OP_M2L, 32>(src, shift, offsets, out, n_targets, accumulate, L);
    return lists_t<Real, OP_L2L, 8>(src, shift, offsets, out, n_targets, accumulate, L);
}

#endif

}  // namespace SFMM_UNROLLED_NS
}  // namespace unrolled
}  // namespace sfmm
