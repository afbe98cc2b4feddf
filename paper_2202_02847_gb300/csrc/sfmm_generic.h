// Launches of the generic (runtime-order) translation kernels.  The kernels
// are heavy to compile, so each (real type, op), the multi-class kernel and
// the phased pass kernel of each real type live in a translation unit of their
// own (sfmm_generic_<type>_<op>.cu, sfmm_generic_<type>_multi.cu,
// sfmm_generic_<type>_pass.cu, all including sfmm_generic_inst.cuh); the
// handle code calls them through these declarations.
#pragma once

#include <cuda_runtime.h>

#include <cstddef>

#include "sfmm_ctx.h"
#include "sfmm_kernels.cuh"
#include "sfmm_wide.cuh"

namespace sfmm {

// launch shape of a generic kernel
struct Geometry {
    bool xg = false;        // rotated solid in global scratch
    int warps = 0;          // warps per block
    size_t smem = 0;        // dynamic shared memory per block
    long long blocks = 0;   // upper bound; the launch caps it at the resident capacity
};

template <typename T, int OP>
void batch_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                  const T *const *I, T *const *O, const T *S, int p_in, int p_out,
                  long long count, int acc, T *scratch, int *status);

template <typename T, int OP>
void lists_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                  const T *const *Sp, const T *S, const long long *offsets, T *const *O,
                  int p_in, int p_out, long long nt, int acc, T *scratch, int *status);

template <typename T, int OP>
void glists_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                   const T *const *Sp, const T *S, const long long *offsets, T *const *O,
                   int p_in, int p_out, long long nt, int acc, int G, T *scratch,
                   unsigned long long *work, int *status);

template <typename T>
void multi_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                  const MultiParams &mp, const T *const *src, const T *shift, const long long *offsets,
                  T *const *out, int acc, T *scratch, int *status);

inline int wide_max_order() { return wide::MAXQ; }
inline size_t wide_warp_bytes(int Q) { return (size_t)wide::warp_units(Q) * 16; }

// the warp-cooperative batch kernel (sfmm_wide.cuh): W solids per warp, the
// block size (wfix warps, or 0: the one that leaves the most warps resident
// per SM) and a persistent grid chosen here; false if it cannot serve these
// orders (above 31, or a warp's area larger than the shared memory)
template <typename T, int OP>
bool wide_launch(const sfmm_ctx *h, int wfix, cudaStream_t stream, const DevTables<T> &tb,
                 const T *const *I, T *const *O, const T *S, int p_in, int p_out, long long count,
                 int acc, int *status);

// the phased pass kernel: a cooperative launch of `blocks` (all resident);
// returns the launch's error code
template <typename T>
cudaError_t pass_launch(const sfmm_ctx *h, const Geometry &g, cudaStream_t stream, const DevTables<T> &tb,
                        const PassParams &pp, T *scratch, unsigned long long *counters, int *status);
template <typename T>
long long pass_resident_blocks(const sfmm_ctx *h, const Geometry &g);

// raise the dynamic shared memory limit of the kernels of one unit
template <typename T, int OP>
void set_generic_attrs(size_t smem);
template <typename T>
void set_multi_attrs(size_t smem);
template <typename T>
void set_pass_attrs(size_t smem);

}  // namespace sfmm
