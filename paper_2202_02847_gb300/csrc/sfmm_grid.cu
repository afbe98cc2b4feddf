// Shift-grouped M2L on a uniform grid of boxes on the tensor cores.
//
// The paper sets aside BLAS-based M2L for a finite set of shift vectors
// (Sec. 2.2): store the translation matrix of every shift and apply it to many
// solids at once.  On a uniform octree level every M2L shift is an integer
// offset u (target - source, in box units) with max|u_i| in {2, 3}, so all
// translations with the same u share one real 256x256 matrix T_u (P = 16) in
// the box-scaled orthonormal basis
//     x_k^m = M_k^m c_k^m / h^{k+1},   y_n^m = L_n^m h^n / c_n^m,   y = T_u x,
// (eq. scaling with s = 1/h), and a target's local expansion is the sum of
// T_u x over its 189 offsets.  Targets of the same child octant share the same
// 189 offsets, so a tile of 128 same-octant targets (64 when the grid side is
// not a multiple of 16) is one GEMM with K = 189 * 256 on the 5th-generation
// tensor cores (tcgen05.mma kind::f16, M = 128, N = tile, K = 16):
//   * operands are split into two FP16 parts, hi + lo (22 significant bits),
//     multiplied as the three products hi*hi, hi*lo, lo*hi with FP32
//     accumulation in tensor memory (the dropped lo*lo is 2^-22 relative).
//     FP16 has 5 exponent bits, so every operator row n is scaled by a power of
//     two that brings its largest entry near 2^12 (fixed when the grid is
//     created), and all sources of a call by one power of two that brings
//     their largest magnitude below 2^14 (found on the device per call); the
//     output undoes both exactly;
//   * every 2 offsets the FP32 accumulator is added into a float-float sum
//     (hi + lo, Knuth's two-sum) kept in tensor memory, so a target's sum over
//     the 189 offsets carries about 48 bits; at the end of its work unit the
//     CTA writes the sum once, in FP64, to its own slot: no atomics, and a
//     target's result is the same on every run;
//   * work units are (tile, operator row half, K half): the CTA computes rows
//     [128 h, 128 h + 128) of T_u x for the offsets of its K half, and the
//     unpack kernel adds the two K halves in a fixed order;
//   * operand chunks (64 of K, four MMAs) are staged in shared memory in three
//     stages of 64 KB: the T_u chunk of the row half (both parts), stored
//     pre-tiled, by one bulk copy; the targets' source vectors (both parts),
//     stored split by coordinate parity, by two 5-D tensor copies with 128-byte
//     rows (rows of 32 bytes, 16 of K, held the tensor copies to a quarter of
//     the rate the MMAs need);
//   * one thread issues copies, one issues MMAs, four warps drain the
//     accumulators (the float-float update of one 2-offset group overlaps the
//     MMAs of the next, two accumulator buffers); one persistent CTA per SM.
// T_u are built once per grid object with the FP64 rotation-based M2L on the
// 256 basis vectors of every offset.  Every mbarrier wait is bounded: on
// time-out the kernel records SFMM_GRID_TIMEOUT in the status word, stops
// issuing work, waits (bounded by time only) for its copies and MMAs in
// flight, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_fp16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <new>
#include <vector>

#include "sfmm.h"
#include "sfmm_ctx.h"
#include "sfmm_kernels.cuh"
#include "sfmm_tables.h"

using namespace sfmm;

namespace {

constexpr int GP = 16;             // order of the grid operators
constexpr int KD = GP * GP;        // 256 reals per box in the reduced layout
constexpr int KC = 64;             // K chunk staged in shared memory (four FP16 MMAs of K = 16)
constexpr int UK = 16;             // K of one tcgen05.mma kind::f16
constexpr int NKC = KD / KC;       // chunks per offset
constexpr int NPART = 2;           // operand parts: hi, lo (FP16 each)
constexpr int HROWS = 128;         // operator rows of one CTA (one half of KD)
constexpr int A_PART = HROWS * KC * 2;   // one part of an A chunk: 128 rows x 64 K x 2 B = 16 KB
constexpr int A_CHUNK = NPART * A_PART;  // A chunk of one row half, both parts: 32 KB
constexpr int FLUSH = 2;           // offsets accumulated in FP32 before the float-float update
constexpr int NU = 189;            // offsets of a child octant
constexpr int KS = 2;              // K halves: offsets [0, 95) and [95, 189)
constexpr int NCODE = 343;         // offset codes ((dx+3)*7 + dy+3)*7 + dz+3
constexpr int OP_ROW_EXP = 12;     // operator rows scaled to a largest entry in [2^11, 2^12)
constexpr int SRC_EXP = 14;        // sources scaled to a largest magnitude below 2^14
constexpr int STATUS_GRID_TIMEOUT = 4;       // a pipeline wait gave up
constexpr int STATUS_GRID_DRAIN = 8;         // work in flight did not finish within 2 s
constexpr int STATUS_GRID_ALIGN = 16;        // shared memory not 1024-byte aligned (nothing ran)

// reduced real layout of a solid of order GP: row n at n^2: Re m=0..n, Im m=1..n
__host__ __device__ inline void reduced_index(int e, int *n, int *m, bool *im) {
    int nn = 0;
    while ((nn + 1) * (nn + 1) <= e) ++nn;
    const int q = e - nn * nn;
    *n = nn;
    *im = q > nn;
    *m = *im ? q - nn : q;
}

// first offset of K half ks (KS halves of the NU offsets)
__host__ __device__ inline int k_begin(int ks) { return (ks * NU + KS - 1) / KS; }

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor of a K-major operand.  layout 0: no swizzle,
// core matrices of 8 rows x 16 bytes, lbo = byte step between core matrices
// along K, sbo = along M/N.  layout 2: 128-byte swizzle, rows of 128 bytes,
// sbo = step between groups of 8 rows; the K = 16 steps inside a row start
// 32 bytes apart.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(layout & 7) << 61;
    return d;
}

// byte offset of (row r, k) inside a [rows x KC] FP16 K-major tile of core
// matrices of 8 rows x 8 K (16 bytes per row)
__host__ __device__ __forceinline__ int koff(int r, int k) {
    return ((r >> 3) * (KC / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// v = hi + lo in FP16 (11 significant bits each, 22 together)
__device__ __forceinline__ void split2(double v, __half *hi, __half *lo) {
    const __half h = __double2half(v);
    *hi = h;
    *lo = __double2half(v - (double)__half2float(h));
}
__device__ __forceinline__ void split2f(float v, __half *hi, __half *lo) {
    const __half h = __float2half_rn(v);
    *hi = h;
    *lo = __float2half_rn(v - __half2float(h));
}

// ----------------------------------------------------------------- kernels

// per-coefficient scale factors (n(n+1)/2 + m): c/h^{n+1} for packing, c/h^n for unpacking
struct Scales {
    double s[GP * (GP + 1) / 2];
};

// index tables of the two layouts (filled by sfmm_grid_create):
//   reduced index e (row n at n^2: Re m = 0..n, Im m = 1..n) -> position in a
//   solid and scale index n(n+1)/2 + m;  solid position p -> reduced index
//   (-1 for Im C_n^0, which the reduced layout drops) and scale index
constexpr int SOLID = GP * (GP + 1);
__constant__ short c_pos_of_e[KD];
__constant__ unsigned char c_sidx_of_e[KD];
__constant__ short c_e_of_pos[SOLID];
__constant__ unsigned char c_sidx_of_pos[SOLID];

// The three kernels below give every thread one fixed coefficient (its
// table entries and scale factor are read once: lanes reading different
// entries of constant or parameter memory would be serialised) and let the
// blocks stride over boxes, four boxes' loads in flight per thread.
constexpr int SOLID_THREADS = 288;             // SOLID rounded up to whole warps

// largest |x| of the level's sources (float bits of a non-negative float
// order like unsigned integers), one atomicMax per block
__global__ void __launch_bounds__(SOLID_THREADS) xmax_kernel(const double *M, long long nboxes, Scales sc,
                                                             unsigned int *xmax) {
    const int p = threadIdx.x;
    float v = 0.f;
    if (p < SOLID) {
        const double f = sc.s[c_sidx_of_pos[p]];
#pragma unroll 4
        for (long long b = blockIdx.x; b < nboxes; b += gridDim.x)
            v = fmaxf(v, fabsf((float)(M[b * SOLID + p] * f)));
    }
    for (int d = 16; d > 0; d >>= 1) v = fmaxf(v, __shfl_xor_sync(0xffffffffu, v, d));
    __shared__ float wmax[SOLID_THREADS / 32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        float b = 0.f;
        for (int w = 0; w < SOLID_THREADS / 32; ++w) b = fmaxf(b, wmax[w]);
        atomicMax(xmax, __float_as_uint(b));
    }
}

// exponent g of the sources' scale 2^g: largest |x| * 2^g < 2^SRC_EXP
__device__ __forceinline__ int source_exp(const unsigned int *xmax) {
    const float m = __uint_as_float(*xmax);
    if (!(m > 0.f)) return 0;
    int e;
    frexpf(m, &e);                       // m < 2^e
    return SRC_EXP - e;
}

// x = M c / h^{k+1} 2^g in the reduced layout on the halo grid, split into FP16
// hi and lo.  The halo grid (side nh = nside + 6, even) is stored split by
// coordinate parity, [px py pz][hx/2][hy/2][hz/2][KD], so that the sources of
// a tile of same-parity targets under one offset form one dense box.  Thread
// e of a block writes coefficient e of the halo boxes the block strides over.
__global__ void __launch_bounds__(KD) pack_kernel(const double *M, int nside, Scales sc,
                                                  const unsigned int *xmax, __half *xhi, __half *xlo) {
    const int nh2 = (nside + 6) / 2, nrows = 8 * nh2 * nh2;
    const int e = threadIdx.x;
    const int pos = c_pos_of_e[e];
    const double f = sc.s[c_sidx_of_e[e]];
    const float g = ldexpf(1.f, source_exp(xmax));
    // blocks stride over rows (parity, hx2, hy2) of the halo grid and walk the
    // row's nh2 boxes along z, so the index divisions happen once per row
    for (int row = blockIdx.x; row < nrows; row += gridDim.x) {
        const int hy2 = row % nh2, hx2 = (row / nh2) % nh2, par = row / (nh2 * nh2);
        const int hx = 2 * hx2 + ((par >> 2) & 1) - 3, hy = 2 * hy2 + ((par >> 1) & 1) - 3;
        const bool xy_in = hx >= 0 && hx < nside && hy >= 0 && hy < nside;
        const long long xy_box = ((long long)hx * nside + hy) * nside;
        const long long blk0 = (long long)row * nh2;
#pragma unroll 4
        for (int hz2 = 0; hz2 < nh2; ++hz2) {
            const int hz = 2 * hz2 + (par & 1) - 3;
            float v = 0.f;
            if (xy_in && hz >= 0 && hz < nside)
                v = (float)(M[(xy_box + hz) * SOLID + pos] * f) * g;   // the power of two is exact
            const long long i = (blk0 + hz2) * KD + e;
            split2f(v, xhi + i, xlo + i);
        }
    }
}

// L (+)= (sum over the K halves, in order) y 2^{-row_exp - g} c / h^n from the
// reduced layout; thread p of a block writes coefficient p of its boxes.
__global__ void __launch_bounds__(SOLID_THREADS) unpack_kernel(const double *ypart, int nside, Scales sc,
                                                               const int *row_exp, const unsigned int *xmax,
                                                               double *L, int accumulate) {
    const long long nb = (long long)nside * nside * nside;
    const int p = threadIdx.x;
    if (p >= SOLID) return;
    const int e = c_e_of_pos[p];
    const double f = e >= 0 ? ldexp(sc.s[c_sidx_of_pos[p]], -row_exp[e] - source_exp(xmax)) : 0.0;
#pragma unroll 4
    for (long long b = blockIdx.x; b < nb; b += gridDim.x) {
        double v = 0.0;
        if (e >= 0) {
            double y = 0.0;
            for (int ks = 0; ks < KS; ++ks) y += ypart[((long long)ks * nb + b) * KD + e];
            v = y * f;
        }
        double *dst = L + b * SOLID + p;
        *dst = accumulate ? *dst + v : v;
    }
}

// largest |T_u[e'][j]| over every offset and column, one block per operator row e'
__global__ void operator_rowmax_kernel(const double *L, int ncodes, const double *c, double *rowmax) {
    const int ep = blockIdx.x;
    int n, m;
    bool im;
    reduced_index(ep, &n, &m, &im);
    const int pos = n * (n + 1) + (im ? n + 1 + m : m);
    const double ic = 1.0 / c[n * (n + 1) / 2 + m];
    double v = 0.0;
    for (int i = threadIdx.x; i < ncodes * KD; i += blockDim.x)
        v = fmax(v, fabs(L[(long long)i * (GP * (GP + 1)) + pos] * ic));
    for (int d = 16; d > 0; d >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, d));
    __shared__ double wmax[32];
    if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double b = 0.0;
        for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmax(b, wmax[w]);
        rowmax[ep] = b;
    }
}

// operators: T[code][e'][j] from the FP64 M2L of basis vector j (raw solid of
// order GP), converted to y = L / c in the reduced layout, scaled by
// 2^row_exp[e'] and split hi/lo; stored pre-tiled as
// [code][chunk][row half][hi | lo][K-major core-matrix tile of 128 rows x KC]
__global__ void operator_kernel(const double *L, const int *codes, int ncodes, const double *c,
                                const int *row_exp, __half *top) {
    const long long total = (long long)ncodes * KD * KD;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const int k = (int)(i / (KD * KD));
        const int ep = (int)((i / KD) % KD);
        const int j = (int)(i % KD);
        int n, m;
        bool im;
        reduced_index(ep, &n, &m, &im);
        const double *s = L + ((long long)k * KD + j) * (GP * (GP + 1));
        const double v = ldexp(s[n * (n + 1) + (im ? n + 1 + m : m)] / c[n * (n + 1) / 2 + m], row_exp[ep]);
        const int ch = j / KC, kk = j % KC, hh = ep / HROWS, r = ep % HROWS;
        unsigned char *base = reinterpret_cast<unsigned char *>(top) +
                              (((long long)codes[k] * NKC + ch) * 2 + hh) * A_CHUNK + koff(r, kk);
        split2(v, reinterpret_cast<__half *>(base), reinterpret_cast<__half *>(base + A_PART));
    }
}

struct GemmArgs {
    const __half *top;          // pre-tiled operators, [NCODE][NKC][2][hi|lo][A_PART bytes]
    double *ypart;              // [KS][ns^3][KD], FP64 sums of the two K halves
    int nside;
    int *status;
    long long inject_after;     // > 0: the copy thread acts as if its wait for a free
                                // stage timed out once it has issued this many chunks
                                // (fault injection for tests of the time-out path)
};

__device__ __forceinline__ bool try_wait(uint32_t bar, uint32_t parity) {
    uint32_t done;
    asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                 "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(parity) : "memory");
    return done != 0;
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// bounded wait (2^22 polls and 2 s at most) that also gives up once another
// role has raised the abort flag
__device__ __forceinline__ bool wait_or_abort(uint32_t bar, uint32_t parity, volatile int *abort_flag) {
    if (try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int it = 1; it < (1 << 22); ++it) {
        if (try_wait(bar, parity)) return true;
        if ((it & 255) == 0 && (*abort_flag || global_ns() - t0 > 2000000000ull)) return false;
    }
    return false;
}

// bounded wait for work already issued (the drains before the CTA frees its
// shared and tensor memory): it ignores the abort flag, because copies and
// MMAs in flight complete whether or not another role has given up, and stops
// after 2 s (or 2^24 polls)
__device__ __forceinline__ bool wait_bounded(uint32_t bar, uint32_t parity) {
    if (try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (int it = 1; it < (1 << 24); ++it) {
        if (try_wait(bar, parity)) return true;
        if ((it & 255) == 0 && global_ns() - t0 > 2000000000ull) return false;
    }
    return false;
}

// 32 consecutive tensor-memory columns of the warp's 32 lanes: thread = lane
__device__ __forceinline__ void tmem_ld32(uint32_t ta, uint32_t *v) {
    asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                 "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                 "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                 : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                   "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                   "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                   "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
                 : "r"(ta));
}
__device__ __forceinline__ void tmem_st32(uint32_t ta, const uint32_t *v) {
    asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
                 "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                 "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                 :: "r"(ta), "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]),
                    "r"(v[8]), "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15]),
                    "r"(v[16]), "r"(v[17]), "r"(v[18]), "r"(v[19]), "r"(v[20]), "r"(v[21]), "r"(v[22]), "r"(v[23]),
                    "r"(v[24]), "r"(v[25]), "r"(v[26]), "r"(v[27]), "r"(v[28]), "r"(v[29]), "r"(v[30]), "r"(v[31])
                 : "memory");
}

// Work units: (tile, operator row half, K half), ordered K half, row half,
// octant, tile, and dealt round-robin to the persistent CTAs, so that the CTAs
// of one round run the same offset sequence on neighbouring tiles at the same
// time and the operator chunks in use stay few and are served from L2.  A unit
// walks the K chunks of its offsets in groups of GW chunks (FLUSH offsets),
// one FP32 accumulation each.
constexpr int GW = NKC * FLUSH;

// pipeline stages: 3 of 64 KB for 128-target tiles, 4 of 48 KB for 64-target tiles
template <int NT>
constexpr int n_stages() { return NT == 128 ? 3 : 4; }

// dynamic shared memory: the stages of A (hi, lo) and B (hi, lo), then 8 KB for
// the mbarriers, the TMEM slot, the abort flags and the offset codes of the 8 octants
template <int NT>
constexpr int smem_gemm() { return n_stages<NT>() * (A_CHUNK + NPART * NT * KC * 2) + 8192; }

// Persistent, warp-specialised GEMM over the work units.
//   warp 4, one thread: copies.  For chunk i it waits until the MMAs of chunk
//     i - NST have freed the stage (`empty`), sets the stage's `full` mbarrier
//     to expect the chunk's bytes and issues one bulk copy of the pre-tiled
//     T_u chunk of the unit's row half (hi and lo) and two 5-D tensor copies of
//     the targets' source vectors (hi and lo, 128-byte swizzled rows).
//   warp 5, one thread: MMA issue.  For chunk i it waits on `full`, issues the
//     chunk's twelve tcgen05.mma into one of two accumulator buffers and commits
//     them to the stage's `empty` mbarrier; the last chunk of a group is also
//     committed to `acc_full` of its buffer.
//   warps 0-3: epilogue.  For every group they wait on `acc_full`, read their
//     32 TMEM lanes (operator rows) of the buffer and add it into the unit's
//     float-float sums (two more TMEM column ranges), then arrive on
//     `acc_empty`, which the MMA thread waits on before it reuses the buffer.
//     After a unit's last group they write its sums once, in FP64.
// Every wait is bounded; a time-out sets the abort flag and the status word,
// the other roles give up their waits, the copy and MMA threads wait for their
// work in flight (bounded by time only, whatever the abort flag says), and the
// CTA frees its tensor memory and returns; if that drain also runs out, bit 8
// of the status word is set and the tensor memory is kept.
template <int NT>
__global__ void __launch_bounds__(192, 1)
grid_gemm_kernel(GemmArgs a, const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_lo) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int NST = n_stages<NT>();
    constexpr int B_PART = NT * KC * 2;             // 16 or 8 KB
    constexpr int STAGE = A_CHUNK + NPART * B_PART;
    constexpr int TZ = NT / 16;                     // tile depth along z
    // tensor memory: [0, 2 NT) FP32 accumulators (two buffers), [2 NT, 3 NT)
    // float-float high parts, [3 NT, 4 NT) low parts
    constexpr uint32_t TCOLS = 4 * NT;
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + NST * STAGE);
    uint64_t *empty = full + NST;
    uint64_t *acc_full = empty + NST;
    uint64_t *acc_empty = acc_full + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(acc_empty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    volatile int *drain_failed = abort_flag + 1;
    int *codes = reinterpret_cast<int *>(sm + NST * STAGE + 1024);   // [8][NU]
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int ns = a.nside, half_ns = ns / 2, tpd = half_ns / 4, tpz = half_ns / TZ;
    const int tiles = tpd * tpd * tpz;
    const int n_tiles = 8 * tiles;
    const int n_units = KS * 2 * n_tiles;
    const int G = gridDim.x;
    const long long nb = (long long)ns * ns * ns;
    // the 128-byte swizzled tiles need 1024-byte aligned stages
    if (smem_u32(sm) & 1023u) {
        if (tid == 0) atomicOr(a.status, STATUS_GRID_ALIGN);
        return;
    }

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tslot)), "r"(TCOLS));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 32) {
        for (int i = 0; i < NST; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(full + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(empty + i)));
        }
        for (int b = 0; b < 2; ++b) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(acc_full + b)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 4;" :: "r"(smem_u32(acc_empty + b)));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *abort_flag = 0;
        *drain_failed = 0;
    }
    if (tid >= 64 && tid < 72) {
        // octant o: offsets u = target - source with u_i in [-3 + b_i, 2 + b_i], max|u_i| >= 2
        const int o = tid - 64, bx = (o >> 2) & 1, by = (o >> 1) & 1, bz = o & 1;
        int nu = 0;
        for (int dx = -3 + bx; dx <= 2 + bx; ++dx)
            for (int dy = -3 + by; dy <= 2 + by; ++dy)
                for (int dz = -3 + bz; dz <= 2 + bz; ++dz) {
                    const int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
                    if ((ax > ay ? (ax > az ? ax : az) : (ay > az ? ay : az)) >= 2)
                        codes[o * NU + nu++] = ((dx + 3) * 7 + (dy + 3)) * 7 + (dz + 3);
                }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(a.status, STATUS_GRID_TIMEOUT);
    };
    auto drain_fail = [&]() {
        *drain_failed = 1;
        atomicOr(a.status, STATUS_GRID_DRAIN);
    };

    if (warp == 4) {
        if (lane == 0) {
            long long i = 0;
            long long last[NST];
            for (int s = 0; s < NST; ++s) last[s] = -1;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += G) {
                const int tile_g = u % n_tiles, hh = (u / n_tiles) & 1, ks = u / (2 * n_tiles);
                const int c_begin = k_begin(ks) * NKC, c_end = k_begin(ks + 1) * NKC;
                const int cls = tile_g / tiles, tile = tile_g % tiles;
                const int bx = (cls >> 2) & 1, by = (cls >> 1) & 1, bz = cls & 1;
                const int tx = tile / (tpd * tpz), ty = (tile / tpz) % tpd, tz = tile % tpz;
                int c1 = 0, c2 = 0, c3 = 0, c4 = 0, code = 0;
                for (int ci = c_begin; ci < c_end; ++ci, ++i) {
                    if (ci == c_begin || ci % NKC == 0) {
                        code = codes[cls * NU + ci / NKC];
                        const int sx = bx - (code / 49 - 3) + 3, sy = by - ((code / 7) % 7 - 3) + 3,
                                  sz = bz - (code % 7 - 3) + 3;
                        c1 = tz * TZ + (sz >> 1);
                        c2 = ty * 4 + (sy >> 1);
                        c3 = tx * 4 + (sx >> 1);
                        c4 = ((sx & 1) << 2) | ((sy & 1) << 1) | (sz & 1);
                    }
                    const int stg = (int)(i % NST), kc = (ci % NKC) * KC;
                    if ((a.inject_after > 0 && i >= a.inject_after) ||
                        (i >= NST && !wait_or_abort(smem_u32(empty + stg), (uint32_t)(((i / NST) - 1) & 1), abort_flag))) {
                        fail();
                        ok = false;
                        break;
                    }
                    const uint32_t dst = smem_u32(sm + stg * STAGE), bar = smem_u32(full + stg);
                    const unsigned char *src = reinterpret_cast<const unsigned char *>(a.top) +
                                               (((long long)code * NKC + (ci % NKC)) * 2 + hh) * A_CHUNK;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(STAGE) : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 :: "r"(dst), "l"(src), "r"(A_CHUNK), "r"(bar) : "memory");
                    const CUtensorMap *maps[NPART] = {&tm_hi, &tm_lo};
#pragma unroll
                    for (int p = 0; p < NPART; ++p)
                        asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                                     " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                                     :: "r"(dst + A_CHUNK + p * B_PART), "l"(reinterpret_cast<uint64_t>(maps[p])),
                                        "r"(kc), "r"(c1), "r"(c2), "r"(c3), "r"(c4), "r"(bar) : "memory");
                    last[stg] = i;
                }
            }
            // drain: every copy issued has landed before the CTA frees its memory
            for (int s = 0; s < NST; ++s)
                if (last[s] >= 0 && !wait_bounded(smem_u32(full + s), (uint32_t)((last[s] / NST) & 1))) drain_fail();
        }
        __syncwarp();
    } else if (warp == 5) {
        if (lane == 0) {
            // D = FP32, A = B = FP16, both K-major, N = NT, M = 128
            const uint32_t idesc = (1u << 4) | ((uint32_t)(NT >> 3) << 17) | ((uint32_t)(128 >> 4) << 24);
            // descriptors of stage 0; stage s adds s * STAGE to the address field.
            // A: no swizzle, core matrices 128 B apart along K, 8-row groups (KC / 8) * 128 B
            // apart, K = 16 steps 256 B apart; B: 128-byte swizzle, 8-row groups of
            // 128-byte rows 1024 B apart, K = 16 steps 32 B apart
            const uint32_t s0 = smem_u32(sm);
            const uint64_t dA = sdesc(s0, 128, (KC / 8) * 128, 0);
            const uint64_t dB = sdesc(s0 + A_CHUNK, 16, 1024, 2);
            long long i = 0, g = 0, last_mma = -1;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += G) {
                const int ks = u / (2 * n_tiles);
                const int c_begin = k_begin(ks) * NKC, c_end = k_begin(ks + 1) * NKC;
                for (int gb = c_begin; gb < c_end && ok; gb += GW, ++g) {
                    const int ge = (gb + GW < c_end) ? gb + GW : c_end;
                    const int b = (int)(g & 1);
                    if (g >= 2 && !wait_or_abort(smem_u32(acc_empty + b), (uint32_t)(((g >> 1) - 1) & 1), abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint32_t d = tmem + (uint32_t)b * NT;
                    for (int ci = gb; ci < ge; ++ci, ++i) {
                        const int stg = (int)(i % NST);
                        if (!wait_or_abort(smem_u32(full + stg), (uint32_t)((i / NST) & 1), abort_flag)) {
                            fail();
                            ok = false;
                            break;
                        }
                        asm volatile("tcgen05.fence::after_thread_sync;");
                        const uint64_t so = (uint64_t)((stg * STAGE) >> 4);
                        // per K = 16 step, three products of the parts: hi*hi, hi*lo, lo*hi
                        constexpr int PA[3] = {0, 0, 1}, PB[3] = {0, 1, 0};
#pragma unroll
                        for (int kk = 0; kk < KC / UK; ++kk)
#pragma unroll
                            for (int t = 0; t < 3; ++t) {
                                const uint64_t ad = dA + so + ((PA[t] * A_PART + kk * (UK / 8) * 128) >> 4);
                                const uint64_t bd = dB + so + ((PB[t] * B_PART + kk * UK * 2) >> 4);
                                const uint32_t acc = (ci == gb && kk == 0 && t == 0) ? 0u : 1u;
                                asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                             "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}"
                                             :: "r"(d), "l"(ad), "l"(bd), "r"(idesc), "r"(acc));
                            }
                        asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                     :: "r"(smem_u32(empty + stg)) : "memory");
                        last_mma = i;
                    }
                    if (!ok) break;
                    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                                 :: "r"(smem_u32(acc_full + b)) : "memory");
                }
            }
            // drain: the MMAs issued have completed before the CTA frees its memory
            if (last_mma >= 0 && !wait_bounded(smem_u32(empty + last_mma % NST), (uint32_t)((last_mma / NST) & 1))) drain_fail();
        }
        __syncwarp();
    } else {
        // epilogue: warp w owns TMEM lanes (operator rows) 32 w .. 32 w + 31
        const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
        long long g = 0;
        bool ok = true;
        for (int u = blockIdx.x; u < n_units && ok; u += G) {
            const int tile_g = u % n_tiles, hh = (u / n_tiles) & 1, ks = u / (2 * n_tiles);
            const int c_begin = k_begin(ks) * NKC, c_end = k_begin(ks + 1) * NKC;
            bool first = true;
            for (int gb = c_begin; gb < c_end; gb += GW, ++g) {
                const int b = (int)(g & 1);
                bool got = true;
                if (lane == 0) got = wait_or_abort(smem_u32(acc_full + b), (uint32_t)((g >> 1) & 1), abort_flag);
                got = __shfl_sync(0xffffffffu, got ? 1 : 0, 0) != 0;
                if (!got) {
                    if (lane == 0) fail();
                    ok = false;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                for (int c0 = 0; c0 < NT; c0 += 32) {
                    uint32_t va[32], vh[32], vl[32];
                    tmem_ld32(tmem + lane_base + (uint32_t)(b * NT + c0), va);
                    if (!first) {
                        tmem_ld32(tmem + lane_base + (uint32_t)(2 * NT + c0), vh);
                        tmem_ld32(tmem + lane_base + (uint32_t)(3 * NT + c0), vl);
                    }
                    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                    for (int j = 0; j < 32; ++j) {
                        const float x = __uint_as_float(va[j]);
                        float hi = x, lo = 0.f;
                        if (!first) {
                            // two-sum: h0 + x = s + err exactly, then lo += err
                            const float h0 = __uint_as_float(vh[j]);
                            const float s = __fadd_rn(h0, x);
                            const float bb = __fsub_rn(s, h0);
                            const float err = __fadd_rn(__fsub_rn(h0, __fsub_rn(s, bb)), __fsub_rn(x, bb));
                            hi = s;
                            lo = __fadd_rn(__uint_as_float(vl[j]), err);
                        }
                        vh[j] = __float_as_uint(hi);
                        vl[j] = __float_as_uint(lo);
                    }
                    tmem_st32(tmem + lane_base + (uint32_t)(2 * NT + c0), vh);
                    tmem_st32(tmem + lane_base + (uint32_t)(3 * NT + c0), vl);
                }
                asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                asm volatile("tcgen05.fence::before_thread_sync;");
                __syncwarp();
                if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(acc_empty + b)) : "memory");
                first = false;
            }
            if (!ok) break;
            // the unit's sums, once, in FP64: row = operator row, column = target
            const int cls = tile_g / tiles, tile = tile_g % tiles;
            const int bx = (cls >> 2) & 1, by = (cls >> 1) & 1, bz = cls & 1;
            const int tx = tile / (tpd * tpz), ty = (tile / tpz) % tpd, tz = tile % tpz;
            const int row = hh * HROWS + warp * 32 + lane;
            double *yk = a.ypart + (long long)ks * nb * KD + row;
            for (int c0 = 0; c0 < NT; c0 += 32) {
                uint32_t vh[32], vl[32];
                tmem_ld32(tmem + lane_base + (uint32_t)(2 * NT + c0), vh);
                tmem_ld32(tmem + lane_base + (uint32_t)(3 * NT + c0), vl);
                asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
                for (int jj = 0; jj < 32; ++jj) {
                    const int j = c0 + jj;
                    const int x = 2 * (tx * 4 + (j / (4 * TZ))) + bx;
                    const int y = 2 * (ty * 4 + ((j / TZ) & 3)) + by;
                    const int z = 2 * (tz * TZ + (j % TZ)) + bz;
                    yk[(((long long)x * ns + y) * ns + z) * KD] =
                        (double)__uint_as_float(vh[jj]) + (double)__uint_as_float(vl[jj]);
                }
            }
        }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    // tensor memory that MMAs may still write is not freed (status bit 8)
    if (warp == 0 && !*drain_failed)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(TCOLS));
}

}  // namespace

struct sfmm_grid_ctx {
    sfmm_handle h = nullptr;
    int P = GP, nside = 0;
    __half *top = nullptr;                   // operators, pre-tiled hi|lo FP16 chunks
    __half *xhi = nullptr, *xlo = nullptr;   // packed sources (FP16 parts)
    double *ypart = nullptr;                 // FP64 sums of the two K halves
    double *c = nullptr;                     // sqrt((n-m)!(n+m)!) on the device
    int *row_exp = nullptr;                  // power-of-two scale of every operator row
    unsigned int *xmax = nullptr;            // largest |x| of the current call (float bits)
    std::vector<double> ch;                  // c on the host
    CUtensorMap tm_hi, tm_lo;                // 5-D maps of the source parts (tile boxes)
    int nt = 0;                              // targets per tile: 128 or 64
    long long inject_after = 0;              // fault injection, see sfmm_grid_inject_timeout
};

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// map of the parity-split halo grid [8][nh/2][nh/2][nh/2][KD] (innermost last)
// with boxes of KC FP16 values x tz x 4 x 4 boxes x 1 parity class, 128-byte swizzle
bool encode_source_map(EncodeTiled enc, CUtensorMap *m, __half *base, int nside, int tz) {
    const cuuint64_t nh2 = (cuuint64_t)(nside + 6) / 2;
    const cuuint64_t dims[5] = {(cuuint64_t)KD, nh2, nh2, nh2, 8};
    const cuuint64_t row = (cuuint64_t)KD * sizeof(__half);
    const cuuint64_t strides[4] = {row, row * nh2, row * nh2 * nh2, row * nh2 * nh2 * nh2};
    const cuuint32_t box[5] = {(cuuint32_t)KC, (cuuint32_t)tz, 4, 4, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 5, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" {

sfmm_status sfmm_grid_create(sfmm_handle h, int P, int nside, sfmm_grid *out) {
    SfmmRange nvtx_range("sfmm_grid_create");
    if (out == nullptr || h == nullptr) return SFMM_ERR_ARG;
    *out = nullptr;
    if (P != GP) return SFMM_ERR_UNSUPPORTED;
    if (h->dtype != SFMM_F64 || h->Pmax < GP) return SFMM_ERR_ORDER;
    if (nside < 8 || nside % 8 != 0) return SFMM_ERR_ARG;
    sfmm_grid_ctx *g = new (std::nothrow) sfmm_grid_ctx;
    if (g == nullptr) return SFMM_ERR_NOMEM;
    g->h = h;
    g->nside = nside;
    const long long nh = nside + 6;
    const size_t op_bytes = (size_t)NCODE * NKC * 2 * A_CHUNK;
    const size_t x_bytes = sizeof(__half) * (size_t)(nh * nh * nh) * KD;
    bool ok = cudaMalloc(&g->top, op_bytes) == cudaSuccess &&
              cudaMalloc(&g->xhi, x_bytes) == cudaSuccess &&
              cudaMalloc(&g->xlo, x_bytes) == cudaSuccess &&
              cudaMalloc(&g->ypart, sizeof(double) * KS * (size_t)nside * nside * nside * KD) == cudaSuccess &&
              cudaMalloc(&g->c, sizeof(double) * GP * (GP + 1) / 2) == cudaSuccess &&
              cudaMalloc(&g->row_exp, sizeof(int) * KD) == cudaSuccess &&
              cudaMalloc(&g->xmax, sizeof(unsigned int)) == cudaSuccess;
    if (!ok) { sfmm_grid_destroy(g); return SFMM_ERR_NOMEM; }
    cudaMemset(g->top, 0, op_bytes);
    std::vector<double> c(GP * (GP + 1) / 2);
    {
        std::vector<double> f(2 * GP + 1, 1.0);
        for (int j = 1; j <= 2 * GP; ++j) f[j] = f[j - 1] * j;
        for (int n = 0; n < GP; ++n)
            for (int m = 0; m <= n; ++m) c[n * (n + 1) / 2 + m] = std::sqrt(f[n - m]) * std::sqrt(f[n + m]);
    }
    cudaMemcpy(g->c, c.data(), sizeof(double) * c.size(), cudaMemcpyHostToDevice);
    g->ch = c;
    {
        short pos_of_e[KD], e_of_pos[SOLID];
        unsigned char sidx_of_e[KD], sidx_of_pos[SOLID];
        for (int e = 0; e < KD; ++e) {
            int n, m;
            bool im;
            reduced_index(e, &n, &m, &im);
            pos_of_e[e] = (short)(n * (n + 1) + (im ? n + 1 + m : m));
            sidx_of_e[e] = (unsigned char)(n * (n + 1) / 2 + m);
        }
        for (int p = 0; p < SOLID; ++p) {
            int n = 0;
            while ((n + 1) * (n + 2) <= p) ++n;
            const int q = p - n * (n + 1);
            const bool im = q > n;
            const int m = im ? q - n - 1 : q;
            e_of_pos[p] = (short)((im && m == 0) ? -1 : n * n + (im ? n + m : m));
            sidx_of_pos[p] = (unsigned char)(n * (n + 1) / 2 + m);
        }
        if (cudaMemcpyToSymbol(c_pos_of_e, pos_of_e, sizeof(pos_of_e)) != cudaSuccess ||
            cudaMemcpyToSymbol(c_sidx_of_e, sidx_of_e, sizeof(sidx_of_e)) != cudaSuccess ||
            cudaMemcpyToSymbol(c_e_of_pos, e_of_pos, sizeof(e_of_pos)) != cudaSuccess ||
            cudaMemcpyToSymbol(c_sidx_of_pos, sidx_of_pos, sizeof(sidx_of_pos)) != cudaSuccess) {
            sfmm_grid_destroy(g);
            return SFMM_ERR_CUDA;
        }
    }
    // operators: M2L (FP64, rotation-based) of the KD basis vectors for every offset
    std::vector<int> codes;
    for (int dx = -3; dx <= 3; ++dx)
        for (int dy = -3; dy <= 3; ++dy)
            for (int dz = -3; dz <= 3; ++dz)
                if (std::max(std::abs(dx), std::max(std::abs(dy), std::abs(dz))) >= 2)
                    codes.push_back(((dx + 3) * 7 + (dy + 3)) * 7 + (dz + 3));
    const int ncodes = (int)codes.size();                   // 316
    const int S = GP * (GP + 1);
    std::vector<double> basis((size_t)KD * S, 0.0);
    for (int j = 0; j < KD; ++j) {
        int n = 0;
        while ((n + 1) * (n + 1) <= j) ++n;
        const int q = j - n * n;
        const bool im = q > n;
        const int m = im ? q - n : q;
        basis[(size_t)j * S + n * (n + 1) + (im ? n + 1 + m : m)] = 1.0 / c[n * (n + 1) / 2 + m];
    }
    const long long count = (long long)ncodes * KD;
    std::vector<double> shift(3 * count);
    std::vector<long long> pin(count), pout(count);
    double *dbasis = nullptr, *dL = nullptr, *dshift = nullptr, *drowmax = nullptr;
    long long *dpin = nullptr, *dpout = nullptr;
    int *dcodes = nullptr;
    ok = cudaMalloc(&dbasis, sizeof(double) * basis.size()) == cudaSuccess &&
         cudaMalloc(&dL, sizeof(double) * count * S) == cudaSuccess &&
         cudaMalloc(&dshift, sizeof(double) * shift.size()) == cudaSuccess &&
         cudaMalloc(&dpin, sizeof(long long) * count) == cudaSuccess &&
         cudaMalloc(&dpout, sizeof(long long) * count) == cudaSuccess &&
         cudaMalloc(&dcodes, sizeof(int) * ncodes) == cudaSuccess &&
         cudaMalloc(&drowmax, sizeof(double) * KD) == cudaSuccess;
    sfmm_status st = ok ? SFMM_OK : SFMM_ERR_NOMEM;
    if (st == SFMM_OK) {
        for (int k = 0; k < ncodes; ++k) {
            const int code = codes[k];
            const double ux = code / 49 - 3, uy = (code / 7) % 7 - 3, uz = code % 7 - 3;
            for (int j = 0; j < KD; ++j) {
                const long long i = (long long)k * KD + j;
                shift[3 * i] = ux;                      // r = target - source = u (unit boxes)
                shift[3 * i + 1] = uy;
                shift[3 * i + 2] = uz;
                pin[i] = (long long)(dbasis + (size_t)j * S);
                pout[i] = (long long)(dL + (size_t)i * S);
            }
        }
        cudaMemcpy(dbasis, basis.data(), sizeof(double) * basis.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dshift, shift.data(), sizeof(double) * shift.size(), cudaMemcpyHostToDevice);
        cudaMemcpy(dpin, pin.data(), sizeof(long long) * count, cudaMemcpyHostToDevice);
        cudaMemcpy(dpout, pout.data(), sizeof(long long) * count, cudaMemcpyHostToDevice);
        cudaMemcpy(dcodes, codes.data(), sizeof(int) * ncodes, cudaMemcpyHostToDevice);
        st = sfmm_m2l_batch(h, reinterpret_cast<const void *const *>(dpin),
                            reinterpret_cast<void *const *>(dpout), dshift, GP, GP, count, 0, nullptr);
    }
    if (st == SFMM_OK) {
        // operator row scales 2^e: the row's largest entry times 2^e lies in
        // [2^(OP_ROW_EXP-1), 2^OP_ROW_EXP)
        operator_rowmax_kernel<<<KD, 256>>>(dL, ncodes, g->c, drowmax);
        std::vector<double> rowmax(KD);
        std::vector<int> rexp(KD, 0);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpy(rowmax.data(), drowmax, sizeof(double) * KD, cudaMemcpyDeviceToHost) != cudaSuccess)
            st = SFMM_ERR_CUDA;
        for (int e = 0; e < KD && st == SFMM_OK; ++e) {
            int ex = 0;
            if (rowmax[e] > 0.0) std::frexp(rowmax[e], &ex);      // rowmax < 2^ex
            rexp[e] = OP_ROW_EXP - ex;
        }
        if (st == SFMM_OK && cudaMemcpy(g->row_exp, rexp.data(), sizeof(int) * KD, cudaMemcpyHostToDevice) != cudaSuccess)
            st = SFMM_ERR_CUDA;
    }
    if (st == SFMM_OK) {
        operator_kernel<<<1024, 256>>>(dL, dcodes, ncodes, g->c, g->row_exp, g->top);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) st = SFMM_ERR_CUDA;
    }
    cudaFree(dbasis);
    cudaFree(dL);
    cudaFree(dshift);
    cudaFree(dpin);
    cudaFree(dpout);
    cudaFree(dcodes);
    cudaFree(drowmax);
    if (st == SFMM_OK &&
        (cudaFuncSetAttribute(grid_gemm_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_gemm<64>()) != cudaSuccess ||
         cudaFuncSetAttribute(grid_gemm_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_gemm<128>()) != cudaSuccess))
        st = SFMM_ERR_CUDA;
    g->nt = (nside % 16 == 0) ? 128 : 64;
    if (st == SFMM_OK) {
        void *fn = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault, &q) != cudaSuccess ||
            q != cudaDriverEntryPointSuccess || fn == nullptr ||
            !encode_source_map(reinterpret_cast<EncodeTiled>(fn), &g->tm_hi, g->xhi, nside, g->nt / 16) ||
            !encode_source_map(reinterpret_cast<EncodeTiled>(fn), &g->tm_lo, g->xlo, nside, g->nt / 16))
            st = SFMM_ERR_CUDA;
    }
    if (st != SFMM_OK) {
        sfmm_grid_destroy(g);
        return st;
    }
    *out = g;
    return SFMM_OK;
}

sfmm_status sfmm_grid_destroy(sfmm_grid g) {
    if (g == nullptr) return SFMM_OK;
    cudaDeviceSynchronize();
    cudaFree(g->top);
    cudaFree(g->xhi);
    cudaFree(g->xlo);
    cudaFree(g->ypart);
    cudaFree(g->c);
    cudaFree(g->row_exp);
    cudaFree(g->xmax);
    delete g;
    return SFMM_OK;
}

sfmm_status sfmm_grid_inject_timeout(sfmm_grid g, long long after_chunks) {
    if (g == nullptr || after_chunks < 0) return SFMM_ERR_ARG;
    g->inject_after = after_chunks;
    return SFMM_OK;
}

sfmm_status sfmm_grid_m2l(sfmm_grid g, double box_size, const void *M, void *L, int accumulate,
                          sfmm_stream stream) {
    SfmmRange nvtx_range("sfmm_grid_m2l");
    if (g == nullptr || M == nullptr || L == nullptr || !(box_size > 0)) return SFMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int ns = g->nside;
    Scales sp, su;
    for (int n = 0; n < GP; ++n) {
        const double hn = std::pow(box_size, n);
        for (int m = 0; m <= n; ++m) {
            sp.s[n * (n + 1) / 2 + m] = g->ch[n * (n + 1) / 2 + m] / (hn * box_size);
            su.s[n * (n + 1) / 2 + m] = g->ch[n * (n + 1) / 2 + m] / hn;
        }
    }
    const long long nb = (long long)ns * ns * ns;
    const int nh2 = (ns + 6) / 2;
    if (cudaMemsetAsync(g->xmax, 0, sizeof(unsigned int), s) != cudaSuccess) return SFMM_ERR_CUDA;
    xmax_kernel<<<(unsigned)(nb < 2048 ? nb : 2048), SOLID_THREADS, 0, s>>>(reinterpret_cast<const double *>(M), nb, sp, g->xmax);
    const int nrows = 8 * nh2 * nh2;
    pack_kernel<<<nrows < 4096 ? nrows : 4096, KD, 0, s>>>(reinterpret_cast<const double *>(M), ns, sp, g->xmax, g->xhi, g->xlo);
    // tiles of 4 x 4 x (nt / 16) same-octant targets; one persistent CTA per SM
    // deals the (tile, row half, K half) units round-robin
    GemmArgs a{g->top, g->ypart, ns, g->h->d_status, g->inject_after};
    const int ctas = g->h->sm_count > 0 ? g->h->sm_count : 1;
    if (g->nt == 128)
        grid_gemm_kernel<128><<<ctas, 192, smem_gemm<128>(), s>>>(a, g->tm_hi, g->tm_lo);
    else
        grid_gemm_kernel<64><<<ctas, 192, smem_gemm<64>(), s>>>(a, g->tm_hi, g->tm_lo);
    unpack_kernel<<<(unsigned)(nb < 4096 ? nb : 4096), SOLID_THREADS, 0, s>>>(g->ypart, ns, su, g->row_exp, g->xmax,
                                                                           reinterpret_cast<double *>(L), accumulate);
    return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
}

}  // extern "C"
