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
// tensor cores:
//   * T_u and x are split into three BF16 parts, hi + mid + lo (about 24
//     significant bits), and multiplied as the six products hi*hi, hi*mid,
//     mid*hi, hi*lo, lo*hi, mid*mid (tcgen05.mma kind::f16) with FP32
//     accumulation in tensor memory (two 128-row halves x 128 columns, two
//     buffers);
//   * every 2 offsets the accumulator is read out (tcgen05.ld) and added into
//     the target's FP64 sum in global memory (FP32 rounding over longer runs
//     of offsets pushed single targets above a 1e-5 relative error);
//   * operand chunks (16 of K) are staged in shared memory in five stages: the
//     T_u chunk, stored pre-tiled, by one bulk copy; the targets' source
//     vectors, stored split by coordinate parity, by three 5-D tensor copies;
//   * one thread issues copies, one issues MMAs, four warps drain the
//     accumulators; one persistent CTA per SM.
// T_u are built once per grid object with the FP64 rotation-based M2L on the
// 256 basis vectors of every offset.  Every mbarrier wait is bounded: on
// time-out the kernel records SFMM_GRID_TIMEOUT in the status word, stops
// issuing work, frees its tensor memory and returns.
#include <cuda.h>
#include <cuda_bf16.h>
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
constexpr int KC = 16;             // K chunk staged in shared memory (one BF16 MMA)
constexpr int NST = 5;             // pipeline stages
constexpr int NKC = KD / KC;       // chunks per offset
constexpr int NPART = 3;           // operand parts: hi, mid, lo (BF16 each)
constexpr int A_PART = KD * KC * 2;   // one part of an A chunk: 256 rows x 16 K x 2 B = 8 KB
constexpr int FLUSH = 2;           // offsets accumulated in FP32 before an FP64 flush
constexpr int NU = 189;            // offsets of a child octant
constexpr int NCH_ALL = NU * NKC;  // K chunks of a tile
constexpr int NCODE = 343;         // offset codes ((dx+3)*7 + dy+3)*7 + dz+3
constexpr int STATUS_GRID_TIMEOUT = 4;       // a pipeline wait gave up
constexpr int STATUS_GRID_DRAIN = 8;         // work in flight did not finish within 2 s

// reduced real layout of a solid of order GP: row n at n^2: Re m=0..n, Im m=1..n
__host__ __device__ inline void reduced_index(int e, int *n, int *m, bool *im) {
    int nn = 0;
    while ((nn + 1) * (nn + 1) <= e) ++nn;
    const int q = e - nn * nn;
    *n = nn;
    *im = q > nn;
    *m = *im ? q - nn : q;
}

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// shared-memory matrix descriptor of a K-major operand.  layout 0: no swizzle,
// core matrices of 8 rows x 16 bytes, lbo = byte step between core matrices
// along K, sbo = along M/N.  layout 4: 64-byte swizzle, rows of 64 bytes,
// sbo = step between groups of 8 rows (lbo unused).
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo, uint32_t layout) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)(layout & 7) << 61;
    return d;
}

// byte offset of (row r, k) inside a [rows x KC] BF16 K-major tile of core
// matrices of 8 rows x 8 K (16 bytes per row)
__device__ __forceinline__ int koff(int r, int k) {
    return ((r >> 3) * (KC / 8) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2;
}

// v = hi + mid + lo in BF16 (8 significant bits each): the three parts carry
// about 24 bits of v, the products dropped below (mid*lo, lo*mid, lo*lo) are
// of relative size 2^-24
__device__ __forceinline__ void split3(double v, unsigned short *hi, unsigned short *mid,
                                       unsigned short *lo) {
    // (FP64 arithmetic: used once per operator entry when a grid is created)
    const __nv_bfloat16 h = __double2bfloat16(v);
    const double r1 = v - (double)__bfloat162float(h);
    const __nv_bfloat16 m = __double2bfloat16(r1);
    const double r2 = r1 - (double)__bfloat162float(m);
    const __nv_bfloat16 l = __double2bfloat16(r2);
    *hi = __bfloat16_as_ushort(h);
    *mid = __bfloat16_as_ushort(m);
    *lo = __bfloat16_as_ushort(l);
}

// the same split of an FP32 value in FP32 arithmetic (the subtractions are
// exact): the per-call packing of the sources, where FP64 work would cost more
// than the copy itself on this GPU's FP64 pipe
__device__ __forceinline__ void split3f(float v, unsigned short *hi, unsigned short *mid,
                                        unsigned short *lo) {
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r1 = v - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r1);
    const float r2 = r1 - __bfloat162float(m);
    *hi = __bfloat16_as_ushort(h);
    *mid = __bfloat16_as_ushort(m);
    *lo = __bfloat16_as_ushort(__float2bfloat16_rn(r2));
}

// ----------------------------------------------------------------- kernels

// per-coefficient scale factors (n(n+1)/2 + m): c/h^{n+1} for packing, c/h^n for unpacking
struct Scales {
    double s[GP * (GP + 1) / 2];
};

// x = M c / h^{k+1} in the reduced layout on the halo grid, split into BF16 hi, mid, lo.
// The halo grid (side nh = nside + 6, even) is stored split by coordinate
// parity, [px py pz][hx/2][hy/2][hz/2][KD], so that the sources of a tile of
// same-parity targets under one offset form one dense box.
__global__ void pack_kernel(const double *M, int nside, Scales sc, unsigned short *xhi,
                            unsigned short *xmid, unsigned short *xlo) {
    const int nh = nside + 6, nh2 = nh / 2;
    const long long total = (long long)nh * nh * nh * KD;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / KD;
        const int e = (int)(i % KD);
        const int hz2 = (int)(b % nh2), hy2 = (int)((b / nh2) % nh2), hx2 = (int)((b / nh2 / nh2) % nh2);
        const int par = (int)(b / ((long long)nh2 * nh2 * nh2));
        const int hx = 2 * hx2 + ((par >> 2) & 1) - 3, hy = 2 * hy2 + ((par >> 1) & 1) - 3,
                  hz = 2 * hz2 + (par & 1) - 3;
        float v = 0.f;
        if (hx >= 0 && hx < nside && hy >= 0 && hy < nside && hz >= 0 && hz < nside) {
            int n, m;
            bool im;
            reduced_index(e, &n, &m, &im);
            const long long box_id = ((long long)hx * nside + hy) * nside + hz;
            const double *s = M + box_id * (GP * (GP + 1));
            const double val = s[n * (n + 1) + (im ? n + 1 + m : m)];
            v = (float)(val * sc.s[n * (n + 1) / 2 + m]);
        }
        split3f(v, xhi + i, xmid + i, xlo + i);
    }
}

// L (+)= y c / h^n from the reduced layout (FP64 accumulator y).
__global__ void unpack_kernel(const double *y, int nside, Scales sc, double *L, int accumulate) {
    const long long total = (long long)nside * nside * nside * (GP * (GP + 1));
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / (GP * (GP + 1));
        const int p = (int)(i % (GP * (GP + 1)));
        int n = 0;
        while ((n + 1) * (n + 2) <= p) ++n;
        const int q = p - n * (n + 1);
        const bool im = q > n;
        const int m = im ? q - n - 1 : q;
        double v = 0.0;
        if (!(im && m == 0)) {
            const int e = n * n + (im ? n + m : m);
            v = y[b * KD + e] * sc.s[n * (n + 1) / 2 + m];
        }
        L[i] = accumulate ? L[i] + v : v;
    }
}

// operators: T[code][e'][j] from the FP64 M2L of basis vector j (raw solid of
// order GP), converted to y = L / c in the reduced layout and split hi/mid/lo.
__global__ void operator_kernel(const double *L, const int *codes, int ncodes, const double *c,
                                unsigned short *top) {
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
        const double v = s[n * (n + 1) + (im ? n + 1 + m : m)] / c[n * (n + 1) / 2 + m];
        // pre-tiled: [code][chunk][hi|mid|lo][K-major core-matrix tile of 256 rows x KC]
        const int ch = j / KC, kk = j % KC;
        unsigned char *base = reinterpret_cast<unsigned char *>(top) +
                              ((long long)codes[k] * NKC + ch) * NPART * A_PART + koff(ep, kk);
        split3(v, reinterpret_cast<unsigned short *>(base), reinterpret_cast<unsigned short *>(base + A_PART),
               reinterpret_cast<unsigned short *>(base + 2 * A_PART));
    }
}

struct GemmArgs {
    const unsigned short *top;  // pre-tiled operators, [NCODE][NKC][hi|mid|lo][A_PART bytes]
    double *y;                  // [ns^3][KD], FP64 sums, zeroed before the launch
    int nside;
    int *status;
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

// Work units: (K slab, tile) pairs in slab-major order, a slab being the K
// chunks of GW consecutive chunks (FLUSH offsets) of a tile; one unit is one
// FP32 accumulation group.  CTA c takes units c, c + G, c + 2G, ... so that at
// any time all CTAs work on the same one or two slabs: the operator chunks and
// source slices in use at once stay few and are served from L2.
constexpr int GW = NKC * FLUSH;
constexpr int NSLAB = (NCH_ALL + GW - 1) / GW;

// dynamic shared memory: NST stages of A (hi, mid, lo) and B (hi, mid, lo), then
// 8 KB for the mbarriers, the TMEM slot, the abort flag and the offset codes of
// the 8 octants
template <int NT>
constexpr int smem_gemm() { return NST * (NPART * A_PART + NPART * NT * KC * 2) + 8192; }

// Persistent, warp-specialised GEMM over (K slab, tile) units dealt round-robin.
//   warp 4, one thread: copies.  For chunk i it waits until the MMAs of chunk
//     i - NST have freed the stage (`empty`), sets the stage's `full` mbarrier
//     to expect the chunk's bytes and issues one bulk copy of the pre-tiled
//     T_u chunk (A, hi, mid and lo) and three 5-D tensor copies of the
//     targets' source vectors (B, hi, mid and lo, 32-byte swizzled rows).
//   warp 5, one thread: MMA issue.  For chunk i it waits on `full`, issues the
//     chunk's tcgen05.mma into one of two accumulator buffers and commits them
//     to the stage's `empty` mbarrier; the last chunk of a unit is also
//     committed to `acc_full` of its buffer.
//   warps 0-3: epilogue.  For every unit they wait on `acc_full`, read their 32
//     TMEM lanes (rows) of the buffer, add the FP32 partial sums into the FP64
//     target sums with atomic adds (the slabs of a tile are spread over CTAs),
//     and arrive on `acc_empty`, which the MMA thread waits on before it reuses
//     the buffer.  The epilogue of one unit overlaps the MMAs of the next.
// Every wait is bounded; a time-out sets the abort flag and the status word,
// the other roles give up their waits, the copy and MMA threads wait for their
// work in flight (bounded by time only, whatever the abort flag says), and the
// CTA frees its tensor memory and returns; if that drain also runs out, bit 8
// of the status word is set and the tensor memory is kept.
template <int NT>
__global__ void __launch_bounds__(192, 1)
grid_gemm_kernel(GemmArgs a, const __grid_constant__ CUtensorMap tm_hi, const __grid_constant__ CUtensorMap tm_mid,
                 const __grid_constant__ CUtensorMap tm_lo) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int B_PART = NT * KC * 2;             // 4 or 2 KB
    constexpr int STAGE = NPART * A_PART + NPART * B_PART;
    constexpr int TZ = NT / 16;                     // tile depth along z
    constexpr uint32_t TCOLS = 4 * NT;              // 2 buffers x 2 row halves x NT columns
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
    const int n_units = NSLAB * n_tiles;
    const int G = gridDim.x;

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
                const int tile_g = u % n_tiles, c_begin = (u / n_tiles) * GW;
                const int c_end = (c_begin + GW < NCH_ALL) ? c_begin + GW : NCH_ALL;
                const int cls = tile_g / tiles, tile = tile_g % tiles;
                const int bx = (cls >> 2) & 1, by = (cls >> 1) & 1, bz = cls & 1;
                const int tx = tile / (tpd * tpz), ty = (tile / tpz) % tpd, tz = tile % tpz;
                int c1 = 0, c2 = 0, c3 = 0, c4 = 0;
                const unsigned char *abase = nullptr;
                for (int ci = c_begin; ci < c_end; ++ci, ++i) {
                    if (ci == c_begin || ci % NKC == 0) {
                        const int code = codes[cls * NU + ci / NKC];
                        const int sx = bx - (code / 49 - 3) + 3, sy = by - ((code / 7) % 7 - 3) + 3,
                                  sz = bz - (code % 7 - 3) + 3;
                        c1 = tz * TZ + (sz >> 1);
                        c2 = ty * 4 + (sy >> 1);
                        c3 = tx * 4 + (sx >> 1);
                        c4 = ((sx & 1) << 2) | ((sy & 1) << 1) | (sz & 1);
                        abase = reinterpret_cast<const unsigned char *>(a.top) + (long long)code * NKC * NPART * A_PART;
                    }
                    const int stg = (int)(i % NST), kc = (ci % NKC) * KC;
                    if (i >= NST && !wait_or_abort(smem_u32(empty + stg), (uint32_t)(((i / NST) - 1) & 1), abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    const uint32_t dst = smem_u32(sm + stg * STAGE), bar = smem_u32(full + stg);
                    const unsigned char *src = abase + (long long)(ci % NKC) * NPART * A_PART;
                    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" :: "r"(bar), "r"(STAGE) : "memory");
                    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                                 :: "r"(dst), "l"(src), "r"(NPART * A_PART), "r"(bar) : "memory");
                    const CUtensorMap *maps[NPART] = {&tm_hi, &tm_mid, &tm_lo};
#pragma unroll
                    for (int p = 0; p < NPART; ++p)
                        asm volatile("cp.async.bulk.tensor.5d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
                                     " [%0], [%1, {%2, %3, %4, %5, %6}], [%7];"
                                     :: "r"(dst + NPART * A_PART + p * B_PART), "l"(reinterpret_cast<uint64_t>(maps[p])),
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
            // D = FP32, A = B = BF16, both K-major, N = NT, M = 128
            const uint32_t idesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(NT >> 3) << 17) |
                                   ((uint32_t)(128 >> 4) << 24);
            // descriptors of stage 0; stage s adds s * STAGE to the address field.
            // A: no swizzle, core matrices 128 B apart along K, 8-row groups (KC / 8) * 128 B
            // apart; B: 32-byte swizzle, 8-row groups of 32-byte rows 256 B apart
            const uint32_t s0 = smem_u32(sm);
            const uint64_t dA = sdesc(s0, 128, (KC / 8) * 128, 0);
            const uint64_t dB = sdesc(s0 + NPART * A_PART, 16, 256, 6);
            long long i = 0, g = 0, last_mma = -1;
            bool ok = true;
            for (int u = blockIdx.x; u < n_units && ok; u += G, ++g) {
                const int c_begin = (u / n_tiles) * GW;
                const int c_end = (c_begin + GW < NCH_ALL) ? c_begin + GW : NCH_ALL;
                const int b = (int)(g & 1);
                if (g >= 2 && !wait_or_abort(smem_u32(acc_empty + b), (uint32_t)(((g >> 1) - 1) & 1), abort_flag)) {
                    fail();
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;");
                const uint32_t dcol = tmem + (uint32_t)b * 2 * NT;
                for (int ci = c_begin; ci < c_end; ++ci, ++i) {
                    const int stg = (int)(i % NST);
                    if (!wait_or_abort(smem_u32(full + stg), (uint32_t)((i / NST) & 1), abort_flag)) {
                        fail();
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;");
                    const uint64_t so = (uint64_t)((stg * STAGE) >> 4);
                    // six products of the parts, (hi, hi) first; the rows of half h
                    // start (128 / 8) * (KC / 8) * 128 bytes into each A part
                    constexpr int PA[6] = {0, 0, 1, 0, 2, 1}, PB[6] = {0, 1, 0, 2, 0, 1};
#pragma unroll
                    for (int h = 0; h < 2; ++h)
#pragma unroll
                        for (int t = 0; t < 6; ++t) {
                            const uint64_t ad = dA + so + ((PA[t] * A_PART + h * (A_PART / 2)) >> 4);
                            const uint64_t bd = dB + so + ((PB[t] * B_PART) >> 4);
                            const uint32_t d = dcol + h * NT;
                            const uint32_t acc = (ci == c_begin && t == 0) ? 0u : 1u;
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
            // drain: the MMAs issued have completed before the CTA frees its memory
            if (last_mma >= 0 && !wait_bounded(smem_u32(empty + last_mma % NST), (uint32_t)((last_mma / NST) & 1))) drain_fail();
        }
        __syncwarp();
    } else {
        long long g = 0;
        for (int u = blockIdx.x; u < n_units; u += G, ++g) {
            const int tile_g = u % n_tiles;
            const int b = (int)(g & 1);
            bool ok = true;
            if (lane == 0) ok = wait_or_abort(smem_u32(acc_full + b), (uint32_t)((g >> 1) & 1), abort_flag);
            ok = __shfl_sync(0xffffffffu, ok ? 1 : 0, 0) != 0;
            if (!ok) {
                if (lane == 0) fail();
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;");
            const int cls = tile_g / tiles, tile = tile_g % tiles;
            const int bx = (cls >> 2) & 1, by = (cls >> 1) & 1, bz = cls & 1;
            const int tx = tile / (tpd * tpz), ty = (tile / tpz) % tpd, tz = tile % tpz;
            for (int hc = 0; hc < 2 * (NT / 64); ++hc) {
                const int h = hc / (NT / 64), c0 = (hc % (NT / 64)) * 64;
                uint32_t v[64];
                const uint32_t ta = tmem + (uint32_t)b * 2 * NT + h * NT + c0 + ((uint32_t)(warp * 32) << 16);
                asm volatile("tcgen05.ld.sync.aligned.32x32b.x64.b32 "
                             "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,"
                             "%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47,%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%64];"
                             : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
                               "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
                               "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
                               "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31]),
                               "=r"(v[32]), "=r"(v[33]), "=r"(v[34]), "=r"(v[35]), "=r"(v[36]), "=r"(v[37]), "=r"(v[38]), "=r"(v[39]),
                               "=r"(v[40]), "=r"(v[41]), "=r"(v[42]), "=r"(v[43]), "=r"(v[44]), "=r"(v[45]), "=r"(v[46]), "=r"(v[47]),
                               "=r"(v[48]), "=r"(v[49]), "=r"(v[50]), "=r"(v[51]), "=r"(v[52]), "=r"(v[53]), "=r"(v[54]), "=r"(v[55]),
                               "=r"(v[56]), "=r"(v[57]), "=r"(v[58]), "=r"(v[59]), "=r"(v[60]), "=r"(v[61]), "=r"(v[62]), "=r"(v[63])
                             : "r"(ta));
                asm volatile("tcgen05.wait::ld.sync.aligned;");
                const int row = h * 128 + warp * 32 + lane;
#pragma unroll
                for (int jj = 0; jj < 64; ++jj) {
                    const int j = c0 + jj;
                    const int x = 2 * (tx * 4 + (j / (4 * TZ))) + bx;
                    const int y = 2 * (ty * 4 + ((j / TZ) & 3)) + by;
                    const int z = 2 * (tz * TZ + (j % TZ)) + bz;
                    atomicAdd(a.y + (((long long)x * ns + y) * ns + z) * KD + row, (double)__uint_as_float(v[jj]));
                }
            }
            asm volatile("tcgen05.fence::before_thread_sync;");
            __syncwarp();
            if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" :: "r"(smem_u32(acc_empty + b)) : "memory");
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
    unsigned short *top = nullptr;           // operators, pre-tiled hi|mid|lo BF16 chunks
    unsigned short *xhi = nullptr, *xmid = nullptr, *xlo = nullptr;   // packed sources (BF16 parts)
    double *y = nullptr;                     // FP64 accumulators
    double *c = nullptr;                     // sqrt((n-m)!(n+m)!) on the device
    std::vector<double> ch;                  // and on the host
    CUtensorMap tm_hi, tm_mid, tm_lo;        // 5-D maps of the source parts (tile boxes)
    int nt = 0;                              // targets per tile: 128 or 64
};

namespace {

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// map of the parity-split halo grid [8][nh/2][nh/2][nh/2][KD] (innermost last)
// with boxes of KC BF16 values x tz x 4 x 4 boxes x 1 parity class, 32-byte swizzle
bool encode_source_map(EncodeTiled enc, CUtensorMap *m, unsigned short *base, int nside, int tz) {
    const cuuint64_t nh2 = (cuuint64_t)(nside + 6) / 2;
    const cuuint64_t dims[5] = {(cuuint64_t)KD, nh2, nh2, nh2, 8};
    const cuuint64_t row = (cuuint64_t)KD * sizeof(unsigned short);
    const cuuint64_t strides[4] = {row, row * nh2, row * nh2 * nh2, row * nh2 * nh2 * nh2};
    const cuuint32_t box[5] = {(cuuint32_t)KC, (cuuint32_t)tz, 4, 4, 1};
    const cuuint32_t estr[5] = {1, 1, 1, 1, 1};
    return enc(m, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 5, base, dims, strides, box, estr,
               CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_32B,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

extern "C" {

sfmm_status sfmm_grid_create(sfmm_handle h, int P, int nside, sfmm_grid *out) {
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
    const size_t op_bytes = (size_t)NCODE * NKC * NPART * A_PART;
    const size_t x_bytes = sizeof(unsigned short) * (size_t)(nh * nh * nh) * KD;
    bool ok = cudaMalloc(&g->top, op_bytes) == cudaSuccess &&
              cudaMalloc(&g->xhi, x_bytes) == cudaSuccess &&
              cudaMalloc(&g->xmid, x_bytes) == cudaSuccess &&
              cudaMalloc(&g->xlo, x_bytes) == cudaSuccess &&
              cudaMalloc(&g->y, sizeof(double) * (size_t)nside * nside * nside * KD) == cudaSuccess &&
              cudaMalloc(&g->c, sizeof(double) * GP * (GP + 1) / 2) == cudaSuccess;
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
    double *dbasis = nullptr, *dL = nullptr, *dshift = nullptr;
    long long *dpin = nullptr, *dpout = nullptr;
    int *dcodes = nullptr;
    ok = cudaMalloc(&dbasis, sizeof(double) * basis.size()) == cudaSuccess &&
         cudaMalloc(&dL, sizeof(double) * count * S) == cudaSuccess &&
         cudaMalloc(&dshift, sizeof(double) * shift.size()) == cudaSuccess &&
         cudaMalloc(&dpin, sizeof(long long) * count) == cudaSuccess &&
         cudaMalloc(&dpout, sizeof(long long) * count) == cudaSuccess &&
         cudaMalloc(&dcodes, sizeof(int) * ncodes) == cudaSuccess;
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
        operator_kernel<<<1024, 256>>>(dL, dcodes, ncodes, g->c, g->top);
        if (cudaGetLastError() != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) st = SFMM_ERR_CUDA;
    }
    cudaFree(dbasis);
    cudaFree(dL);
    cudaFree(dshift);
    cudaFree(dpin);
    cudaFree(dpout);
    cudaFree(dcodes);
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
            !encode_source_map(reinterpret_cast<EncodeTiled>(fn), &g->tm_mid, g->xmid, nside, g->nt / 16) ||
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
    cudaFree(g->xmid);
    cudaFree(g->xlo);
    cudaFree(g->y);
    cudaFree(g->c);
    delete g;
    return SFMM_OK;
}

sfmm_status sfmm_grid_m2l(sfmm_grid g, double box_size, const void *M, void *L, int accumulate,
                          sfmm_stream stream) {
    if (g == nullptr || M == nullptr || L == nullptr || !(box_size > 0)) return SFMM_ERR_ARG;
    cudaStream_t s = reinterpret_cast<cudaStream_t>(stream);
    const int ns = g->nside;
    if (cudaMemsetAsync(g->y, 0, sizeof(double) * (size_t)ns * ns * ns * KD, s) != cudaSuccess)
        return SFMM_ERR_CUDA;
    Scales sp, su;
    for (int n = 0; n < GP; ++n) {
        const double hn = std::pow(box_size, n);
        for (int m = 0; m <= n; ++m) {
            sp.s[n * (n + 1) / 2 + m] = g->ch[n * (n + 1) / 2 + m] / (hn * box_size);
            su.s[n * (n + 1) / 2 + m] = g->ch[n * (n + 1) / 2 + m] / hn;
        }
    }
    pack_kernel<<<2048, 256, 0, s>>>(reinterpret_cast<const double *>(M), ns, sp, g->xhi, g->xmid, g->xlo);
    // tiles of 4 x 4 x (nt / 16) same-octant targets; one persistent CTA per SM
    // deals the (K slab, tile) units round-robin
    GemmArgs a{g->top, g->y, ns, g->h->d_status};
    const int ctas = g->h->sm_count > 0 ? g->h->sm_count : 1;
    if (g->nt == 128)
        grid_gemm_kernel<128><<<ctas, 192, smem_gemm<128>(), s>>>(a, g->tm_hi, g->tm_mid, g->tm_lo);
    else
        grid_gemm_kernel<64><<<ctas, 192, smem_gemm<64>(), s>>>(a, g->tm_hi, g->tm_mid, g->tm_lo);
    unpack_kernel<<<2048, 256, 0, s>>>(g->y, ns, su, reinterpret_cast<double *>(L), accumulate);
    return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
}

}  // extern "C"
