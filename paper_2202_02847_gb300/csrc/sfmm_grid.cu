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
// 189 offsets, so one CTA computes y for 64 targets of one octant as a GEMM
// with K = 189 * 256 on the 5th-generation tensor cores:
//   * T_u and x are split into TF32 hi + lo parts and multiplied as
//     hi*hi + hi*lo + lo*hi (3xTF32, about 21 significant bits) with FP32
//     accumulation in tensor memory (two 128-row halves x 64 columns);
//   * every 8 offsets the accumulator is read out (tcgen05.ld) and added into
//     an FP64 accumulator in global memory (the target's sum is FP64);
//   * operand chunks (16 of K) are staged in shared memory in the canonical
//     K-major layout in a four-stage pipeline: the T_u chunk is stored
//     pre-tiled in global memory and arrives by one TMA bulk copy, the
//     targets' source vectors are gathered by 16-byte cp.async copies;
//   * a CTA holds 128 targets (64 on grids below 16^3), so every T_u chunk
//     read from L2 serves 128 target columns.
// T_u are built once per grid object with the FP64 rotation-based M2L on the
// 256 basis vectors of every offset.  Every mbarrier wait is bounded: on
// time-out the kernel records SFMM_GRID_TIMEOUT in the status word, stops
// issuing work, frees its tensor memory and returns.
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
constexpr int KC = 16;             // K chunk staged in shared memory
constexpr int NST = 4;             // pipeline stages
constexpr int NKC = KD / KC;       // chunks per offset
constexpr int A_PART = KD * KC * 4;   // one operand part (hi or lo) of an A chunk: 16 KB
constexpr int FLUSH = 8;           // offsets accumulated in FP32 before an FP64 flush
constexpr int NCODE = 343;         // offset codes ((dx+3)*7 + dy+3)*7 + dz+3
constexpr int STATUS_GRID_TIMEOUT = 4;

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

// shared-memory matrix descriptor: K-major, no swizzle, core matrices of
// 8 rows x 16 bytes; lbo = byte step between core matrices along K, sbo = along M/N
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFF);
    d |= (uint64_t)((lbo >> 4) & 0x3FFF) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFF) << 32;
    d |= (uint64_t)1 << 46;
    return d;
}

// byte offset of (row r, k) inside a [rows x KC] K-major tile
__device__ __forceinline__ int koff(int r, int k) {
    return ((r >> 3) * (KC / 4) + (k >> 2)) * 128 + (r & 7) * 16 + (k & 3) * 4;
}

__device__ __forceinline__ float tf32_round(float x) {
    uint32_t r;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
    return __uint_as_float(r);
}

__device__ __forceinline__ bool bar_wait(uint32_t bar, uint32_t phase) {
    uint32_t done = 0;
    for (int it = 0; it < (1 << 22) && !done; ++it)
        asm volatile("{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
                     "selp.u32 %0, 1, 0, p;\n}" : "=r"(done) : "r"(bar), "r"(phase));
    return done != 0;
}

// ----------------------------------------------------------------- kernels

// per-coefficient scale factors (n(n+1)/2 + m): c/h^{n+1} for packing, c/h^n for unpacking
struct Scales {
    double s[GP * (GP + 1) / 2];
};

// x = M c / h^{k+1} in the reduced layout on the halo grid, split into TF32 hi, lo.
__global__ void pack_kernel(const double *M, int nside, Scales sc, float *xhi, float *xlo) {
    const int nh = nside + 6;
    const long long total = (long long)nh * nh * nh * KD;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
         i += (long long)gridDim.x * blockDim.x) {
        const long long b = i / KD;
        const int e = (int)(i % KD);
        const int hx = (int)(b / (nh * nh)) - 3, hy = (int)((b / nh) % nh) - 3, hz = (int)(b % nh) - 3;
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
        const float hi = tf32_round(v);
        xhi[i] = hi;
        xlo[i] = v - hi;
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
// order GP), converted to y = L / c in the reduced layout and split hi/lo.
__global__ void operator_kernel(const double *L, const int *codes, int ncodes, const double *c,
                                float *thi) {
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
        const float v = (float)(s[n * (n + 1) + (im ? n + 1 + m : m)] / c[n * (n + 1) / 2 + m]);
        const float hi = tf32_round(v);
        // pre-tiled: [code][chunk][hi|lo][K-major core-matrix tile of 256 rows x KC]
        const int ch = j / KC, kk = j % KC;
        unsigned char *base = reinterpret_cast<unsigned char *>(thi) +
                              ((long long)codes[k] * NKC + ch) * 2 * A_PART;
        *reinterpret_cast<float *>(base + koff(ep, kk)) = hi;
        *reinterpret_cast<float *>(base + A_PART + koff(ep, kk)) = v - hi;
    }
}

struct GemmArgs {
    const float *thi;           // pre-tiled operators, [NCODE][NKC][hi|lo][A_PART bytes]
    const float *xhi, *xlo;     // [(ns+6)^3][KD]
    double *y;                  // [ns^3][KD]
    int nside;
    int *status;
};

__device__ __forceinline__ void cp16(void *smem_dst, const void *gsrc) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" :: "r"(smem_u32(smem_dst)), "l"(gsrc));
}

// dynamic shared memory: NST stages of A (hi, lo) and B (hi, lo), then 1 KB
// for the mbarriers, the TMEM slot, the abort flag and the 189 offset codes
template <int NT>
constexpr int smem_gemm() { return NST * (2 * A_PART + 2 * NT * KC * 4) + 1024; }

// One CTA: NT targets of one child octant (a 4x4x(NT/16) block of the
// octant's sub-grid), all 256 output rows, all 189 offsets of the octant, as
// a pipeline of NST stages of K = 16:
//   A (the pre-tiled T_u chunk, hi and lo, 32 KB) arrives by one TMA bulk copy
//   completing on the stage's `full` mbarrier;
//   B (the targets' source vectors, hi and lo) is gathered with 16-byte
//   cp.async copies;
//   thread 0 issues the tcgen05.mma of a stage and commits them to the stage's
//   `mmad` mbarrier, which gates the reuse of the stage and the FP64 flushes.
template <int NT>
__global__ void __launch_bounds__(128, 1) grid_gemm_kernel(GemmArgs a) {
    extern __shared__ __align__(1024) unsigned char sm[];
    constexpr int B_PART = NT * KC * 4;             // 8 or 4 KB
    constexpr int STAGE = 2 * A_PART + 2 * B_PART;
    constexpr int TZ = NT / 16;                     // tile depth along z
    constexpr int NU = 189;                         // offsets of an octant
    constexpr int NCH = NU * NKC;                   // chunks of a CTA
    // after the stages: 2 x NST mbarriers, the TMEM slot, the abort flag, the offset codes
    uint64_t *full = reinterpret_cast<uint64_t *>(sm + NST * STAGE);
    uint64_t *mmad = full + NST;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(mmad + NST);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    int *codes = reinterpret_cast<int *>(tslot + 4);
    const int tid = threadIdx.x, warp = tid >> 5;
    const int ns = a.nside, half_ns = ns / 2, tpd = half_ns / 4, tpz = half_ns / TZ;
    const int tiles = tpd * tpd * tpz;
    const int cls = blockIdx.x / tiles, tile = blockIdx.x % tiles;
    const int bx = (cls >> 2) & 1, by = (cls >> 1) & 1, bz = cls & 1;
    const int tx = tile / (tpd * tpz), ty = (tile / tpz) % tpd, tz = tile % tpz;
    const int nh = ns + 6;

    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" :: "r"(smem_u32(tslot)), "r"(2 * NT));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    if (tid == 0) {
        for (int i = 0; i < NST; ++i) {
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(full + i)));
            asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" :: "r"(smem_u32(mmad + i)));
        }
        asm volatile("fence.mbarrier_init.release.cluster;");
        *abort_flag = 0;
        // the octant's offsets u = target - source: u_i in [-3 + b_i, 2 + b_i], max|u_i| >= 2
        int nu = 0;
        for (int dx = -3 + bx; dx <= 2 + bx; ++dx)
            for (int dy = -3 + by; dy <= 2 + by; ++dy)
                for (int dz = -3 + bz; dz <= 2 + bz; ++dz) {
                    const int ax = dx < 0 ? -dx : dx, ay = dy < 0 ? -dy : dy, az = dz < 0 ? -dz : dz;
                    if ((ax > ay ? (ax > az ? ax : az) : (ay > az ? ay : az)) >= 2)
                        codes[nu++] = ((dx + 3) * 7 + (dy + 3)) * 7 + (dz + 3);
                }
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t tmem = *tslot;
    const uint32_t idesc = (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(NT >> 3) << 17) |
                           ((uint32_t)(128 >> 4) << 24);

    auto target_of = [&](int j, int *x, int *y, int *z) {
        *x = 2 * (tx * 4 + (j / (4 * TZ))) + bx;
        *y = 2 * (ty * 4 + ((j / TZ) & 3)) + by;
        *z = 2 * (tz * TZ + (j % TZ)) + bz;
    };
    // A of chunk ci: one bulk copy of the pre-tiled hi|lo chunk (thread 0 only)
    auto load_a = [&](int ci) {
        const int stg = ci % NST;
        const unsigned char *src = reinterpret_cast<const unsigned char *>(a.thi) +
                                   ((long long)codes[ci / NKC] * NKC + ci % NKC) * 2 * A_PART;
        asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;"
                     :: "r"(smem_u32(full + stg)), "r"(2 * A_PART) : "memory");
        asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                     :: "r"(smem_u32(sm + stg * STAGE)), "l"(src), "r"(2 * A_PART), "r"(smem_u32(full + stg))
                     : "memory");
    };
    // B of chunk ci: the targets' source vectors, 16-byte copies by every thread
    auto load_b = [&](int ci) {
        unsigned char *st = sm + (ci % NST) * STAGE + 2 * A_PART;
        const int code = codes[ci / NKC], kc = (ci % NKC) * KC;
        const int dx = code / 49 - 3, dy = (code / 7) % 7 - 3, dz = code % 7 - 3;
#pragma unroll
        for (int i = tid; i < NT * (KC / 4); i += 128) {
            const int j = i / (KC / 4), k4 = (i % (KC / 4)) * 4;
            int x, y, z;
            target_of(j, &x, &y, &z);
            const long long sb = ((long long)(x - dx + 3) * nh + (y - dy + 3)) * nh + (z - dz + 3);
            cp16(st + koff(j, k4), a.xhi + sb * KD + kc + k4);
            cp16(st + B_PART + koff(j, k4), a.xlo + sb * KD + kc + k4);
        }
    };
    // A failed wait sets the abort flag; every thread reads it only after a
    // __syncthreads that follows the write, so all threads leave the loop at
    // the same iteration.
    auto fail = [&]() {
        *abort_flag = 1;
        atomicOr(a.status, STATUS_GRID_TIMEOUT);
    };

    int a_issued = 0, a_consumed = 0, last_mma = -1, first_in_group = 1;   // thread 0's bookkeeping
    for (int c = 0; c < NST - 1; ++c) {
        if (tid == 0) { load_a(c); a_issued = c + 1; }
        load_b(c);
        asm volatile("cp.async.commit_group;");
    }
    for (int ci = 0; ci < NCH; ++ci) {
        const int stg = ci % NST;
        const uint32_t par = (uint32_t)((ci / NST) & 1);
        // this thread's B copies of chunk ci are done (later chunks stay in flight)
        asm volatile("cp.async.wait_group %0;" :: "n"(NST - 2));
        asm volatile("fence.proxy.async.shared::cta;");
        asm volatile("tcgen05.fence::before_thread_sync;");
        __syncthreads();
        asm volatile("tcgen05.fence::after_thread_sync;");
        if (*abort_flag) break;
        if (tid == 0) {
            if (!bar_wait(smem_u32(full + stg), par)) {
                fail();
            } else {
                a_consumed = ci + 1;
                const uint32_t sa = smem_u32(sm + stg * STAGE);
                for (int h = 0; h < 2; ++h)
                    for (int s = 0; s < KC / 8; ++s) {
                        const uint64_t ahi = sdesc(sa + h * (A_PART / 2) + s * 256, 128, (KC / 4) * 128);
                        const uint64_t alo = sdesc(sa + A_PART + h * (A_PART / 2) + s * 256, 128, (KC / 4) * 128);
                        const uint64_t bhi = sdesc(sa + 2 * A_PART + s * 256, 128, (KC / 4) * 128);
                        const uint64_t blo = sdesc(sa + 2 * A_PART + B_PART + s * 256, 128, (KC / 4) * 128);
                        const uint32_t d = tmem + h * NT;
                        const uint32_t acc0 = (first_in_group && s == 0) ? 0u : 1u;
                        asm volatile("{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                                     "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}"
                                     :: "r"(d), "l"(ahi), "l"(bhi), "r"(idesc), "r"(acc0));
                        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                                     :: "r"(d), "l"(ahi), "l"(blo), "r"(idesc));
                        asm volatile("tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, 1;"
                                     :: "r"(d), "l"(alo), "l"(bhi), "r"(idesc));
                    }
                asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                             :: "r"(smem_u32(mmad + stg)));
                last_mma = ci;
                first_in_group = 0;
            }
        }
        // refill the stage of chunk ci - 1 with chunk ci + NST - 1 once the MMAs of ci - 1 are done
        const int nc = ci + NST - 1;
        if (nc < NCH) {
            if (ci == 0 || bar_wait(smem_u32(mmad + (ci - 1) % NST), (uint32_t)(((ci - 1) / NST) & 1))) {
                if (tid == 0) { load_a(nc); a_issued = nc + 1; }
                load_b(nc);
            } else {
                fail();
            }
        }
        asm volatile("cp.async.commit_group;");
        if ((ci + 1) % (NKC * FLUSH) == 0 || ci + 1 == NCH) {
            // FP32 partial sums of the last FLUSH offsets -> FP64 accumulators
            if (tid == 0 && !*abort_flag && !bar_wait(smem_u32(mmad + stg), par)) fail();
            __syncthreads();
            if (*abort_flag) break;
            asm volatile("tcgen05.fence::after_thread_sync;");
            // rows 32 * warp + lane of both halves, NT target columns each
            for (int hc = 0; hc < 2 * (NT / 64); ++hc) {
                const int h = hc / (NT / 64), c0 = (hc % (NT / 64)) * 64;
                uint32_t v[64];
                const uint32_t ta = tmem + h * NT + c0 + ((uint32_t)(warp * 32) << 16);
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
                const int row = h * 128 + warp * 32 + (tid & 31);
#pragma unroll
                for (int jj = 0; jj < 64; ++jj) {
                    int x, y, z;
                    target_of(c0 + jj, &x, &y, &z);
                    double *dst = a.y + (((long long)x * ns + y) * ns + z) * KD + row;
                    *dst += (double)__uint_as_float(v[jj]);
                }
            }
            first_in_group = 1;
        }
    }
    // drain: no copy or MMA of this CTA may outlive it
    asm volatile("cp.async.wait_group 0;");
    if (tid == 0) {
        if (last_mma >= 0 && !bar_wait(smem_u32(mmad + last_mma % NST), (uint32_t)((last_mma / NST) & 1))) fail();
        for (int c = a_consumed; c < a_issued; ++c)
            if (!bar_wait(smem_u32(full + c % NST), (uint32_t)((c / NST) & 1))) fail();
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(tmem), "r"(2 * NT));
}

}  // namespace

struct sfmm_grid_ctx {
    sfmm_handle h = nullptr;
    int P = GP, nside = 0;
    float *thi = nullptr;                    // operators, pre-tiled hi|lo chunks
    float *xhi = nullptr, *xlo = nullptr;    // packed sources on the halo grid
    double *y = nullptr;                     // FP64 accumulators
    double *c = nullptr;                     // sqrt((n-m)!(n+m)!) on the device
    std::vector<double> ch;                  // and on the host
};

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
    const size_t op_bytes = (size_t)NCODE * NKC * 2 * A_PART;
    bool ok = cudaMalloc(&g->thi, op_bytes) == cudaSuccess &&
              cudaMalloc(&g->xhi, sizeof(float) * (size_t)(nh * nh * nh) * KD) == cudaSuccess &&
              cudaMalloc(&g->xlo, sizeof(float) * (size_t)(nh * nh * nh) * KD) == cudaSuccess &&
              cudaMalloc(&g->y, sizeof(double) * (size_t)nside * nside * nside * KD) == cudaSuccess &&
              cudaMalloc(&g->c, sizeof(double) * GP * (GP + 1) / 2) == cudaSuccess;
    if (!ok) { sfmm_grid_destroy(g); return SFMM_ERR_NOMEM; }
    cudaMemset(g->thi, 0, op_bytes);
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
        operator_kernel<<<1024, 256>>>(dL, dcodes, ncodes, g->c, g->thi);
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
    cudaFree(g->thi);
    cudaFree(g->xhi);
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
    pack_kernel<<<2048, 256, 0, s>>>(reinterpret_cast<const double *>(M), ns, sp, g->xhi, g->xlo);
    GemmArgs a{g->thi, g->xhi, g->xlo, g->y, ns, g->h->d_status};
    if (ns % 16 == 0) {      // 128 targets per CTA: 4 x 4 x 8 blocks of an octant
        const int tiles = (ns / 8) * (ns / 8) * (ns / 16);
        grid_gemm_kernel<128><<<8 * tiles, 128, smem_gemm<128>(), s>>>(a);
    } else {                 // 64 targets per CTA: 4 x 4 x 4 blocks
        const int tiles = (ns / 8) * (ns / 8) * (ns / 8);
        grid_gemm_kernel<64><<<8 * tiles, 128, smem_gemm<64>(), s>>>(a);
    }
    unpack_kernel<<<2048, 256, 0, s>>>(g->y, ns, su, reinterpret_cast<double *>(L), accumulate);
    return cudaGetLastError() == cudaSuccess ? SFMM_OK : SFMM_ERR_CUDA;
}

}  // extern "C"
