// Fully unrolled translation kernels for fixed orders p_in = p_out = P <= 12.
//
// Same algorithm as sfmm_kernels.cuh (Sec. 3.4 steps 1-4 with the
// orthonormal-basis tables), specialised at compile time so that
//   * the row buffers and the powers of e^{i alpha}, e^{i beta} live in
//     registers and every table entry is a __constant__ operand at a
//     compile-time offset (no address arithmetic, no table loads in L1);
//   * only the solid itself stays in shared memory (P(P+1) reals per thread,
//     interleaved across the warp with an odd stride, conflict-free for
//     per-lane and for cooperative accesses), which lets 8 warps share an SM
//     at P = 10 in FP64.  GB300's FP64 pipe issues one warp
//     instruction per 64 cycles per SM sub-partition with a 64-cycle dependent
//     latency, so two warps per sub-partition keep it busy while the other
//     waits on memory;
//   * the solid is transformed in place: input rows are rotated into the
//     rotated frame row by row, the z-axis translation replaces it column by
//     column, and the rotation back replaces it row by row;
//   * solids move between global and shared memory with coalesced
//     warp-cooperative copies.
// Lists run one group of G lanes per target (G = 32 for long M2L lists, 8 for
// the 8 children of an M2M parent): each member translates one source per
// round and the group sums its members' results in a fixed order.
#pragma once

#include <cuda_runtime.h>

#include <type_traits>

#include "sfmm_kernels.cuh"
#include "sfmm_tables.h"

namespace sfmm {
namespace unrolled {

constexpr int PC = 12;   // largest compiled order; the constant tables cover n < PC

// ---- packed table geometry (must match the host packing in sfmm_tables.cpp)
__host__ __device__ constexpr int cF(int n, int m) { return (n - ((n + m) & 1)) / 2 + 1; }
__host__ __device__ constexpr int l0G(int n, int m) { return ((n + m + 1) & 1) ? 1 : 2; }
__host__ __device__ constexpr int cG(int n, int m) {
    return (m == 0 || n < l0G(n, m)) ? 0 : (n - l0G(n, m)) / 2 + 1;
}
__host__ __device__ constexpr int FM(int n, int m) {
    int s = 0;
    for (int i = 0; i < m; ++i) s += cF(n, i);
    return s;
}
__host__ __device__ constexpr int GM(int n, int m) {
    int s = 0;
    for (int i = 1; i < m; ++i) s += cG(n, i);
    return s;
}
__host__ __device__ constexpr int FR(int n) {
    int s = 0;
    for (int i = 0; i < n; ++i) s += FM(i, i + 1);
    return s;
}
__host__ __device__ constexpr int GR(int n) {
    int s = 0;
    for (int i = 0; i < n; ++i) s += GM(i, i + 1);
    return s;
}
__host__ __device__ constexpr int QT(int P) {
    int s = 0;
    for (int m = 0; m < P; ++m) s += (P - m) * (P - m);
    return s;
}
__host__ __device__ constexpr int TB(int m) {       // start of z-translation block m
    int s = 0;
    for (int i = 0; i < m; ++i) s += (PC - i) * (PC - i);
    return s;
}

constexpr int OFF_F = 0;
constexpr int OFF_G = OFF_F + FR(PC);
constexpr int OFF_C = OFF_G + GR(PC);
constexpr int OFF_IC = OFF_C + PC * (PC + 1) / 2;
constexpr int OFF_T = OFF_IC + PC * (PC + 1) / 2;
// M2L only: the basis factors c folded into the swap next to them, F diag(c)
// and G diag(c) for the first input swap, diag(c) F and diag(c) G for the
// last output swap (same packing as F and G), which saves one multiply per
// coefficient on either side.
constexpr int OFF_FI = OFF_T + 3 * QT(PC);
constexpr int OFF_GI = OFF_FI + FR(PC);
constexpr int OFF_FO = OFF_GI + GR(PC);
constexpr int OFF_GO = OFF_FO + FR(PC);
constexpr int NTAB = OFF_GO + GR(PC);

// One copy per translation unit (each unit is its own module); filled by
// fill_constants() of that unit.
static __constant__ double c_tab64[NTAB];
static __constant__ float c_tab32[NTAB];

template <typename T>
__device__ __forceinline__ T ct(int i);
template <>
__device__ __forceinline__ double ct<double>(int i) { return c_tab64[i]; }
template <>
__device__ __forceinline__ float ct<float>(int i) { return c_tab32[i]; }

// Per-lane view of the warp's solid area: element e of lane j at e*33 + j.
// The odd stride keeps both access patterns conflict-free (a lane walking its
// own solid, and the warp copying one solid with consecutive elements per
// lane), and a lane's addresses are its base plus compile-time offsets.
constexpr int XSTRIDE = 33;
template <typename T>
struct Sw {
    T *wb;      // warp base
    int lane;
    __device__ __forceinline__ T &operator[](int e) const { return wb[e * XSTRIDE + lane]; }
    __device__ __forceinline__ T &at(int e, int j) const { return wb[e * XSTRIDE + j]; }
};

// One axis swap of row N (eq. Mswapxz / FGmappings) on register rows, with
// the packed F and G found at table offsets OF and OG.
template <typename T, int N, int OF = OFF_F, int OG = OFF_G>
__device__ __forceinline__ void swap_u(const T *ir, const T *ii, T *orr, T *oi) {
#pragma unroll
    for (int m = 0; m <= N; ++m) {
        T acc = T(0);
        int i = 0;
#pragma unroll
        for (int l = (N + m) & 1; l <= N; l += 2, ++i)
            acc = fma_t(ct<T>(OF + FR(N) + FM(N, m) + i), ir[l], acc);
        orr[m] = acc;
    }
    oi[0] = T(0);
#pragma unroll
    for (int m = 1; m <= N; ++m) {
        T acc = T(0);
        int i = 0;
#pragma unroll
        for (int l = l0G(N, m); l <= N; l += 2, ++i)
            acc = fma_t(ct<T>(OG + GR(N) + GM(N, m) + i), ii[l], acc);
        oi[m] = acc;
    }
}

// Rotation powers of one translation: e^{i m alpha} and e^{i m beta}, m < P.
template <typename T, int P>
struct Powers {
    T ar[P], ai[P], br[P], bi[P];
};

// Input row N: scale, orthonormal basis, rotate alpha, swap, rotate beta, swap.
template <typename T, int P, int OP, int N>
__device__ __forceinline__ void rows_in(Sw<T> X, const Powers<T, P> &pw, T s) {
    if constexpr (N < P) {
        constexpr int o = N * (N + 1);
        T ar[N + 1], ai[N + 1], br[N + 1], bi[N + 1];
        // M2L: the basis factor is folded into the first swap's tables.
        // m = 0: the rotation is the identity and Im C_n^0 is not read by the
        // swap (its G rows start at l >= 1).
#pragma unroll
        for (int m = 0; m <= N; ++m) {
            const T f = (OP == OP_M2L) ? s : s * ct<T>((OP == OP_L2L ? OFF_IC : OFF_C) + N * (N + 1) / 2 + m);
            if (m == 0) {
                ar[0] = X[o] * f;
                ai[0] = T(0);
                continue;
            }
            const T re = X[o + m] * f, im = X[o + N + 1 + m] * f;
            ar[m] = re * pw.ar[m] - im * pw.ai[m];
            ai[m] = fma_t(re, pw.ai[m], im * pw.ar[m]);
        }
        if constexpr (OP == OP_M2L) swap_u<T, N, OFF_FI, OFF_GI>(ar, ai, br, bi);
        else swap_u<T, N>(ar, ai, br, bi);
#pragma unroll
        for (int m = 1; m <= N; ++m) {
            const T re = br[m], im = bi[m];
            br[m] = re * pw.br[m] - im * pw.bi[m];
            bi[m] = fma_t(re, pw.bi[m], im * pw.br[m]);
        }
        swap_u<T, N>(br, bi, ar, ai);
#pragma unroll
        for (int m = 0; m <= N; ++m) { X[o + m] = ar[m]; X[o + N + 1 + m] = ai[m]; }
    }
}

// z-axis translation of column M in place (eq. zm2lkernels for M2L).
template <typename T, int P, int OP, int M>
__device__ __forceinline__ void columns_z(Sw<T> X) {
    if constexpr (M < P) {
        T xr[P - M], xi[P - M];
#pragma unroll
        for (int k = M; k < P; ++k) { xr[k - M] = X[k * (k + 1) + M]; xi[k - M] = X[k * (k + 1) + k + 1 + M]; }
#pragma unroll
        for (int n = M; n < P; ++n) {
            const int kb = (OP == OP_L2L) ? n : M;
            const int ke = (OP == OP_M2M) ? n + 1 : P;
            T accr = T(0), acci = T(0);
#pragma unroll
            for (int k = kb; k < ke; ++k) {
                const T t = ct<T>(OFF_T + OP * QT(PC) + TB(M) + (n - M) * (PC - M) + (k - M));
                accr = fma_t(t, xr[k - M], accr);
                if (M > 0) acci = fma_t(t, xi[k - M], acci);
            }
            X[n * (n + 1) + M] = accr;
            X[n * (n + 1) + n + 1 + M] = acci;
        }
    }
}

// Tensor memory as per-lane storage (the lists kernel's running sums): a
// warp reads and writes its own 32 lanes, `NC` consecutive 32-bit columns.
template <int NC>
__device__ __forceinline__ void tm_ld(uint32_t ta, uint32_t *r) {
    if constexpr (NC >= 32) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x32.b32 "
                     "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
                     "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                       "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
                       "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
                       "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
                     : "r"(ta));
        tm_ld<NC - 32>(ta + 32, r + 32);
    } else if constexpr (NC >= 16) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x16.b32 "
                     "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
                       "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                     : "r"(ta));
        tm_ld<NC - 16>(ta + 16, r + 16);
    } else if constexpr (NC >= 8) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7])
                     : "r"(ta));
        tm_ld<NC - 8>(ta + 8, r + 8);
    } else if constexpr (NC >= 4) {
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x4.b32 {%0,%1,%2,%3}, [%4];"
                     : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]) : "r"(ta));
        tm_ld<NC - 4>(ta + 4, r + 4);
    }
}
template <int NC>
__device__ __forceinline__ void tm_st(uint32_t ta, const uint32_t *r) {
    if constexpr (NC >= 32) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x32.b32 [%0], "
                     "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,"
                     "%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31,%32};"
                     :: "r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15]),
                        "r"(r[16]), "r"(r[17]), "r"(r[18]), "r"(r[19]), "r"(r[20]), "r"(r[21]), "r"(r[22]), "r"(r[23]),
                        "r"(r[24]), "r"(r[25]), "r"(r[26]), "r"(r[27]), "r"(r[28]), "r"(r[29]), "r"(r[30]), "r"(r[31])
                     : "memory");
        tm_st<NC - 32>(ta + 32, r + 32);
    } else if constexpr (NC >= 16) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
                     "{%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
                     :: "r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7]),
                        "r"(r[8]), "r"(r[9]), "r"(r[10]), "r"(r[11]), "r"(r[12]), "r"(r[13]), "r"(r[14]), "r"(r[15])
                     : "memory");
        tm_st<NC - 16>(ta + 16, r + 16);
    } else if constexpr (NC >= 8) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x8.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8};"
                     :: "r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]), "r"(r[4]), "r"(r[5]), "r"(r[6]), "r"(r[7])
                     : "memory");
        tm_st<NC - 8>(ta + 8, r + 8);
    } else if constexpr (NC >= 4) {
        asm volatile("tcgen05.st.sync.aligned.32x32b.x4.b32 [%0], {%1,%2,%3,%4};"
                     :: "r"(ta), "r"(r[0]), "r"(r[1]), "r"(r[2]), "r"(r[3]) : "memory");
        tm_st<NC - 4>(ta + 4, r + 4);
    }
}
__device__ __forceinline__ void tm_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ void tm_wait_st() { asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory"); }
__device__ __forceinline__ double tm_double(const uint32_t *w) { return __hiloint2double((int)w[1], (int)w[0]); }
__device__ __forceinline__ void tm_put(uint32_t *w, double v) {
    w[0] = (uint32_t)__double2loint(v);
    w[1] = (uint32_t)__double2hiint(v);
}

// Running sums of the lists kernel in tensor memory: `ta` addresses the lane's
// solid (element e at columns 2e, 2e+1); `first` = the target's first round.
struct TAcc {
    uint32_t ta;
    bool first;
};

// Output row N: swap, rotate -beta, swap, rotate -alpha, undo basis and scaling.
// ACC (FP64 M2L lists kernel): instead of storing the row into X, add it to the
// lane's running sum in tensor memory, folded into the last rotation's
// multiply-adds (the sums over a target's list are then added across lanes
// once per target, not once per round).
template <typename T, int P, int OP, int N, bool ACC = false>
__device__ __forceinline__ void rows_out(Sw<T> X, const Powers<T, P> &pw, T so, TAcc acc = TAcc{0, true}) {
    if constexpr (N < P) {
        constexpr int o = N * (N + 1);
        T ar[N + 1], ai[N + 1], br[N + 1], bi[N + 1];
#pragma unroll
        for (int m = 0; m <= N; ++m) { ar[m] = X[o + m]; ai[m] = X[o + N + 1 + m]; }
        swap_u<T, N>(ar, ai, br, bi);
#pragma unroll
        for (int m = 1; m <= N; ++m) {
            const T re = br[m], im = bi[m];
            br[m] = fma_t(re, pw.br[m], im * pw.bi[m]);
            bi[m] = im * pw.br[m] - re * pw.bi[m];
        }
        // M2L: the basis factor is folded into the last swap's tables.
        // m = 0: the rotation is the identity and the swap leaves Im = 0.
        if constexpr (OP == OP_M2L) swap_u<T, N, OFF_FO, OFF_GO>(br, bi, ar, ai);
        else swap_u<T, N>(br, bi, ar, ai);
        if constexpr (ACC) {
            static_assert(sizeof(T) == 8, "tensor-memory sums hold FP64 solids");
            constexpr int NC = 4 * (N + 1);                 // 2 (N+1) doubles
            uint32_t w[NC];
            if (!acc.first) {
                tm_ld<NC>(acc.ta + 2 * o, w);
                tm_wait_ld();
            } else {
#pragma unroll
                for (int c = 0; c < NC; ++c) w[c] = 0u;
            }
#pragma unroll
            for (int m = 0; m <= N; ++m) {
                const T f = (OP == OP_M2L) ? so : so * ct<T>((OP == OP_M2M ? OFF_IC : OFF_C) + N * (N + 1) / 2 + m);
                if (m == 0) {
                    tm_put(w, fma_t(ar[0], f, tm_double(w)));
                    continue;
                }
                const T re = ar[m] * f, im = ai[m] * f;
                tm_put(w + 2 * m, fma_t(re, pw.ar[m], fma_t(im, pw.ai[m], tm_double(w + 2 * m))));
                tm_put(w + 2 * (N + 1 + m), fma_t(im, pw.ar[m], fma_t(-re, pw.ai[m], tm_double(w + 2 * (N + 1 + m)))));
            }
            tm_st<NC>(acc.ta + 2 * o, w);
        } else {
#pragma unroll
            for (int m = 0; m <= N; ++m) {
                const T f = (OP == OP_M2L) ? so : so * ct<T>((OP == OP_M2M ? OFF_IC : OFF_C) + N * (N + 1) / 2 + m);
                if (m == 0) {
                    X[o] = ar[0] * f;
                    X[o + N + 1] = T(0);
                    continue;
                }
                const T re = ar[m] * f, im = ai[m] * f;
                X[o + m] = fma_t(re, pw.ar[m], im * pw.ai[m]);
                X[o + N + 1 + m] = im * pw.ar[m] - re * pw.ai[m];
            }
        }
    }
}

// The step bodies.  Unpaired: step K < P is input row K, P <= K < 2P column
// K - P, 2P <= K < 3P output row K - 2P.
template <typename T, int P, int OP, int K>
__device__ __forceinline__ void step_body(Sw<T> X, const Powers<T, P> &pw, T s, T so) {
    if constexpr (K < P) rows_in<T, P, OP, K>(X, pw, s);
    else if constexpr (K < 2 * P) columns_z<T, P, OP, K - P>(X);
    else if constexpr (K < 3 * P) rows_out<T, P, OP, K - 2 * P>(X, pw, so);
}

// Paired steps: rows n and P-1-n (columns M and P-1-M) share one step, so
// every step carries about the same work, (n+1)^2 + (P-n)^2 multiply-adds,
// and two independent sets of FMA chains for the scheduler to interleave.
// Only the M2L lists kernel pairs its steps: the batch kernels and the M2M and
// L2L lists kernels have no registers to spare for a second row and the row
// scales of every row (they would spill).
template <typename T, int P, int OP, int K, bool ACC>
__device__ __forceinline__ void step_body2(Sw<T> X, const Powers<T, P> &pw, const T *sin,
                                           const T *sout, TAcc acc) {
    constexpr int H = (P + 1) / 2;
    if constexpr (K < 3 * H) {
        constexpr int ph = K / H, i = K % H, j = P - 1 - i;
        if constexpr (ph == 0) {
            rows_in<T, P, OP, i>(X, pw, sin[i]);
            if constexpr (j != i) rows_in<T, P, OP, j>(X, pw, sin[j]);
        } else if constexpr (ph == 1) {
            columns_z<T, P, OP, i>(X);
            if constexpr (j != i) columns_z<T, P, OP, j>(X);
        } else {
            rows_out<T, P, OP, i, ACC>(X, pw, sout[i], acc);
            if constexpr (j != i) rows_out<T, P, OP, j, ACC>(X, pw, sout[j], acc);
        }
    }
}

// One row or column (or pair) per step, selected by one switch over the step
// number (a jump table; at most 3 PC = 36 steps), not by a chain of
// comparisons.  Cases past the last step are empty.
#define SFMM_STEP_CASES(C)                                                                     \
    C(0) C(1) C(2) C(3) C(4) C(5) C(6) C(7) C(8) C(9) C(10) C(11) C(12) C(13) C(14) C(15)       \
    C(16) C(17) C(18) C(19) C(20) C(21) C(22) C(23) C(24) C(25) C(26) C(27) C(28) C(29) C(30)   \
    C(31) C(32) C(33) C(34) C(35)
static_assert(3 * PC <= 36, "one switch case per step");

template <typename T, int P, int OP>
__device__ __forceinline__ void step_switch(int st, Sw<T> X, const Powers<T, P> &pw, T s, T so) {
    switch (st) {
#define SFMM_CASE(K) case K: step_body<T, P, OP, K>(X, pw, s, so); break;
        SFMM_STEP_CASES(SFMM_CASE)
#undef SFMM_CASE
        default: break;
    }
}

template <typename T, int P, int OP, bool ACC>
__device__ __forceinline__ void step_switch2(int st, Sw<T> X, const Powers<T, P> &pw, const T *sin,
                                             const T *sout, TAcc acc) {
    switch (st) {
#define SFMM_CASE(K) case K: step_body2<T, P, OP, K, ACC>(X, pw, sin, sout, acc); break;
        SFMM_STEP_CASES(SFMM_CASE)
#undef SFMM_CASE
        default: break;
    }
}

// One translation of order P by the calling thread, in place on its solid X.
// PAIRED (M2L in the lists kernel) runs two rows or columns per step.
template <typename T, int P, int OP, bool PAIRED = false, bool ACC = false>
__device__ __forceinline__ void translate_u(Sw<T> X, T x, T y, T z, TAcc acc = TAcc{0, true}) {
    // |r| and rho from one reciprocal square root each (cheaper on the FP64
    // pipe than a square root and a division).
    const T rho2 = x * x + y * y;
    const T R2 = rho2 + z * z;
    if (OP != OP_M2L && !(R2 > T(0))) return;           // zero shift: identity
    const T iR = rsqrt_t(R2);
    const T R = R2 * iR;
    T ca = T(1), sa = T(0), rho = T(0);                   // cos(alpha) = y/rho, sin(alpha) = x/rho
    if (rho2 > T(0)) { const T ir = rsqrt_t(rho2); ca = y * ir; sa = x * ir; rho = rho2 * ir; }
    const T cb = z * iR, sb = -rho * iR;                  // cos(beta) = z/|r|, sin(beta) = -rho/|r|
    Powers<T, P> pw;
    pw.ar[0] = T(1); pw.ai[0] = T(0); pw.br[0] = T(1); pw.bi[0] = T(0);
    if constexpr (P > 1) { pw.ar[1] = ca; pw.ai[1] = sa; pw.br[1] = cb; pw.bi[1] = sb; }
    if constexpr (sizeof(T) == 8) {
        // FP64: the three-term recurrence X_m = 2 cos(theta) X_{m-1} - X_{m-2} for
        // both components, one FMA each instead of a complex multiplication
        // (rounding below 1e-14 for m < 12)
        const T ta = T(2) * ca, tb = T(2) * cb;
#pragma unroll
        for (int m = 2; m < P; ++m) {
            pw.ar[m] = fma_t(ta, pw.ar[m - 1], -pw.ar[m - 2]);
            pw.ai[m] = fma_t(ta, pw.ai[m - 1], -pw.ai[m - 2]);
            pw.br[m] = fma_t(tb, pw.br[m - 1], -pw.br[m - 2]);
            pw.bi[m] = fma_t(tb, pw.bi[m - 1], -pw.bi[m - 2]);
        }
    } else {
#pragma unroll
        for (int m = 2; m < P; ++m) {
            pw.ar[m] = pw.ar[m - 1] * ca - pw.ai[m - 1] * sa;
            pw.ai[m] = fma_t(pw.ar[m - 1], sa, pw.ai[m - 1] * ca);
            pw.br[m] = pw.br[m - 1] * cb - pw.bi[m - 1] * sb;
            pw.bi[m] = fma_t(pw.br[m - 1], sb, pw.bi[m - 1] * cb);
        }
    }
    // Row scales: input |r|^{-(n+1)} (M2L), |r|^{-n} (M2M), |r|^{n} (L2L);
    // output |r|^{-n} (M2L, L2L), |r|^{n} (M2M).
    const T s0 = (OP == OP_M2L) ? iR : T(1);
    const T step_in = (OP == OP_L2L) ? R : iR;
    const T step_out = (OP == OP_M2M) ? R : iR;
    // One basic block per row or column step (or pair of them): a runtime loop
    // over the steps with a switch keeps the instruction scheduler from
    // interleaving more steps (which would keep more rows of tables and data
    // alive at once).
    if constexpr (PAIRED) {
        T sin[P], sout[P];
        sin[0] = s0;
        sout[0] = T(1);
#pragma unroll
        for (int n = 1; n < P; ++n) { sin[n] = sin[n - 1] * step_in; sout[n] = sout[n - 1] * step_out; }
#pragma unroll 1
        for (int st = 0; st < 3 * ((P + 1) / 2); ++st) step_switch2<T, P, OP, ACC>(st, X, pw, sin, sout, acc);
    } else {
        T s = s0, so = T(1);
#pragma unroll 1
        for (int st = 0; st < 3 * P; ++st) {
            step_switch<T, P, OP>(st, X, pw, s, so);
            if (st < P) s *= step_in;
            else if (st >= 2 * P) so *= step_out;
        }
    }
}

// Copy the 32 solids of the warp's lanes from global memory into the
// swizzled area (null pointer: zeros).  All 32 lanes take part.  Every element
// is an asynchronous global-to-shared copy (cp.async), so all of a round's
// loads are in flight together and the warp waits once, instead of once per
// batch of loads held in registers; the caller's __syncwarp() then publishes
// the copies to the whole warp.  A null solid is copied with a source size of
// zero, which fills the destination with zeros and reads nothing (the source
// address is then `dummy`, any readable global address), so the copies need
// no branch on the pointer.
template <typename T>
__device__ __forceinline__ void copy_async(T *dst, const T *src, uint32_t nbytes) {
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2, %3;"
                 :: "r"((uint32_t)__cvta_generic_to_shared(dst)), "l"(src), "n"((int)sizeof(T)), "r"(nbytes)
                 : "memory");
}
template <typename T, int S>
__device__ __forceinline__ void copy_solid(Sw<T> X, const T *mine, const void *dummy, int j) {
    const T *p = reinterpret_cast<const T *>(
        __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(mine), j));
    const uint32_t nb = p ? (uint32_t)sizeof(T) : 0u;
    const T *q = p ? p : reinterpret_cast<const T *>(dummy);
#pragma unroll
    for (int e0 = 0; e0 < S; e0 += 32) {
        const int e = e0 + X.lane;
        if (e < S) copy_async(&X.at(e, j), p ? q + e : q, nb);
    }
}
// The loop over the 32 solids is unrolled fully in FP64 and four times in FP32
// (measured: full unrolling gains 0.5 % on the FP64 octree pass and loses
// 1.5 % on the FP32 one, whose larger number of resident warps at different
// steps already strains the instruction cache).
template <typename T, int S>
__device__ __forceinline__ void load_solids(Sw<T> X, const T *mine, const void *dummy) {
    if constexpr (sizeof(T) == 8) {
#pragma unroll
        for (int j = 0; j < 32; ++j) copy_solid<T, S>(X, mine, dummy, j);
    } else {
#pragma unroll 4
        for (int j = 0; j < 32; ++j) copy_solid<T, S>(X, mine, dummy, j);
    }
    asm volatile("cp.async.commit_group;\ncp.async.wait_group 0;" ::: "memory");
}

template <typename T, int P, int OP>
__global__ void __launch_bounds__(256, 1) ubatch_kernel(const T *const *in, T *const *out,
                                                        const T *shift, long long count,
                                                        int accumulate, int *status) {
    constexpr int S = P * (P + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    Sw<T> X{reinterpret_cast<T *>(smem_raw) + (size_t)warp * S * XSTRIDE, lane};
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + warp; c * 32 < count; c += nw) {
        const long long i = c * 32 + lane;
        const bool valid = i < count;
        const T *src = valid ? in[i] : nullptr;
        T *dst = valid ? out[i] : nullptr;
        if (valid && (src == nullptr || dst == nullptr)) {
            atomicOr(status, STATUS_NULL_POINTER);
            src = nullptr;
            dst = nullptr;
        }
        load_solids<T, S>(X, src, in);
        __syncwarp();
        T x = T(0), y = T(0), z = T(1);
        if (src) { x = shift[3 * i]; y = shift[3 * i + 1]; z = shift[3 * i + 2]; }
        translate_u<T, P, OP>(X, x, y, z);
        __syncwarp();
#pragma unroll 4
        for (int j = 0; j < 32; ++j) {
            T *p = reinterpret_cast<T *>(
                __shfl_sync(0xffffffffu, reinterpret_cast<unsigned long long>(dst), j));
            if (p == nullptr) continue;
#pragma unroll
            for (int e0 = 0; e0 < S; e0 += 32) {
                const int e = e0 + lane;
                if (e < S) {
                    T v = X.at(e, j);
                    if (accumulate) v += p[e];
                    p[e] = v;
                }
            }
        }
        __syncwarp();
    }
}

// Target-major CSR lists, one group of G lanes per target, sources dealt to
// the members in rounds of G; each round's G results are summed per
// coefficient in member order and added to the group's running sum.
template <typename T, int P, int OP, int G>
__global__ void __launch_bounds__(256, 1) ulists_kernel(const T *const *src, const T *shift,
                                                        const long long *offsets, T *const *out,
                                                        long long n_targets, int accumulate,
                                                        int *status) {
    constexpr int S = P * (P + 1);
    constexpr int NG = 32 / G;                 // groups per warp
    constexpr int NA = (S + G - 1) / G;        // coefficients per member
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int q = lane / G, mem = lane % G;
    Sw<T> X{reinterpret_cast<T *>(smem_raw) + (size_t)warp * S * XSTRIDE, lane};
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    const long long w = (long long)blockIdx.x * (blockDim.x >> 5) + warp;
    for (long long k = 0; k * nw * NG < n_targets; ++k) {
        const long long c = deal_chunk(k, nw, w);
        if (c * NG >= n_targets) continue;
        const long long t = c * NG + q;
        long long j0 = 0, j1 = 0;
        if (t < n_targets) {
            j0 = offsets[t];
            j1 = offsets[t + 1];
            if (j1 < j0) { atomicOr(status, STATUS_BAD_OFFSETS); j1 = j0; }
        }
        int rounds = (int)((j1 - j0 + G - 1) / G);
#pragma unroll
        for (int d = 16; d > 0; d >>= 1) rounds = max(rounds, __shfl_xor_sync(0xffffffffu, rounds, d));
        T acc[NA];
#pragma unroll
        for (int a = 0; a < NA; ++a) acc[a] = T(0);
        for (int r = 0; r < rounds; ++r) {
            const long long j = j0 + (long long)r * G + mem;
            const T *s = (j < j1) ? src[j] : nullptr;
            if (j < j1 && s == nullptr) atomicOr(status, STATUS_NULL_POINTER);
            load_solids<T, S>(X, s, src);
            __syncwarp();
            T x = T(0), y = T(0), z = T(1);
            if (s) { x = shift[3 * j]; y = shift[3 * j + 1]; z = shift[3 * j + 2]; }
            translate_u<T, P, OP, OP == OP_M2L>(X, x, y, z);
            __syncwarp();
#pragma unroll
            for (int a = 0; a < NA; ++a) {
                const int e = mem + a * G;
                if (e < S) {
#pragma unroll
                    for (int i = 0; i < G; ++i) acc[a] += X.at(e, q * G + i);
                }
            }
            __syncwarp();
        }
        if (t < n_targets) {
            T *dst = out[t];
            if (dst == nullptr) {
                atomicOr(status, STATUS_NULL_POINTER);
            } else {
#pragma unroll
                for (int a = 0; a < NA; ++a) {
                    const int e = mem + a * G;
                    if (e < S) dst[e] = accumulate ? dst[e] + acc[a] : acc[a];
                }
            }
        }
    }
}

// The lane sums of a target, from tensor memory back into the lane's solid
// area X (rows N .. P-1), for the cross-lane reduction.
template <typename T, int P, int N>
__device__ __forceinline__ void flush_rows(Sw<T> X, uint32_t ta) {
    if constexpr (N < P) {
        constexpr int o = N * (N + 1), NC = 4 * (N + 1);
        uint32_t w[NC];
        tm_ld<NC>(ta + 2 * o, w);
        tm_wait_ld();
#pragma unroll
        for (int k = 0; k < 2 * (N + 1); ++k) X[o + k] = tm_double(w + 2 * k);
        flush_rows<T, P, N + 1>(X, ta);
    }
}

// The lanes' sums, flushed into X, back into tensor memory, with zeros for the
// lanes for which `zero` is set (all lanes take part: tcgen05.st is collective).
template <typename T, int P, int N>
__device__ __forceinline__ void refill_rows(Sw<T> X, uint32_t ta, bool zero) {
    if constexpr (N < P) {
        constexpr int o = N * (N + 1), NC = 4 * (N + 1);
        uint32_t w[NC];
#pragma unroll
        for (int k = 0; k < 2 * (N + 1); ++k) tm_put(w + 2 * k, zero ? T(0) : X[o + k]);
        tm_st<NC>(ta + 2 * o, w);
        refill_rows<T, P, N + 1>(X, ta, zero);
    }
}

// The flushed sums of lanes [lo, hi) added coefficient by coefficient in lane
// order, stored into dst (added to it when `add`); a null dst sets
// STATUS_NULL_POINTER.  Ends with a warp barrier (X is free afterwards).
template <typename T, int S>
__device__ __forceinline__ void sum_lanes(Sw<T> X, T *dst, int lo, int hi, bool add, int *status) {
    constexpr int NA = (S + 31) / 32;          // coefficients per lane
    if (dst == nullptr) {
        if (X.lane == 0) atomicOr(status, STATUS_NULL_POINTER);
    } else {
#pragma unroll
        for (int a = 0; a < NA; ++a) {
            const int e = X.lane + a * 32;
            if (e < S) {
                T v = T(0);
                for (int i = lo; i < hi; ++i) v += X.at(e, i);
                dst[e] = add ? dst[e] + v : v;
            }
        }
    }
    __syncwarp();
}

// Sources [a, b) of target t's list (an inverted range sets STATUS_BAD_OFFSETS
// and counts as empty).
__device__ __forceinline__ void list_range(const long long *offsets, long long t, int *status, int lane,
                                           long long &a, long long &b) {
    a = offsets[t];
    b = offsets[t + 1];
    if (b < a) {
        if (lane == 0) atomicOr(status, STATUS_BAD_OFFSETS);
        b = a;
    }
}

// FP64 M2L interaction lists, one target per warp at a time, with each lane's
// running sum of its translations kept in tensor memory (free in this kernel:
// 256 KB per SM, a warp's sums take 2 P(P+1) columns of its lane quadrant).
// The last rotation of every output row adds into the sum with its
// multiply-adds; a target's sums are added across lanes, in lane order, once
// the list is done.  A warp takes its targets in deal order and packs its
// rounds: when a list ends k < 32 sources into a round and the warp's next list
// has at least 32 sources, lanes k..31 of that round already translate the next
// list's first sources (no lane translates a missing source there).  Lanes
// k..31 then hand their sums of the ending list to the target before the round
// (summed, written, and reset to zero) and lanes 0..k-1 theirs after it, so a
// lane's sum only ever holds one target's translations.  A target's result is
// deterministic (it depends on the list and on the lengths of the lists dealt
// to the same warp).  `tcols` = tensor-memory columns of the CTA (a power of
// two >= ceil(warps / 4) * 2 P(P+1)); the launch checks that the CTAs resident
// on an SM fit in its 512 columns.
template <typename T, int P>
__global__ void __launch_bounds__(256, 1) ulists_acc_kernel(const T *const *src, const T *shift,
                                                            const long long *offsets, T *const *out,
                                                            long long n_targets, int accumulate,
                                                            int *status, int tcols) {
    constexpr int S = P * (P + 1);
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    Sw<T> X{reinterpret_cast<T *>(smem_raw) + (size_t)warp * S * XSTRIDE, lane};
    uint32_t *tslot = reinterpret_cast<uint32_t *>(smem_raw + (size_t)nwarps * S * XSTRIDE * sizeof(T));
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                     :: "r"((uint32_t)__cvta_generic_to_shared(tslot)), "r"(tcols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    const uint32_t ta = *tslot + ((uint32_t)((warp & 3) * 32) << 16) + (uint32_t)((warp >> 2) * 2 * S);
    const long long nw = (long long)gridDim.x * nwarps;
    const long long w = (long long)blockIdx.x * nwarps + warp;

    // (only k, t, pos, j1 and the flags live across a round's translation, and
    // the round has one call site of the translation)
    long long k = 0;
    long long t = deal_chunk(0, nw, w);
    long long j1 = 0, pos = 0;   // end of target t's list, its next source (lane 0's)
    if (t < n_targets) list_range(offsets, t, status, lane, pos, j1);
    bool fresh = true;           // the lanes' sums hold nothing yet
    bool partial = false;        // out[t] already holds part of the result
    while (t < n_targets) {
        const long long rem = j1 - pos;
        long long u0 = 0;        // start of the next list, if it is packed into this round
        bool pack = false;
        if (rem > 0 && rem < 32) {
            const long long tn = deal_chunk(k + 1, nw, w);
            if (tn < n_targets) {
                long long u1;
                list_range(offsets, tn, status, lane, u0, u1);
                pack = u1 - u0 >= 32;
            }
        }
        const int ka = pack ? (int)rem : 32;           // lanes 0..ka-1 on target t
        if (pack && !fresh) {                          // lanes ka..31 hand over their sums
            tm_wait_st();
            flush_rows<T, P, 0>(X, ta);
            __syncwarp();
            sum_lanes<T, S>(X, out[t], ka, 32, accumulate, status);
            refill_rows<T, P, 0>(X, ta, lane >= ka);
            __syncwarp();                              // X is read before the copies overwrite it
            partial = true;
        }
        if (rem > 0) {                                 // the round
            const long long j = lane < ka ? pos + lane : u0 + (lane - ka);
            const bool valid = lane >= ka || j < j1;
            const T *s = valid ? src[j] : nullptr;
            if (valid && s == nullptr) atomicOr(status, STATUS_NULL_POINTER);
            load_solids<T, S>(X, s, src);
            __syncwarp();
            T x = T(0), y = T(0), z = T(1);
            if (s) { x = shift[3 * j]; y = shift[3 * j + 1]; z = shift[3 * j + 2]; }
            if (!fresh) tm_wait_st();                  // earlier writes of the sums are done
            translate_u<T, P, OP_M2L, true, true>(X, x, y, z, TAcc{ta, fresh});
            __syncwarp();
            fresh = false;
            pos += ka;
        }
        if (pos >= j1) {                               // target t is done (or its list empty)
            if (!fresh) {
                tm_wait_st();
                flush_rows<T, P, 0>(X, ta);
                __syncwarp();
            }
            sum_lanes<T, S>(X, out[t], 0, fresh ? 0 : ka, partial || accumulate, status);
            ++k;
            t = deal_chunk(k, nw, w);
            if (t < n_targets) list_range(offsets, t, status, lane, pos, j1);
            if (pack) {                                // lanes 0..ka-1 restart at zero; the
                refill_rows<T, P, 0>(X, ta, lane < ka);   // next list's first 32-ka are done
                __syncwarp();
                pos += 32 - ka;
            } else {
                fresh = true;
            }
            partial = false;
        }
    }
    tm_wait_st();
    asm volatile("tcgen05.fence::before_thread_sync;");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;");
    if (warp == 0) asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" :: "r"(*tslot), "r"(tcols));
}

}  // namespace unrolled
}  // namespace sfmm
