// Device kernels of the rotation-based translations (Sec. 2.4, Sec. 3.4).
//
// Design: one GPU thread computes one translation from start to finish, the
// way the paper lays nu solids side by side in SIMD lanes (Sec. 3.2); a warp
// therefore runs 32 translations in lock-step with identical control flow
// and no idle lanes.  Each thread keeps its rotated solid, two row buffers and
// the powers of e^{i alpha}, e^{i beta} in shared memory, interleaved across
// the 32 lanes of its warp (element e of lane j at word e*32 + j), so every
// shared access of a warp is conflict-free.  The shared tables (swap
// matrices, z-translation matrices, basis factors) are read from global
// memory through L1 with warp-uniform addresses (one broadcast per warp).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include "sfmm_tables.h"

namespace sfmm {

template <typename T>
struct DevTables {
    const T *F, *G;          // packed reduced swap matrices (see sfmm_tables.h)
    const int *Frow, *Grow;  // row starts, Pmax+1 each
    const T *c, *ic;         // sqrt((n-m)!(n+m)!) and its inverse, n(n+1)/2+m
                             // (FP32: times 2^-n and 2^n, see row_pow2)
    const T *Tz[3];          // z-axis translation blocks per op
    // The same matrices transposed for the warp-cooperative kernels
    // (sfmm_wide.cuh), whose lanes each take one output and read entry i of
    // their rows together: FT row n holds entry i of the packed F row m at
    // i (n+1) + m (n/2+1 entries deep, zero past a row's end), GT row n entry
    // i of the G row m >= 1 at i n + m - 1 ((n+1)/2 deep), TzT block m entry
    // (n-m, k-m) of Tz at (k-m) (Pmax-m) + n-m.
    const T *FT, *GT;
    const int *FTrow, *GTrow;
    const T *TzT[3];
    // FP64 only (null in FP32, whose range the products leave above order ~25):
    // M2L's swaps with the basis factors folded in, packed like F and G:
    // F diag(c), G diag(c) for the first input swap and diag(c) F, diag(c) G for
    // the last output swap (one multiplication per coefficient fewer per side)
    const T *FI, *GI, *FO, *GO;
    int Pmax;
};

// The basis factors leave the FP32 range at order 30 (c_29^29 = sqrt(58!)
// ~ 1.5e39 > FLT_MAX, 1/c_29^29 is subnormal), although their products with
// the row scales |r|^{-(n+1)}, |r|^n stay in range for unit-sized boxes.  FP32
// tables therefore hold c_n^m 2^-n and 2^n / c_n^m, and a row's factor is
// formed as (scale * table) * 2^{+-n}: the same value as scale * c with one
// more exact multiplication.  FP64 tables are unscaled (row_pow2 = 1, not
// issued).
template <typename T>
__device__ __forceinline__ T row_pow2(int e) { return T(1); }
template <>
__device__ __forceinline__ float row_pow2<float>(int e) {
    return __int_as_float((127 + e) << 23);            // 2^e, |e| <= 63
}
template <typename T>
__device__ __forceinline__ T basis_factor(T scale, T table, T p2) {
    if constexpr (sizeof(T) == 4) return (scale * table) * p2;
    else return scale * table;
}

// status bits written by kernels (atomicOr into the handle's status word)
enum { STATUS_NULL_POINTER = 1, STATUS_BAD_OFFSETS = 2 };

constexpr int WARP = 32;

// per-thread working set in elements for (p_in, p_out): the rotated solid
// (x_elems) and two complex row buffers, plus for orders up to PTAB_MAX the
// powers of e^{i alpha} and e^{i beta} (row_elems).  Above PTAB_MAX the
// powers are regenerated per row: the tables would cost the shared memory of
// half the resident warps, the regeneration ~4 FLOP per element and row.
constexpr int PTAB_MAX = 12;
__host__ __device__ inline bool power_tables(int p_in, int p_out) {
    return (p_in > p_out ? p_in : p_out) <= PTAB_MAX;
}
__host__ __device__ inline int x_elems(int p_in) { return p_in * (p_in + 1); }
__host__ __device__ inline int row_elems(int p_in, int p_out) {
    return (power_tables(p_in, p_out) ? 8 : 4) * (p_in > p_out ? p_in : p_out);
}

__device__ __forceinline__ double fma_t(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float fma_t(float a, float b, float c) { return fmaf(a, b, c); }
__device__ __forceinline__ double sqrt_t(double a) { return sqrt(a); }
__device__ __forceinline__ float sqrt_t(float a) { return sqrtf(a); }
__device__ __forceinline__ double rsqrt_t(double a) { return rsqrt(a); }
__device__ __forceinline__ float rsqrt_t(float a) { return rsqrtf(a); }

template <typename T>
__device__ __forceinline__ T ldt(const T *p) { return __ldg(p); }

// Chunk of persistent warp w (of nw) in round k.  Rounds alternate direction,
// so that with chunks ordered by decreasing cost (lists sorted by length) the
// warps' totals, and the SMs' (whose warps are consecutive), stay within one
// chunk of each other; round-robin in one direction gives the first warps the
// largest chunk of every round.
__device__ __forceinline__ long long deal_chunk(long long k, long long nw, long long w) {
    return k * nw + ((k & 1) ? nw - 1 - w : w);
}

// Lane-strided view: element e lives at base[e * WARP].
template <typename T>
struct LaneArr {
    T *p;
    __device__ __forceinline__ T &operator[](int e) const { return p[e * WARP]; }
    __device__ __forceinline__ LaneArr operator+(int e) const { return LaneArr{p + e * WARP}; }
};

// G outputs of one parity class of a swap: out[m + 2j] = sum_l t_j[i] in[l],
// l = l0, l0+2, ..., <= n, where t_j = t + j*tstep is the packed table row of
// output m + 2j.  Outputs of one class share the same l (chequerboard,
// Fig. 2), so each input is loaded once for G independent FMA chains.
template <typename T, int G>
__device__ __forceinline__ void swap_group(const T *__restrict__ t, int tstep, int l0, int n,
                                           LaneArr<T> in, LaneArr<T> out, int m) {
    T acc[G];
#pragma unroll
    for (int j = 0; j < G; ++j) acc[j] = T(0);
    int i = 0;
#pragma unroll 2
    for (int l = l0; l <= n; l += 2, ++i) {
        const T x = in[l];
#pragma unroll
        for (int j = 0; j < G; ++j) acc[j] = fma_t(ldt(t + j * tstep + i), x, acc[j]);
    }
#pragma unroll
    for (int j = 0; j < G; ++j) out[m + 2 * j] = acc[j];
}

// All outputs m = m_first, m_first+2, ... < mmax of one parity class, in
// groups of 4, 2, 1.  off0 = packed offset of output m_first; consecutive
// outputs of the class are tstep entries apart.
template <typename T>
__device__ __forceinline__ void swap_class(const T *__restrict__ t, int off0, int tstep, int l0,
                                           int n, LaneArr<T> in, LaneArr<T> out, int m_first,
                                           int mmax) {
    int m = m_first, off = off0;
    for (; m + 6 < mmax; m += 8, off += 4 * tstep) swap_group<T, 4>(t + off, tstep, l0, n, in, out, m);
    if (m + 2 < mmax) { swap_group<T, 2>(t + off, tstep, l0, n, in, out, m); m += 4; off += 2 * tstep; }
    if (m < mmax) swap_group<T, 1>(t + off, tstep, l0, n, in, out, m);
}

// One axis swap of row n (eq. Mswapxz / FGmappings):
//   Re out_m = sum_l F_n[m][l] Re in_l,   Im out_m = sum_l G_n[m][l] Im in_l
// for m < mmax, skipping the chequerboard zeros (Fig. 2).  F_n[m] has its
// non-zeros at l = (n+m)&1, +2, ...; G_n[m] (m >= 1) at l = 1 or 2, +2, ...
// with n+m+l odd.  The packed tables hold the rows one after the other, so
// rows of one parity class are a constant stride apart.
// Fb, Gb: packed tables to use instead of F and G (same layout), e.g. FI, GI.
template <typename T>
__device__ __forceinline__ void swap_row(const DevTables<T> &tb, int n, LaneArr<T> in_re,
                                         LaneArr<T> in_im, LaneArr<T> out_re,
                                         LaneArr<T> out_im, int mmax, const T *Fb = nullptr,
                                         const T *Gb = nullptr) {
    const T *__restrict__ F = (Fb ? Fb : tb.F) + __ldg(tb.Frow + n);
    const int fe = n / 2 + 1;                  // entries of a row with n+m even (l0 = 0)
    const int fo = (n + 1) / 2;                // entries of a row with n+m odd (l0 = 1)
    const int f0 = (n & 1) ? fo : fe;          // row m = 0
    swap_class(F, 0, fe + fo, n & 1, n, in_re, out_re, 0, mmax);
    swap_class(F, f0, fe + fo, (n + 1) & 1, n, in_re, out_re, 1, mmax);
    const T *__restrict__ G = (Gb ? Gb : tb.G) + __ldg(tb.Grow + n);
    const int ge = (n + 1) / 2;                // rows with n+m even: l0 = 1
    const int go = n / 2;                      // rows with n+m odd:  l0 = 2
    const int g1 = ((n + 1) & 1) ? go : ge;    // row m = 1
    out_im[0] = T(0);
    swap_class(G, 0, ge + go, ((n + 1) & 1) ? 2 : 1, n, in_im, out_im, 1, mmax);
    swap_class(G, g1, ge + go, (n & 1) ? 2 : 1, n, in_im, out_im, 2, mmax);
}

// z-axis translation of output row n, columns m0 .. m0+G-1 (eq. zm2lkernels
// for M2L): out_m = sum_k Tz_m[n][k] X[k][m] for the op's range of k, real
// and imaginary parts (which do not couple) as 2G independent FMA chains.
template <typename T, int OP, int G>
__device__ __forceinline__ void ztrans_block(const T *__restrict__ Tz, int Pm, int n, int m0,
                                             int p_in, LaneArr<T> Xre, LaneArr<T> Xim,
                                             LaneArr<T> Are, LaneArr<T> Aim) {
    const T *Tr[G];
#pragma unroll
    for (int j = 0; j < G; ++j) {
        const int m = m0 + j;
        Tr[j] = Tz + ztrans_block_offset(Pm, m) + (long long)(n - m) * (Pm - m) - m;
    }
    // k ranges: M2L [m, p_in), M2M [m, min(n+1, p_in)), L2L [n, p_in)
    const int k1 = (OP == OP_M2M) ? ((n + 1 < p_in) ? n + 1 : p_in) : p_in;
    const int kfull = (OP == OP_L2L) ? n : m0 + G - 1;     // every column active from here
    int k = (OP == OP_L2L) ? n : m0;
    T ar[G], ai[G];
#pragma unroll
    for (int j = 0; j < G; ++j) { ar[j] = T(0); ai[j] = T(0); }
    const bool has_im0 = m0 > 0;                            // Im of column 0 is zero
    // head: columns start one after the other (M2L, M2M)
    for (; k < kfull && k < k1; ++k) {
        const int xi = k * (k + 1) / 2 + m0;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            if (m0 + j <= k) {
                const T t = ldt(Tr[j] + k);
                ar[j] = fma_t(t, Xre[xi + j], ar[j]);
                if (j > 0 || has_im0) ai[j] = fma_t(t, Xim[xi + j], ai[j]);
            }
        }
    }
#pragma unroll 2
    for (; k < k1; ++k) {
        const int xi = k * (k + 1) / 2 + m0;
#pragma unroll
        for (int j = 0; j < G; ++j) {
            const T t = ldt(Tr[j] + k);
            ar[j] = fma_t(t, Xre[xi + j], ar[j]);
            if (j > 0 || has_im0) ai[j] = fma_t(t, Xim[xi + j], ai[j]);
        }
    }
#pragma unroll
    for (int j = 0; j < G; ++j) { Are[m0 + j] = ar[j]; Aim[m0 + j] = ai[j]; }
}

// Powers e^{i m theta}, m = 0, 1, 2, ... in that order, from two interleaved
// recurrences (even and odd m, each stepping by e^{2 i theta}), so that
// consecutive powers do not wait on each other and need no storage.
template <typename T>
struct PowSeq {
    T er, ei, od_r, od_i, c2, s2;
    __device__ __forceinline__ PowSeq(T c, T s)
        : er(T(1)), ei(T(0)), od_r(c), od_i(s), c2(c * c - s * s), s2(T(2) * c * s) {}
    __device__ __forceinline__ void next(int m, T &pr, T &pi) {
        if (m & 1) {
            pr = od_r; pi = od_i;
            const T r = od_r * c2 - od_i * s2, i = fma_t(od_r, s2, od_i * c2);
            od_r = r; od_i = i;
        } else {
            pr = er; pi = ei;
            const T r = er * c2 - ei * s2, i = fma_t(er, s2, ei * c2);
            er = r; ei = i;
        }
    }
};

// In FP64 each chain steps by the three-term (Chebyshev) recurrence
// X_{m+2} = 2 cos(2 theta) X_m - X_{m-2}, one FMA per component instead of a
// complex multiplication (rounding error below 2e-13 up to m = 63, against
// 2e-14 for the multiplications; in FP32 it would reach 2e-5 by m = 28, so FP32
// keeps the multiplications).
template <>
struct PowSeq<double> {
    double er, ei, qer, qei, od_r, od_i, qor, qoi, t2;
    __device__ __forceinline__ PowSeq(double c, double s) {
        const double c2 = c * c - s * s, s2 = 2.0 * c * s;
        er = 1.0; ei = 0.0; qer = c2; qei = -s2;          // X_0, X_{-2}
        od_r = c; od_i = s; qor = c; qoi = -s;             // X_1, X_{-1}
        t2 = 2.0 * c2;
    }
    __device__ __forceinline__ void next(int m, double &pr, double &pi) {
        if (m & 1) {
            pr = od_r; pi = od_i;
            const double r = fma(t2, od_r, -qor), i = fma(t2, od_i, -qoi);
            qor = od_r; qoi = od_i; od_r = r; od_i = i;
        } else {
            pr = er; pi = ei;
            const double r = fma(t2, er, -qer), i = fma(t2, ei, -qei);
            qer = er; qei = ei; er = r; ei = i;
        }
    }
};

// Output sink: overwrite or add one coefficient of the result (a solid in
// memory, or a lane's interleaved slot in the scratch).
// Loads of solids: CG = true reads through L2 only (ld.global.cg), for data
// that other SMs write during the same launch (the phased pass kernel);
// otherwise ordinary loads.
template <bool CG, typename T>
__device__ __forceinline__ T ldd(const T *p) {
    if constexpr (CG) return __ldcg(p);
    else return *p;
}

template <bool CG, typename T>
__device__ __forceinline__ void put(T *dst, T v, bool add) {
    if (add) v += ldd<CG>(dst);
    *dst = v;
}
template <bool CG, typename T>
__device__ __forceinline__ void put(LaneArr<T> dst, T v, bool add) {
    if (add) v += dst[0];
    dst[0] = v;
}

// One translation computed by the calling thread (Sec. 3.4 steps 1-4, with
// the z-axis translation of the op).  `buf` is this lane's shared memory of
// lane_elems(p_in, p_out) elements.  add = accumulate into dst.
template <typename T, int OP, bool PT, bool CG, typename D>
__device__ void translate_impl(const DevTables<T> &tb, int p_in, int p_out,
                               const T *__restrict__ src, const T *__restrict__ shift,
                               D dst, bool add, LaneArr<T> X, LaneArr<T> buf) {
    const int P = p_in > p_out ? p_in : p_out;
    constexpr bool FOLD = OP == OP_M2L && sizeof(T) == sizeof(double);
    // lane memory map: X = rotated solid (rows k < p_in, p_in(p_in+1) elements),
    // buf = two complex row buffers (4P), then for P <= PTAB_MAX the powers of
    // e^{i alpha} and e^{i beta} (4P); above, the powers are regenerated per
    // row (PowSeq)
    const int xhalf = p_in * (p_in + 1) / 2;
    LaneArr<T> Xre = X, Xim = X + xhalf;
    LaneArr<T> Are = buf, Aim = Are + P;                     // row buffer A
    LaneArr<T> Bre = Aim + P, Bim = Bre + P;                 // row buffer B
    constexpr bool ptab = PT;                                // == power_tables(p_in, p_out)
    LaneArr<T> PAre = Bim + P, PAim = PAre + P;              // e^{i m alpha} (ptab)
    LaneArr<T> PBre = PAim + P, PBim = PBre + P;             // e^{i m beta} (ptab)

    // --- step 1: shift geometry without trigonometric functions (Sec. 3.4)
    const T x = shift[0], y = shift[1], z = shift[2];
    const T rho2 = x * x + y * y;
    const T R = sqrt_t(rho2 + z * z);
    if (!(R > T(0))) {
        if (OP != OP_M2L) {
            // zero shift: M2M / L2L are the identity (truncated or zero-padded)
            for (int n = 0; n < p_out; ++n)
                for (int j = 0; j < 2 * (n + 1); ++j)
                    put<CG>(dst + n * (n + 1) + j, n < p_in ? ldd<CG>(src + n * (n + 1) + j) : T(0), add);
            return;
        }
    }
    const T rho = sqrt_t(rho2);
    T ca = T(1), sa = T(0);                     // cos(alpha) = y/rho, sin(alpha) = x/rho
    if (rho > T(0)) { const T ir = T(1) / rho; ca = y * ir; sa = x * ir; }
    const T iR = T(1) / R;
    const T cb = z * iR, sb = -rho * iR;        // cos(beta) = z/|r|, sin(beta) = -rho/|r|
    if constexpr (ptab) {
        T ar = T(1), ai = T(0), br = T(1), bi = T(0);
        for (int m = 0; m < P; ++m) {
            PAre[m] = ar; PAim[m] = ai; PBre[m] = br; PBim[m] = bi;
            const T ar2 = ar * ca - ai * sa, ai2 = fma_t(ar, sa, ai * ca);
            const T br2 = br * cb - bi * sb, bi2 = fma_t(br, sb, bi * cb);
            ar = ar2; ai = ai2; br = br2; bi = bi2;
        }
    }

    // --- step 2: rows of the input -> rotated frame, shift along +z, |r| = 1
    // input scale (eq. scaling): M2L |r|^{-(n+1)}, M2M |r|^{-n}, L2L |r|^{n}
    const T step_in = (OP == OP_L2L) ? R : iR;
    T s = (OP == OP_M2L) ? iR : T(1);
    const int krows = (OP == OP_M2M) ? (p_in < p_out ? p_in : p_out) : p_in;
    for (int n = 0; n < krows; ++n) {
        const T *row = src + n * (n + 1);
        const T *cf = ((OP == OP_L2L) ? tb.ic : tb.c) + n * (n + 1) / 2;
        const T p2 = row_pow2<T>((OP == OP_L2L) ? -n : n);
        // (b) scale, change to the orthonormal basis, rotate by alpha
        // (FP64 M2L: the basis factor is folded into the first swap's tables)
        PowSeq<T> pa(ca, sa);
        for (int m = 0; m <= n; ++m) {
            const T f = FOLD ? s : basis_factor(s, ldt(cf + m), p2);
            const T re = ldd<CG>(row + m) * f, im = ldd<CG>(row + n + 1 + m) * f;
            T pr, pi;
            if constexpr (ptab) { pr = PAre[m]; pi = PAim[m]; } else { pa.next(m, pr, pi); }
            Are[m] = re * pr - im * pi;
            Aim[m] = fma_t(re, pi, im * pr);
        }
        // (c) swap x and z
        swap_row(tb, n, Are, Aim, Bre, Bim, n + 1, FOLD ? tb.FI : nullptr, FOLD ? tb.GI : nullptr);
        // (d) rotate by beta
        PowSeq<T> pb(cb, sb);
        T pr, pi;
        pb.next(0, pr, pi);
        for (int m = 1; m <= n; ++m) {
            if constexpr (ptab) { pr = PBre[m]; pi = PBim[m]; } else { pb.next(m, pr, pi); }
            const T re = Bre[m], im = Bim[m];
            Bre[m] = re * pr - im * pi;
            Bim[m] = fma_t(re, pi, im * pr);
        }
        // (e) swap again, straight into the column-ordered rotated solid
        const int mm = (n + 1 < p_out) ? n + 1 : p_out;
        const int xo = n * (n + 1) / 2;
        swap_row(tb, n, Bre, Bim, Xre + xo, Xim + xo, mm);
        s *= step_in;
    }

    // --- steps 3-4: per output row, z-axis translation then rotate back
    // output scale: M2L |r|^{-n}, M2M |r|^{n}, L2L |r|^{-n}
    const T step_out = (OP == OP_M2M) ? R : iR;
    T so = T(1);
    const T *__restrict__ Tz = tb.Tz[OP];
    const int Pm = tb.Pmax;
    for (int n = 0; n < p_out; ++n) {
        int m0 = 0;
        for (; m0 + 3 <= n; m0 += 4) ztrans_block<T, OP, 4>(Tz, Pm, n, m0, p_in, Xre, Xim, Are, Aim);
        if (m0 + 1 <= n) { ztrans_block<T, OP, 2>(Tz, Pm, n, m0, p_in, Xre, Xim, Are, Aim); m0 += 2; }
        if (m0 <= n) ztrans_block<T, OP, 1>(Tz, Pm, n, m0, p_in, Xre, Xim, Are, Aim);
        // swap, rotate by -beta, swap
        swap_row(tb, n, Are, Aim, Bre, Bim, n + 1);
        {
            PowSeq<T> pb(cb, sb);
            T pr, pi;
            pb.next(0, pr, pi);
            for (int m = 1; m <= n; ++m) {
                if constexpr (ptab) { pr = PBre[m]; pi = PBim[m]; } else { pb.next(m, pr, pi); }
                const T re = Bre[m], im = Bim[m];
                Bre[m] = fma_t(re, pr, im * pi);
                Bim[m] = im * pr - re * pi;
            }
        }
        swap_row(tb, n, Bre, Bim, Are, Aim, n + 1, FOLD ? tb.FO : nullptr, FOLD ? tb.GO : nullptr);
        // rotate by -alpha, undo the scaling and the basis change (FP64 M2L:
        // folded into the last swap's tables), store
        const T *cf = ((OP == OP_M2M) ? tb.ic : tb.c) + n * (n + 1) / 2;
        const T p2 = row_pow2<T>((OP == OP_M2M) ? -n : n);
        D orow = dst + n * (n + 1);
        PowSeq<T> pa(ca, sa);
        for (int m = 0; m <= n; ++m) {
            const T f = FOLD ? so : basis_factor(so, ldt(cf + m), p2);
            const T re = Are[m] * f, im = Aim[m] * f;
            T pr, pi;
            if constexpr (ptab) { pr = PAre[m]; pi = PAim[m]; } else { pa.next(m, pr, pi); }
            put<CG>(orow + m, fma_t(re, pr, im * pi), add);
            put<CG>(orow + n + 1 + m, im * pr - re * pi, add);
        }
        so *= step_out;
    }
}

// Dispatch on the storage of the rotation powers (compile-time in the loops).
// TABLES = false always regenerates them (one code path: the multi-class
// kernel, which serves all three ops, keeps its compile time down that way;
// its row buffers are still sized by row_elems).
template <typename T, int OP, bool TABLES = true, bool CG = false, typename D>
__device__ __forceinline__ void translate_one(const DevTables<T> &tb, int p_in, int p_out,
                                              const T *__restrict__ src, const T *__restrict__ shift,
                                              D dst, bool add, LaneArr<T> X, LaneArr<T> buf) {
    if (TABLES && power_tables(p_in, p_out))
        translate_impl<T, OP, TABLES, CG>(tb, p_in, p_out, src, shift, dst, add, X, buf);
    else
        translate_impl<T, OP, false, CG>(tb, p_in, p_out, src, shift, dst, add, X, buf);
}

// ---------------------------------------------------------------- kernels

// Lane storage.  XG = false: everything in shared memory.  XG = true (orders
// whose rotated solid does not fit): the rotated solid lives in a global
// scratch area with one slot per resident warp, interleaved like shared
// memory, and the kernel runs as a persistent grid of exactly `nslots` warps.
template <typename T, bool XG>
struct LaneStore {
    LaneArr<T> X, buf;
    __device__ __forceinline__ LaneStore(T *smem, T *scratch, int p_in, int p_out) {
        const int lane = threadIdx.x & (WARP - 1), warp = threadIdx.x / WARP;
        const int ex = x_elems(p_in), er = row_elems(p_in, p_out);
        if (XG) {
            const long long slot = (long long)blockIdx.x * (blockDim.x / WARP) + warp;
            X = LaneArr<T>{scratch + slot * ex * WARP + lane};
            buf = LaneArr<T>{smem + (size_t)warp * er * WARP + lane};
        } else {
            X = LaneArr<T>{smem + (size_t)warp * (ex + er) * WARP + lane};
            buf = X + ex;
        }
    }
};

// Work distribution: the units (translations or targets) are cut into chunks
// of 32 (or 32 / G targets), one per warp, dealt over a persistent grid sized
// to the resident capacity: in order for translations (equal costs), in
// alternating directions (deal_chunk) for lists, which callers sort by
// decreasing length.
template <typename T, int OP, bool XG>
__global__ void __launch_bounds__(256, 1) batch_kernel(DevTables<T> tb, const T *const *in,
                                                    T *const *out, const T *shift, int p_in,
                                                    int p_out, long long count, int accumulate,
                                                    T *scratch, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LaneStore<T, XG> ls(reinterpret_cast<T *>(smem_raw), scratch, p_in, p_out);
    const int lane = threadIdx.x & (WARP - 1);
    const long long nw = (long long)gridDim.x * (blockDim.x / WARP);
    for (long long c = (long long)blockIdx.x * (blockDim.x / WARP) + threadIdx.x / WARP;
         c * WARP < count; c += nw) {
        const long long i = c * WARP + lane;
        if (i >= count) continue;
        const T *src = in[i];
        T *dst = out[i];
        if (src == nullptr || dst == nullptr) { atomicOr(status, STATUS_NULL_POINTER); continue; }
        translate_one<T, OP>(tb, p_in, p_out, src, shift + 3 * i, dst, accumulate != 0, ls.X, ls.buf);
    }
}

template <typename T, int OP, bool XG>
__global__ void __launch_bounds__(256, 1) lists_kernel(DevTables<T> tb, const T *const *src,
                                                    const T *shift, const long long *offsets,
                                                    T *const *out, int p_in, int p_out,
                                                    long long n_targets, int accumulate,
                                                    T *scratch, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    LaneStore<T, XG> ls(reinterpret_cast<T *>(smem_raw), scratch, p_in, p_out);
    const int lane = threadIdx.x & (WARP - 1);
    const long long nw = (long long)gridDim.x * (blockDim.x / WARP);
    const long long w = (long long)blockIdx.x * (blockDim.x / WARP) + threadIdx.x / WARP;
    for (long long k = 0; k * nw * WARP < n_targets; ++k) {
        const long long c = deal_chunk(k, nw, w);
        const long long t = c * WARP + lane;
        if (t >= n_targets) continue;
        T *dst = out[t];
        const long long j0 = offsets[t], j1 = offsets[t + 1];
        if (dst == nullptr) { atomicOr(status, STATUS_NULL_POINTER); continue; }
        if (j1 < j0) { atomicOr(status, STATUS_BAD_OFFSETS); continue; }
        bool add = accumulate != 0;
        if (j0 == j1 && !add)
            for (int e = 0; e < p_out * (p_out + 1); ++e) dst[e] = T(0);
        for (long long j = j0; j < j1; ++j) {
            const T *s = src[j];
            if (s == nullptr) { atomicOr(status, STATUS_NULL_POINTER); continue; }
            translate_one<T, OP>(tb, p_in, p_out, s, shift + 3 * j, dst, add, ls.X, ls.buf);
            add = true;
        }
    }
}

// Lists with G lanes per target (G = 2, 4, 8, 16 or 32; 32/G targets per
// warp), so that a long list is spread over the lanes of its group and a
// target's cost is ceil(length / G) translations.  Lane `mem` of a group
// takes the sources j0 + mem, j0 + mem + G, ... and accumulates their
// translations in its own output slot Y (interleaved in the scratch); then
// member mem adds the coefficients mem, mem + G, ... of the group's slots, in
// lane order, into the target.  The order of the additions is fixed, so the
// result does not depend on timing.
template <typename T, int OP, bool TABLES = true, bool CG = false>
__device__ void group_chunk(const DevTables<T> &tb, int p_in, int p_out, int G, long long t,
                            long long t_end, const T *const *src, const T *shift,
                            const long long *offsets, T *const *out, int accumulate,
                            LaneArr<T> X, LaneArr<T> Y, LaneArr<T> buf, int *status) {
    const int lane = threadIdx.x & (WARP - 1), mem = lane % G, q0 = lane - mem;
    long long j0 = 0, j1 = 0;
    T *dst = nullptr;
    if (t < t_end) {
        j0 = offsets[t];
        j1 = offsets[t + 1];
        dst = out[t];
        if (j1 < j0) {
            if (mem == 0) atomicOr(status, STATUS_BAD_OFFSETS);
            j1 = j0;
        }
        if (dst == nullptr && mem == 0) atomicOr(status, STATUS_NULL_POINTER);
    }
    bool any = false;
    for (long long j = j0 + mem; j < j1; j += G) {
        const T *s = src[j];
        if (s == nullptr) { atomicOr(status, STATUS_NULL_POINTER); continue; }
        translate_one<T, OP, TABLES, CG>(tb, p_in, p_out, s, shift + 3 * j, Y, any, X, buf);
        any = true;
    }
    const unsigned has = __ballot_sync(0xffffffffu, any);
    __syncwarp();
    if (dst != nullptr) {
        const int ey = p_out * (p_out + 1);
        const LaneArr<T> Y0{Y.p - lane};               // lane 0's slot; lane i at Y0.p + i
        for (int e = mem; e < ey; e += G) {
            T acc = T(0);
            for (int i = 0; i < G; ++i)
                if ((has >> (q0 + i)) & 1u) acc += Y0.p[(size_t)e * WARP + q0 + i];
            dst[e] = accumulate ? ldd<CG>(dst + e) + acc : acc;
        }
    }
    __syncwarp();                                       // slots are reused by the next chunk
}

// Single-class lists, G lanes per target, rotated solid and output slot in the
// global scratch (slot of x_elems(p_in) + p_out (p_out + 1) elements per lane).
template <typename T, int OP>
__global__ void __launch_bounds__(256, 1) glists_kernel(DevTables<T> tb, const T *const *src,
                                                     const T *shift, const long long *offsets,
                                                     T *const *out, int p_in, int p_out,
                                                     long long n_targets, int accumulate, int G,
                                                     T *scratch, unsigned long long *work, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & (WARP - 1), warp = threadIdx.x / WARP;
    const long long slot = (long long)blockIdx.x * (blockDim.x / WARP) + warp;
    const int ex = x_elems(p_in), ey = p_out * (p_out + 1);
    LaneArr<T> X{scratch + slot * (long long)(ex + ey) * WARP + lane};
    LaneArr<T> Y = X + ex;
    LaneArr<T> buf{reinterpret_cast<T *>(smem_raw) + (size_t)warp * row_elems(p_in, p_out) * WARP + lane};
    const int ng = WARP / G;
    for (;;) {
        // chunks from a counter (zeroed before the launch), in the callers'
        // order of decreasing list length
        long long c = 0;
        if (lane == 0) c = (long long)atomicAdd(work, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c * ng >= n_targets) break;
        group_chunk<T, OP>(tb, p_in, p_out, G, c * ng + lane / G, n_targets, src, shift, offsets, out,
                           accumulate, X, Y, buf, status);
    }
}

// Several classes of lists in one persistent launch.  The class table travels
// as a kernel parameter; chunk c belongs to the class k with
// chunk_begin[k] <= c < chunk_begin[k+1] and holds 32 / g targets of it, g its
// lanes per target (1: one lane walks a whole list; else as group_chunk).
// The rotated solid (and for g > 1 the lane's output slot) lives in the global
// scratch (slot of x_slot elements per lane); shared memory holds the row
// buffers and powers for the largest order of the launch.
constexpr int MAX_CLASSES = 256;
struct MultiClass {
    int op, p_in, p_out, g;
    long long tb, te, chunk_begin;
};
struct MultiParams {
    unsigned long long *work;    // zeroed before the launch; warps take chunks from it
    int n;
    int x_slot;                  // scratch elements per lane
    int row_slot;                // shared elements per lane
    long long total_chunks;
    MultiClass c[MAX_CLASSES];
};

template <typename T>
__global__ void __launch_bounds__(256, 1) multi_lists_kernel(DevTables<T> tb, MultiParams mp,
                                                             const T *const *src, const T *shift,
                                                             const long long *offsets,
                                                             T *const *out, int accumulate,
                                                             T *scratch, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & (WARP - 1), warp = threadIdx.x / WARP;
    const long long slot = (long long)blockIdx.x * (blockDim.x / WARP) + warp;
    LaneArr<T> X{scratch + slot * mp.x_slot * WARP + lane};
    LaneArr<T> buf{reinterpret_cast<T *>(smem_raw) + (size_t)warp * mp.row_slot * WARP + lane};
    for (;;) {
        // dynamic deal: classes come ordered by decreasing chunk cost, so the
        // longest chunks start first and the short ones fill the tail
        long long c = 0;
        if (lane == 0) c = (long long)atomicAdd(mp.work, 1ull);
        c = __shfl_sync(0xffffffffu, c, 0);
        if (c >= mp.total_chunks) break;
        int k = 0, hi = mp.n - 1;                     // last class with chunk_begin <= c
        while (k < hi) {
            const int mid = (k + hi + 1) >> 1;
            if (mp.c[mid].chunk_begin <= c) k = mid; else hi = mid - 1;
        }
        const MultiClass cl = mp.c[k];
        if (cl.g > 1) {
            const long long tg = cl.tb + (c - cl.chunk_begin) * (WARP / cl.g) + lane / cl.g;
            const LaneArr<T> Y = X + x_elems(cl.p_in);
            if (cl.op == OP_M2M)
                group_chunk<T, OP_M2M, false>(tb, cl.p_in, cl.p_out, cl.g, tg, cl.te, src, shift, offsets, out, accumulate, X, Y, buf, status);
            else if (cl.op == OP_M2L)
                group_chunk<T, OP_M2L, false>(tb, cl.p_in, cl.p_out, cl.g, tg, cl.te, src, shift, offsets, out, accumulate, X, Y, buf, status);
            else
                group_chunk<T, OP_L2L, false>(tb, cl.p_in, cl.p_out, cl.g, tg, cl.te, src, shift, offsets, out, accumulate, X, Y, buf, status);
            continue;
        }
        const long long t = cl.tb + (c - cl.chunk_begin) * WARP + lane;
        if (t >= cl.te) continue;
        T *dst = out[t];
        const long long j0 = offsets[t], j1 = offsets[t + 1];
        if (dst == nullptr) { atomicOr(status, STATUS_NULL_POINTER); continue; }
        if (j1 < j0) { atomicOr(status, STATUS_BAD_OFFSETS); continue; }
        bool add = accumulate != 0;
        if (j0 == j1 && !add)
            for (int e = 0; e < cl.p_out * (cl.p_out + 1); ++e) dst[e] = T(0);
        for (long long j = j0; j < j1; ++j) {
            const T *s = src[j];
            if (s == nullptr) { atomicOr(status, STATUS_NULL_POINTER); continue; }
            if (cl.op == OP_M2M) translate_one<T, OP_M2M, false>(tb, cl.p_in, cl.p_out, s, shift + 3 * j, dst, add, X, buf);
            else if (cl.op == OP_M2L) translate_one<T, OP_M2L, false>(tb, cl.p_in, cl.p_out, s, shift + 3 * j, dst, add, X, buf);
            else translate_one<T, OP_L2L, false>(tb, cl.p_in, cl.p_out, s, shift + 3 * j, dst, add, X, buf);
            add = true;
        }
    }
}

// A whole translation pass in one persistent launch: phases run one after the
// other, and inside a phase warps take chunks of its classes from the phase's
// counter (as in multi_lists_kernel).  Every class carries its own target-major
// lists.  Between phases the CTAs meet at a grid barrier (the launch is
// cooperative, so every CTA is resident); solids written in one phase are read
// in later phases by other SMs, so all reads of solids go through L2 (CG).
constexpr int MAX_PASS_CLASSES = 320;
constexpr int MAX_PASS_PHASES = 64;
enum { STATUS_PASS_TIMEOUT = 32 };
struct PassClass {
    const void *src;             // nnz pointers to input solids
    const void *shift;           // 3 nnz reals
    const long long *offsets;    // n_targets + 1
    void *out;                   // n_targets pointers to output solids
    long long n_targets;
    long long chunk_begin;       // first chunk of the class in the launch's numbering
    int op, p_in, p_out, g, accumulate, pad;
};
struct PassPhase {
    long long chunk_begin, chunk_end;
    int class_begin, class_end;
};
struct PassParams {
    int n_phases;
    int x_slot;                  // scratch elements per lane
    int row_slot;                // shared elements per lane
    PassPhase ph[MAX_PASS_PHASES];
    PassClass c[MAX_PASS_CLASSES];
};

// wait until *ctr reaches target (acquire at GPU scope); bounded by 2^26 polls
// and 2 s
__device__ __forceinline__ bool wait_count(unsigned long long *ctr, unsigned long long target) {
    unsigned long long t0;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
    for (int it = 0; it < (1 << 26); ++it) {
        unsigned long long v;
        asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(ctr) : "memory");
        if (v >= target) return true;
        if ((it & 63) == 63) {
            unsigned long long t;
            asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
            if (t - t0 > 2000000000ull) return false;
        }
        __nanosleep(64);
    }
    return false;
}

template <typename T>
__global__ void __launch_bounds__(256, 1) pass_kernel(DevTables<T> tb, const __grid_constant__ PassParams pp,
                                                      T *scratch, unsigned long long *counters, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & (WARP - 1), warp = threadIdx.x / WARP;
    const long long slot = (long long)blockIdx.x * (blockDim.x / WARP) + warp;
    LaneArr<T> X{scratch + slot * pp.x_slot * WARP + lane};
    LaneArr<T> buf{reinterpret_cast<T *>(smem_raw) + (size_t)warp * pp.row_slot * WARP + lane};
    for (int ph = 0; ph < pp.n_phases; ++ph) {
        const long long c0 = pp.ph[ph].chunk_begin, nch = pp.ph[ph].chunk_end - c0;
        for (;;) {
            long long c = 0;
            if (lane == 0) c = (long long)atomicAdd(counters + ph, 1ull);
            c = __shfl_sync(0xffffffffu, c, 0);
            if (c >= nch) break;
            c += c0;
            int k = pp.ph[ph].class_begin, hi = pp.ph[ph].class_end - 1;   // last class with chunk_begin <= c
            while (k < hi) {
                const int mid = (k + hi + 1) >> 1;
                if (pp.c[mid].chunk_begin <= c) k = mid; else hi = mid - 1;
            }
            const PassClass &cl = pp.c[k];
            const int op = cl.op, p_in = cl.p_in, p_out = cl.p_out, g = cl.g, acc = cl.accumulate;
            const T *const *src = reinterpret_cast<const T *const *>(cl.src);
            const T *shift = reinterpret_cast<const T *>(cl.shift);
            const long long *offsets = cl.offsets;
            T *const *out = reinterpret_cast<T *const *>(cl.out);
            if (g > 1) {
                const long long tg = (c - cl.chunk_begin) * (WARP / g) + lane / g;
                const LaneArr<T> Y = X + x_elems(p_in);
                if (op == OP_M2M)
                    group_chunk<T, OP_M2M, false, true>(tb, p_in, p_out, g, tg, cl.n_targets, src, shift, offsets, out, acc, X, Y, buf, status);
                else if (op == OP_M2L)
                    group_chunk<T, OP_M2L, false, true>(tb, p_in, p_out, g, tg, cl.n_targets, src, shift, offsets, out, acc, X, Y, buf, status);
                else
                    group_chunk<T, OP_L2L, false, true>(tb, p_in, p_out, g, tg, cl.n_targets, src, shift, offsets, out, acc, X, Y, buf, status);
                continue;
            }
            const long long t = (c - cl.chunk_begin) * WARP + lane;
            if (t >= cl.n_targets) continue;
            T *dst = out[t];
            const long long j0 = offsets[t], j1 = offsets[t + 1];
            if (dst == nullptr) { atomicOr(status, STATUS_NULL_POINTER); continue; }
            if (j1 < j0) { atomicOr(status, STATUS_BAD_OFFSETS); continue; }
            bool add = acc != 0;
            if (j0 == j1 && !add)
                for (int e = 0; e < p_out * (p_out + 1); ++e) dst[e] = T(0);
            for (long long j = j0; j < j1; ++j) {
                const T *s = src[j];
                if (s == nullptr) { atomicOr(status, STATUS_NULL_POINTER); continue; }
                if (op == OP_M2M) translate_one<T, OP_M2M, false, true>(tb, p_in, p_out, s, shift + 3 * j, dst, add, X, buf);
                else if (op == OP_M2L) translate_one<T, OP_M2L, false, true>(tb, p_in, p_out, s, shift + 3 * j, dst, add, X, buf);
                else translate_one<T, OP_L2L, false, true>(tb, p_in, p_out, s, shift + 3 * j, dst, add, X, buf);
                add = true;
            }
        }
        if (ph + 1 == pp.n_phases) break;
        // grid barrier: this CTA's writes of the phase are released before it
        // arrives; the next phase starts once every CTA has arrived
        __syncthreads();
        int gave_up = 0;
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(counters + MAX_PASS_PHASES + ph, 1ull);
            if (!wait_count(counters + MAX_PASS_PHASES + ph, gridDim.x)) {
                atomicOr(status, STATUS_PASS_TIMEOUT);
                gave_up = 1;
            }
            __threadfence();
        }
        if (__syncthreads_or(gave_up)) return;
    }
}

// P2M / P2L for boxes of sorted points: one thread per box, the harmonics of
// each point by the Appendix recurrences.  Only the three latest rows of a
// point's harmonics are kept (the column recurrence reaches back two rows), in
// a ring of 3 rows x 2P reals in shared memory; q_j times each row is added
// straight into the box's output solid, which the thread owns.
template <typename T, bool SINGULAR>
__global__ void __launch_bounds__(128) p2x_kernel(int P, const T *points, const T *q,
                                                  const long long *offsets, const T *centres,
                                                  T *out, long long n_boxes, int *status) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *smem = reinterpret_cast<T *>(smem_raw);
    const int lane = threadIdx.x & (WARP - 1), warp = threadIdx.x / WARP;
    const int E = 6 * P;                                      // 3 rows of (re[P], im[P])
    LaneArr<T> H{smem + (size_t)warp * E * WARP + lane};
    const long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (b >= n_boxes) return;
    const long long j0 = offsets[b], j1 = offsets[b + 1];
    if (j1 < j0) { atomicOr(status, STATUS_BAD_OFFSETS); return; }
    T *dst = out + b * (long long)(P * (P + 1));
    for (int e = 0; e < P * (P + 1); ++e) dst[e] = T(0);
    const T cx = centres[3 * b], cy = centres[3 * b + 1], cz = centres[3 * b + 2];
    for (long long j = j0; j < j1; ++j) {
        const T x = points[3 * j] - cx, y = points[3 * j + 1] - cy, z = points[3 * j + 2] - cz;
        const T r2 = x * x + y * y + z * z;
        const T ir2 = T(1) / r2;
        const T qj = q[j];
        for (int n = 0; n < P; ++n) {
            LaneArr<T> hr = H + (n % 3) * 2 * P, hi = hr + P;                 // row n
            LaneArr<T> h1r = H + ((n + 2) % 3) * 2 * P, h1i = h1r + P;        // row n-1
            LaneArr<T> h2r = H + ((n + 1) % 3) * 2 * P, h2i = h2r + P;        // row n-2
            T *orow = dst + n * (n + 1);
            for (int m = 0; m <= n; ++m) {
                T vr, vi;
                if (n == 0) {
                    vr = SINGULAR ? T(1) / sqrt_t(r2) : T(1);
                    vi = T(0);
                } else if (m == n) {
                    // diagonal: R_n^n = (x+iy)/(2n) R_{n-1}^{n-1},
                    //           S_n^n = (2n-1)(x+iy)/|r|^2 S_{n-1}^{n-1}
                    const T pr = h1r[n - 1], pi = h1i[n - 1];
                    const T f = SINGULAR ? T(2 * n - 1) * ir2 : T(1) / T(2 * n);
                    vr = (x * pr - y * pi) * f;
                    vi = (x * pi + y * pr) * f;
                } else {
                    const T ar = h1r[m], ai = h1i[m];
                    T br = T(0), bi = T(0);
                    if (n - 2 >= m) { br = h2r[m]; bi = h2i[m]; }
                    if (SINGULAR) {
                        const T g = T((n - 1) * (n - 1) - m * m);
                        vr = (T(2 * n - 1) * z * ar - g * br) * ir2;
                        vi = (T(2 * n - 1) * z * ai - g * bi) * ir2;
                    } else {
                        const T g = T(1) / T(n * n - m * m);
                        vr = (T(2 * n - 1) * z * ar - r2 * br) * g;
                        vi = (T(2 * n - 1) * z * ai - r2 * bi) * g;
                    }
                }
                hr[m] = vr;
                hi[m] = vi;
                orow[m] = fma_t(qj, vr, orow[m]);
                orow[n + 1 + m] = fma_t(qj, vi, orow[n + 1 + m]);
            }
        }
    }
}

}  // namespace sfmm
