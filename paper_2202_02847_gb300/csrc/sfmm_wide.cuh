// Warp-cooperative translations for high orders (Sec. 3.4 steps 1-4).
//
// The per-thread kernels (sfmm_kernels.cuh, sfmm_unrolled.cuh) give every lane
// a translation of its own.  At high orders that leaves few warps per SM (a
// lane's rotated solid alone is P(P+1) reals of shared memory), every table
// entry is loaded once per translation, and every solid is read and written
// with one transaction per lane.  Here a warp translates W solids together
// (W = 4 in FP32, 2 in FP64: one 16-byte vector per coefficient) and splits
// every step across its lanes by coefficient index:
//   * rows (input rows, output rows): lane m computes coefficient m of a row's
//     scaling, rotation and two axis swaps for the W solids; rows n and
//     R-1-n share one step (n+1 + R-n = R+1 <= 32 lanes, and the longer row
//     brings the lanes with the longer sums);
//   * columns (the z-axis translation): lane n computes output row n of one
//     column; columns M and Q-1-M share one step.
// Every table entry is loaded once per warp step and multiplies W solids;
// every solid value is read from shared memory as one 16-byte vector
// (broadcast when the lanes of a row all need it); the inputs and outputs move
// in coalesced rows.  The warp's shared memory holds the W rotated solids
// (column-addressable, as in the per-thread kernels), two row buffers, and the
// rotation powers and row scales of the W shifts, which lane l forms for
// power l by binary powering.  Orders up to 31 (R+1 <= 32 lanes).
#pragma once

#include <cuda_runtime.h>

#include "sfmm_kernels.cuh"

namespace sfmm {
namespace wide {

constexpr int MAXQ = 31;                 // largest order: a row pair takes Q+1 lanes

// W solids' values of one coefficient, 16 bytes.
template <typename T>
struct alignas(16) Pk {
    static constexpr int W = 16 / sizeof(T);
    T v[W];
};

template <typename T>
__device__ __forceinline__ Pk<T> ldp(const Pk<T> *p) {
    Pk<T> r;
    if constexpr (sizeof(T) == 4) {
        const float4 x = *reinterpret_cast<const float4 *>(p);
        r.v[0] = x.x; r.v[1] = x.y; r.v[2] = x.z; r.v[3] = x.w;
    } else {
        const double2 x = *reinterpret_cast<const double2 *>(p);
        r.v[0] = x.x; r.v[1] = x.y;
    }
    return r;
}
template <typename T>
__device__ __forceinline__ void stp(Pk<T> *p, const Pk<T> &r) {
    if constexpr (sizeof(T) == 4) *reinterpret_cast<float4 *>(p) = make_float4(r.v[0], r.v[1], r.v[2], r.v[3]);
    else *reinterpret_cast<double2 *>(p) = make_double2(r.v[0], r.v[1]);
}
template <typename T>
__device__ __forceinline__ Pk<T> zero_pk() {
    Pk<T> r;
#pragma unroll
    for (int g = 0; g < Pk<T>::W; ++g) r.v[g] = T(0);
    return r;
}

// Warp shared-memory map, in 16-byte units, for orders up to Q:
//   [0, xh)            Re of the rotated solids, row n at n(n+1)/2 (xh = Q(Q+1)/2)
//   [xh, 2xh)          Im
//   2xh + 32 (2s + p)  row buffer s in {0, 1}, part p (0 Re, 1 Im), 32 entries
//   2xh + 128          e^{i l alpha}: Re at +l, Im at +32+l
//   2xh + 192          e^{i l beta}:  Re at +l, Im at +32+l
//   2xh + 256          input row scales, +l;   2xh + 288: output row scales
__host__ __device__ inline int warp_units(int Q) { return Q * (Q + 1) + 320; }

// z^l (c + i s)^l for l >= 0, by binary powering.
template <typename T>
__device__ __forceinline__ void cpow(T c, T s, int l, T &pr, T &pi) {
    T rr = T(1), ri = T(0), br = c, bi = s;
    while (l) {
        if (l & 1) {
            const T t = rr * br - ri * bi;
            ri = fma_t(rr, bi, ri * br);
            rr = t;
        }
        l >>= 1;
        if (l) {
            const T t = br * br - bi * bi;
            bi = T(2) * br * bi;
            br = t;
        }
    }
    pr = rr;
    pi = ri;
}
template <typename T>
__device__ __forceinline__ T rpow(T x, int l) {
    T r = T(1);
    while (l) {
        if (l & 1) r *= x;
        l >>= 1;
        if (l) x *= x;
    }
    return r;
}

// Lane -> (row n, coefficient m) of a step that handles rows a and b >= a
// (b == a: one row); slot = which row buffer.
struct RowLane {
    int n, m, slot;
    bool on;
};
__device__ __forceinline__ RowLane row_lane(int lane, int a, int b) {
    if (lane <= a) return RowLane{a, lane, 0, true};
    const int m = lane - a - 1;
    if (b != a && m <= b) return RowLane{b, m, 1, true};
    return RowLane{a, 0, 0, false};
}

// Coefficient m of one axis swap of row n (eq. Mswapxz / FGmappings) for W
// solids: Re out = sum_l F_n[m][l] Re in_l, Im out = sum_l G_n[m][l] Im in_l
// over the chequerboard non-zeros (Fig. 2), from the transposed tables: the
// lanes of a row read entry i of their rows from consecutive addresses, and
// the inputs l = (n+m)&1 + 2i (two addresses per row: a broadcast).
template <typename T>
__device__ __forceinline__ void swap_lane(const DevTables<T> &tb, int n, int m, const Pk<T> *re,
                                          const Pk<T> *im, Pk<T> &outr, Pk<T> &outi) {
    constexpr int W = Pk<T>::W;
    outr = zero_pk<T>();
    outi = zero_pk<T>();
    const int odd = (n + m) & 1;
    {
        const int cnt = odd ? (n + 1) / 2 : n / 2 + 1;
        const T *__restrict__ F = tb.FT + __ldg(tb.FTrow + n) + m;
        const Pk<T> *x = re + odd;
#pragma unroll 4
        for (int i = 0; i < cnt; ++i, F += n + 1, x += 2) {
            const T t = ldt(F);
            const Pk<T> v = ldp(x);
#pragma unroll
            for (int g = 0; g < W; ++g) outr.v[g] = fma_t(t, v.v[g], outr.v[g]);
        }
    }
    if (m >= 1) {
        const int cnt = odd ? n / 2 : (n + 1) / 2;
        const T *__restrict__ G = tb.GT + __ldg(tb.GTrow + n) + (m - 1);
        const Pk<T> *x = im + (odd ? 2 : 1);
#pragma unroll 4
        for (int i = 0; i < cnt; ++i, G += n, x += 2) {
            const T t = ldt(G);
            const Pk<T> v = ldp(x);
#pragma unroll
            for (int g = 0; g < W; ++g) outi.v[g] = fma_t(t, v.v[g], outi.v[g]);
        }
    }
}

// Batch translations, W per warp (Sec. 3.4): in[i] of order p_in, out[i] of
// order p_out (row n at n(n+1): Re m = 0..n, then Im m = 0..n), shift
// (x, y, z) at 3i; accumulate = add into out.  Null pointers set
// STATUS_NULL_POINTER and skip the translation; a zero shift makes M2M and
// L2L the identity (truncated or zero-padded).  Grid-stride over groups of W.
template <typename T, int OP>
__global__ void __launch_bounds__(256) wbatch_kernel(DevTables<T> tb, const T *const *in, T *const *out,
                                                    const T *shift, int p_in, int p_out, long long count,
                                                    int accumulate, int *status) {
    constexpr int W = Pk<T>::W;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int Q = p_in > p_out ? p_in : p_out;
    const int xh = Q * (Q + 1) / 2;
    Pk<T> *const XRe = reinterpret_cast<Pk<T> *>(smem_raw) + (size_t)warp * warp_units(Q);
    Pk<T> *const XIm = XRe + xh;
    Pk<T> *const RB = XRe + 2 * xh;                        // row buffers: RB + 64 s (+32 Im)
    Pk<T> *const PAr = RB + 128, *const PAi = PAr + 32;    // e^{i l alpha}
    Pk<T> *const PBr = PAr + 64, *const PBi = PAr + 96;    // e^{i l beta}
    Pk<T> *const SI = PAr + 128, *const SO = SI + 32;      // row scales in, out
    const int Rin = (OP == OP_M2M) ? (p_in < p_out ? p_in : p_out) : p_in;
    const int Pm = tb.Pmax;
    const long long nw = (long long)gridDim.x * (blockDim.x >> 5);
    for (long long c = (long long)blockIdx.x * (blockDim.x >> 5) + warp; c * W < count; c += nw) {
        const T *src[W];
        T *dst[W];
        bool ident[W];
        // --- step 1: shift geometry without trigonometric functions (every
        // lane, all W shifts), then lane l forms the powers l of e^{i alpha}
        // and e^{i beta} and the row-l scales (eq. scaling): input M2L
        // |r|^{-(l+1)}, M2M |r|^{-l}, L2L |r|^l; output M2L and L2L |r|^{-l},
        // M2M |r|^l
        Pk<T> par, pai, pbr, pbi, si, so;
#pragma unroll
        for (int g = 0; g < W; ++g) {
            const long long i = c * W + g;
            const T *s = nullptr;
            T *d = nullptr;
            T x = T(0), y = T(0), z = T(1);
            if (i < count) {
                s = in[i];
                d = out[i];
                if (s == nullptr || d == nullptr) {
                    if (lane == 0) atomicOr(status, STATUS_NULL_POINTER);
                    s = nullptr;
                    d = nullptr;
                } else {
                    x = shift[3 * i];
                    y = shift[3 * i + 1];
                    z = shift[3 * i + 2];
                }
            }
            src[g] = s;
            dst[g] = d;
            const T rho2 = x * x + y * y, R2 = rho2 + z * z;
            ident[g] = OP != OP_M2L && !(R2 > T(0));
            const T iR = rsqrt_t(R2), R = R2 * iR;
            T ca = T(1), sa = T(0), rho = T(0);            // cos(alpha) = y/rho, sin(alpha) = x/rho
            if (rho2 > T(0)) {
                const T ir = rsqrt_t(rho2);
                ca = y * ir;
                sa = x * ir;
                rho = rho2 * ir;
            }
            cpow(ca, sa, lane, par.v[g], pai.v[g]);
            cpow(z * iR, -rho * iR, lane, pbr.v[g], pbi.v[g]);   // cos(beta) = z/|r|, sin(beta) = -rho/|r|
            const T pin = rpow((OP == OP_L2L) ? R : iR, lane);
            si.v[g] = (OP == OP_M2L) ? pin * iR : pin;
            so.v[g] = rpow((OP == OP_M2M) ? R : iR, lane);
        }
        stp(PAr + lane, par);
        stp(PAi + lane, pai);
        stp(PBr + lane, pbr);
        stp(PBi + lane, pbi);
        stp(SI + lane, si);
        stp(SO + lane, so);
        __syncwarp();

        // --- step 2: input rows -> rotated frame (scale, basis, rotate alpha,
        // swap, rotate beta, swap), into the column-addressable solid.  The
        // lane's input coefficients of the next step are loaded one step
        // ahead, so that the memory latency overlaps a step of arithmetic.
        const int nst = (Rin + 1) / 2;
        T cre[W], cim[W];
        auto load_in = [&](int st, T *re, T *im) {
            const RowLane q = row_lane(lane, st, Rin - 1 - st);
            const int o = q.n * (q.n + 1);
#pragma unroll
            for (int g = 0; g < W; ++g) {
                re[g] = T(0);
                im[g] = T(0);
                if (q.on && src[g]) {
                    re[g] = src[g][o + q.m];
                    im[g] = src[g][o + q.n + 1 + q.m];
                }
            }
        };
        load_in(0, cre, cim);
        for (int st = 0; st < nst; ++st) {
            const RowLane rl = row_lane(lane, st, Rin - 1 - st);
            const int n = rl.n, m = rl.m;
            Pk<T> *const Br = RB + 64 * rl.slot, *const Bi = Br + 32;
            T nre[W], nim[W];
            if (st + 1 < nst) load_in(st + 1, nre, nim);
            if (rl.on) {
                const T cf = ldt(((OP == OP_L2L) ? tb.ic : tb.c) + n * (n + 1) / 2 + m);
                const T p2 = row_pow2<T>((OP == OP_L2L) ? -n : n);
                const Pk<T> sc = ldp(SI + n), pr = ldp(PAr + m), pi = ldp(PAi + m);
                Pk<T> ar, ai;
#pragma unroll
                for (int g = 0; g < W; ++g) {
                    const T f = basis_factor(sc.v[g], cf, p2);
                    const T re = cre[g] * f, im = cim[g] * f;
                    ar.v[g] = re * pr.v[g] - im * pi.v[g];
                    ai.v[g] = fma_t(re, pi.v[g], im * pr.v[g]);
                }
                stp(Br + m, ar);
                stp(Bi + m, ai);
            }
            __syncwarp();
            Pk<T> br, bi;
            if (rl.on) {
                swap_lane(tb, n, m, Br, Bi, br, bi);
                if (m >= 1) {
                    const Pk<T> pr = ldp(PBr + m), pi = ldp(PBi + m);
#pragma unroll
                    for (int g = 0; g < W; ++g) {
                        const T re = br.v[g], im = bi.v[g];
                        br.v[g] = re * pr.v[g] - im * pi.v[g];
                        bi.v[g] = fma_t(re, pi.v[g], im * pr.v[g]);
                    }
                }
            }
            __syncwarp();
            if (rl.on) {
                stp(Br + m, br);
                stp(Bi + m, bi);
            }
            __syncwarp();
            if (rl.on && m < p_out) {
                Pk<T> xr, xi;
                swap_lane(tb, n, m, Br, Bi, xr, xi);
                stp(XRe + n * (n + 1) / 2 + m, xr);
                stp(XIm + n * (n + 1) / 2 + m, xi);
            }
            __syncwarp();
            if (st + 1 < nst) {
#pragma unroll
                for (int g = 0; g < W; ++g) {
                    cre[g] = nre[g];
                    cim[g] = nim[g];
                }
            }
        }

        // --- step 3: z-axis translation (eq. zm2lkernels for M2L), in place,
        // one column per lane group: out_n = sum_k Tz_M[n][k] X[k][M] over
        // k in [M, p_in) (M2L), [M, min(n+1, p_in)) (M2M), [n, p_in) (L2L)
        for (int st = 0; st < (p_out + 1) / 2; ++st) {
            const int a = st, b = p_out - 1 - st, na = p_out - a;
            int M = a, n = a + lane;
            bool on = lane < na;
            if (!on && b != a && lane - na < p_out - b) {
                M = b;
                n = b + lane - na;
                on = true;
            }
            Pk<T> ar = zero_pk<T>(), ai = zero_pk<T>();
            if (on) {
                const int kb = (OP == OP_L2L) ? n : M;
                const int ke = (OP == OP_M2M) ? ((n + 1 < p_in) ? n + 1 : p_in) : p_in;
                const int ld = Pm - M;
                const T *__restrict__ Tc = tb.TzT[OP] + ztrans_block_offset(Pm, M) + (n - M) +
                                           (long long)(kb - M) * ld;
                int xo = kb * (kb + 1) / 2 + M;
                if (M > 0) {
#pragma unroll 4
                    for (int k = kb; k < ke; ++k, Tc += ld, xo += k) {
                        const T t = ldt(Tc);
                        const Pk<T> xr = ldp(XRe + xo), xi = ldp(XIm + xo);
#pragma unroll
                        for (int g = 0; g < W; ++g) {
                            ar.v[g] = fma_t(t, xr.v[g], ar.v[g]);
                            ai.v[g] = fma_t(t, xi.v[g], ai.v[g]);
                        }
                    }
                } else {                                    // Im of column 0 is zero
#pragma unroll 4
                    for (int k = kb; k < ke; ++k, Tc += ld, xo += k) {
                        const T t = ldt(Tc);
                        const Pk<T> xr = ldp(XRe + xo);
#pragma unroll
                        for (int g = 0; g < W; ++g) ar.v[g] = fma_t(t, xr.v[g], ar.v[g]);
                    }
                }
            }
            __syncwarp();
            if (on) {
                stp(XRe + n * (n + 1) / 2 + M, ar);
                stp(XIm + n * (n + 1) / 2 + M, ai);
            }
            __syncwarp();
        }

        // --- step 4: output rows back (swap, rotate -beta, swap, rotate
        // -alpha, undo the basis change and the scaling), stored or added
        for (int st = 0; st < (p_out + 1) / 2; ++st) {
            const RowLane rl = row_lane(lane, st, p_out - 1 - st);
            const int n = rl.n, m = rl.m;
            Pk<T> *const Br = RB + 64 * rl.slot, *const Bi = Br + 32;
            if (rl.on) {
                Pk<T> br, bi;
                swap_lane(tb, n, m, XRe + n * (n + 1) / 2, XIm + n * (n + 1) / 2, br, bi);
                if (m >= 1) {
                    const Pk<T> pr = ldp(PBr + m), pi = ldp(PBi + m);
#pragma unroll
                    for (int g = 0; g < W; ++g) {
                        const T re = br.v[g], im = bi.v[g];
                        br.v[g] = fma_t(re, pr.v[g], im * pi.v[g]);
                        bi.v[g] = im * pr.v[g] - re * pi.v[g];
                    }
                }
                stp(Br + m, br);
                stp(Bi + m, bi);
            }
            __syncwarp();
            if (rl.on) {
                Pk<T> cr, ci;
                swap_lane(tb, n, m, Br, Bi, cr, ci);
                const T cf = ldt(((OP == OP_M2M) ? tb.ic : tb.c) + n * (n + 1) / 2 + m);
                const T p2 = row_pow2<T>((OP == OP_M2M) ? -n : n);
                const Pk<T> sc = ldp(SO + n), pr = ldp(PAr + m), pi = ldp(PAi + m);
                const int o = n * (n + 1);
#pragma unroll
                for (int g = 0; g < W; ++g) {
                    T *const d = dst[g];
                    if (d == nullptr) continue;
                    const T f = basis_factor(sc.v[g], cf, p2);
                    const T re = cr.v[g] * f, im = ci.v[g] * f;
                    T vr = fma_t(re, pr.v[g], im * pi.v[g]);
                    T vi = im * pr.v[g] - re * pi.v[g];
                    if (ident[g]) {
                        vr = n < p_in ? src[g][o + m] : T(0);
                        vi = n < p_in ? src[g][o + n + 1 + m] : T(0);
                    }
                    if (accumulate) {
                        vr += d[o + m];
                        vi += d[o + n + 1 + m];
                    }
                    d[o + m] = vr;
                    d[o + n + 1 + m] = vi;
                }
            }
            __syncwarp();
        }
    }
}

}  // namespace wide
}  // namespace sfmm
