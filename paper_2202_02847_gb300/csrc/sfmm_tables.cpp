// Host-side precomputation of the translation tables (Sec. 3.1).
//
// Dehnen's axis-swap matrices B_n^{m,l} follow the recurrence printed in the
// Appendix ("The Matrices B_n^{m,l}"), starting from B_0^{0,0} = 1:
//   2 B_{n+1}^{m,l}   = B_n^{m,l-1} - B_n^{m,l+1}                  (|m| <= n)
//   2 B_{n+1}^{n+1,l} = B_n^{n,l-1} + 2 B_n^{n,l} + B_n^{n,l+1}    (new top row)
//   2 B_{n+1}^{-n-1,l}= B_n^{-n,l-1} - 2 B_n^{-n,l} + B_n^{-n,l+1} (new bottom row)
// (the printed "m +- 1" equation is over-determined for interior rows; it is
// used only to open the two new edge rows).  The recurrence only halves, so
// N_n = 2^n B_n is an integer matrix; it is carried exactly in 128-bit
// integers (|N_63| < 2^123) and rounded to double once per table entry.
//
// The tables are expressed in the orthonormal basis
//   Mhat_n^m = M_n^m c_n^m,  Lhat_n^m = L_n^m / c_n^m,  c_n^m = sqrt((n-m)!(n+m)!)
// in which the M-side swap (M_n^m -> sum_l B^{l,m} M_n^l, eq. swaptransform)
// and the L-side swap (L_n^m -> sum_l B^{m,l} L_n^l) are one and the same
// symmetric orthogonal matrix Bhat^{m,l} = c_m B^{l,m} / c_l.  (Sec. 3.1 and
// Sec. 3.4 step 4(b) use the transposes of F, G for the L side; with the
// paper's own normalisation of R and S that is not the inverse operation, but
// in the orthonormal basis the same F, G serve both sides.)
#include "sfmm_tables.h"

#include <cmath>
#include <cstring>

namespace sfmm {

namespace {

typedef __int128 i128;

// Integer numerators N_n (2n+1 x 2n+1, row m+n, column l+n) of B_n.
struct Bint {
    int n = 0;
    std::vector<i128> a;
    i128 at(int m, int l) const {
        if (m < -n || m > n || l < -n || l > n) return 0;
        return a[(size_t)(m + n) * (2 * n + 1) + (l + n)];
    }
};

Bint next_B(const Bint &b) {
    const int n = b.n, N = n + 1, W = 2 * N + 1;
    Bint r;
    r.n = N;
    r.a.assign((size_t)W * W, 0);
    auto set = [&](int m, int l, i128 v) { r.a[(size_t)(m + N) * W + (l + N)] = v; };
    for (int m = -n; m <= n; ++m)
        for (int l = -N; l <= N; ++l) set(m, l, b.at(m, l - 1) - b.at(m, l + 1));
    for (int l = -N; l <= N; ++l) {
        set(N, l, b.at(n, l - 1) + 2 * b.at(n, l) + b.at(n, l + 1));
        set(-N, l, b.at(-n, l - 1) - 2 * b.at(-n, l) + b.at(-n, l + 1));
    }
    return r;
}

// c_m / c_l for row n, c_j = sqrt((n-j)!(n+j)!), 0 <= m, l <= n, as a
// product of the quotients f(j+1)/f(j) = (n+j+1)/(n-j) of f(j) = c_j^2.
double c_ratio(int n, int m, int l) {
    double q = 1.0;
    if (m > l)
        for (int j = l; j < m; ++j) q *= (double)(n + j + 1) / (double)(n - j);
    else
        for (int j = m; j < l; ++j) q /= (double)(n + j + 1) / (double)(n - j);
    return std::sqrt(q);
}

double to_double(i128 v) {
    // exact split into two 64-bit halves, each converted once
    const bool neg = v < 0;
    unsigned __int128 u = neg ? (unsigned __int128)(-v) : (unsigned __int128)v;
    const unsigned long long hi = (unsigned long long)(u >> 64), lo = (unsigned long long)u;
    double d = std::ldexp((double)hi, 64) + (double)lo;
    return neg ? -d : d;
}

// Reduced real swap matrices of row n (dense, row m, column l) from N_n.
void reduce(const Bint &b, double *F, double *G) {
    const int n = b.n, W = n + 1;
    const double scale = std::ldexp(1.0, -n);
    for (int m = 0; m <= n; ++m)
        for (int l = 0; l <= n; ++l) {
            const double cr = c_ratio(n, m, l) * scale;
            const double s = (l & 1) ? -1.0 : 1.0;
            i128 f, g;
            if (l == 0) {
                f = b.at(0, m);
                g = 0;
            } else {
                f = b.at(l, m) + (s < 0 ? -b.at(-l, m) : b.at(-l, m));
                g = (m == 0) ? 0 : b.at(l, m) - (s < 0 ? -b.at(-l, m) : b.at(-l, m));
            }
            F[m * W + l] = to_double(f) * cr;
            G[m * W + l] = to_double(g) * cr;
        }
}

}  // namespace

int dense_swap_matrices(int n, double *F, double *G) {
    if (n < 0 || n > 63) return -1;
    Bint b;
    b.n = 0;
    b.a.assign(1, 1);
    for (int k = 0; k < n; ++k) b = next_B(b);
    reduce(b, F, G);
    return 0;
}

int build_tables(int Pmax, HostTables *t) {
    if (Pmax < 1 || Pmax > 64) return -1;
    t->Pmax = Pmax;
    t->F.clear();
    t->G.clear();
    t->Frow.assign(Pmax + 1, 0);
    t->Grow.assign(Pmax + 1, 0);

    Bint b;
    b.n = 0;
    b.a.assign(1, 1);
    std::vector<double> F, G;
    for (int n = 0; n < Pmax; ++n) {
        if (n > 0) b = next_B(b);
        const int W = n + 1;
        F.assign((size_t)W * W, 0.0);
        G.assign((size_t)W * W, 0.0);
        reduce(b, F.data(), G.data());
        t->Frow[n] = (int)t->F.size();
        t->Grow[n] = (int)t->G.size();
        for (int m = 0; m <= n; ++m)
            for (int l = (n + m) & 1; l <= n; l += 2) t->F.push_back(F[m * W + l]);
        for (int m = 1; m <= n; ++m)
            for (int l = ((n + m + 1) & 1) ? 1 : 2; l <= n; l += 2) t->G.push_back(G[m * W + l]);
    }
    t->Frow[Pmax] = (int)t->F.size();
    t->Grow[Pmax] = (int)t->G.size();

    // factorials 0! .. (2 Pmax - 2)! (Sec. 3.1) and the basis factors
    std::vector<double> fact(2 * Pmax + 1, 1.0);
    for (int j = 1; j <= 2 * Pmax; ++j) fact[j] = fact[j - 1] * (double)j;
    const int nc = Pmax * (Pmax + 1) / 2;
    t->c.assign(nc, 0.0);
    t->ic.assign(nc, 0.0);
    for (int n = 0; n < Pmax; ++n)
        for (int m = 0; m <= n; ++m) {
            const double v = std::sqrt(fact[n - m]) * std::sqrt(fact[n + m]);
            t->c[n * (n + 1) / 2 + m] = v;
            t->ic[n * (n + 1) / 2 + m] = 1.0 / v;
        }
    auto C = [&](int n, int m) { return t->c[n * (n + 1) / 2 + m]; };

    // z-axis translations with unit shift along +z, orthonormal basis:
    //  M2L (eq. zm2lkernels, double height): L_n^m = (-1)^{n+m} sum_k (n+k)! M_k^m
    //  M2M: M'_n^m = sum_{k<=n} (-1)^{n-k}/(n-k)! M_k^m  (R_j^0(0,0,-1) = (-1)^j/j!)
    //  L2L: L'_n^m = sum_{k>=n} L_k^m/(k-n)!             (R_j^0(0,0,1) = 1/j!)
    const long long total = ztrans_block_offset(Pmax, Pmax);
    for (int op = 0; op < 3; ++op) t->Tz[op].assign((size_t)total, 0.0);
    for (int m = 0; m < Pmax; ++m) {
        const long long base = ztrans_block_offset(Pmax, m);
        const int W = Pmax - m;
        for (int n = m; n < Pmax; ++n)
            for (int k = m; k < Pmax; ++k) {
                const size_t i = (size_t)(base + (long long)(n - m) * W + (k - m));
                const double s = ((n + m) & 1) ? -1.0 : 1.0;
                t->Tz[OP_M2L][i] = s * (fact[n + k] / C(n, m)) / C(k, m);
                if (k <= n) {
                    const double s2 = ((n - k) & 1) ? -1.0 : 1.0;
                    t->Tz[OP_M2M][i] = s2 * (C(n, m) / fact[n - k]) / C(k, m);
                }
                if (k >= n) t->Tz[OP_L2L][i] = (C(k, m) / fact[k - n]) / C(n, m);
            }
    }
    return 0;
}

}  // namespace sfmm
