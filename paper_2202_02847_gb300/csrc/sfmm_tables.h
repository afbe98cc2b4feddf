// Host-side precomputation of the translation tables (Sec. 3.1).
#pragma once
#include <vector>

#ifdef __CUDACC__
#define SFMM_HD __host__ __device__
#else
#define SFMM_HD
#endif

namespace sfmm {

enum { OP_M2M = 0, OP_M2L = 1, OP_L2L = 2 };

// All tables are double precision, built on the host in a fixed operation
// order so that x86-64 and aarch64 hosts produce identical bits.
struct HostTables {
    int Pmax = 0;
    // Reduced real swap matrices in the orthonormal basis (eq. FGmappings with
    // Bhat), chequerboard-packed (Fig. 2): for row n, output m = 0..n, the
    // non-zero entries F_n[m][l], l = (n+m)&1, +2, ..., <= n, one m after the
    // other; G_n the same for m >= 1 with l = 1 or 2 (first l >= 1 with n+m+l
    // odd), +2, ..., <= n.  Frow/Grow hold the start of row n (Pmax+1 entries).
    std::vector<double> F, G;
    std::vector<int> Frow, Grow;
    // c_n^m = sqrt((n-m)!(n+m)!) and 1/c_n^m at index n(n+1)/2 + m.
    std::vector<double> c, ic;
    // z-axis translation matrices per op in the orthonormal basis: for every
    // column m a dense (Pmax-m) x (Pmax-m) block, entry (n-m, k-m) maps
    // input row k to output row n.  Block m starts at Q(Pmax) - Q(Pmax-m),
    // Q(x) = x(x+1)(2x+1)/6.
    std::vector<double> Tz[3];
};

// Returns 0 on success, -1 if Pmax is outside [1, 64].
int build_tables(int Pmax, HostTables *t);

// Dense (n+1)x(n+1) F_n and G_n (row m, column l) for 0 <= n < 64.
int dense_swap_matrices(int n, double *F, double *G);

SFMM_HD inline long long ztrans_block_offset(int Pmax, int m) {
    const long long a = Pmax, b = Pmax - m;
    return a * (a + 1) * (2 * a + 1) / 6 - b * (b + 1) * (2 * b + 1) / 6;
}

}  // namespace sfmm
