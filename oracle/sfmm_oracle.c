/*
 * sfmm_oracle.c -- plain, slow, obviously-correct CPU reference for the
 * solid-harmonic translations M2M, M2L and L2L (Laplace kernel 1/|x-y|).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, loads or
 * calls this file.  Only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it.  It shares no code, table or helper with the
 * CUDA path: its harmonics come from the Appendix recurrences evaluated here,
 * and every translation is the plain O(P^4) double sum.
 *
 * All arithmetic is IEEE double precision (fp64).
 *
 * Conventions (Kirchhart, solidfmm, arXiv 2202.02847):
 *   - Expansions (Sec. 2.1, eq. MLexpansions):
 *       phi_M(x) = sum_{n<P} sum_{|m|<=n} M_n^m conj(S_n^m(x - x_A))
 *       phi_L(x) = sum_{n<P} sum_{|m|<=n} L_n^m conj(R_n^m(x - x_B))
 *   - Symmetry (Sec. 2.1): C_n^{-m} = (-1)^m conj(C_n^m), Im C_n^0 = 0.
 *   - Solid layout (Sec. 2.1, Fig. 1; the figure's position numbers are lost,
 *     this is the documented reading): P(P+1) doubles, row n occupies
 *     [n(n+1), (n+1)(n+2)) and holds Re C_n^0..Re C_n^n followed by
 *     Im C_n^0..Im C_n^n.
 *   - Shift vectors: r = (new centre) - (old centre); for M2L r = x_B - x_A
 *     (Sec. 2.1, r_AB).
 *
 * Parity pins: every public function here is pinned by tests that do not
 * reuse its code (closed forms, scipy's associated Legendre functions,
 * discrete harmonicity, direct sums, exact re-expansion identities,
 * composition, conjugate symmetry, hand-derived low orders and planted
 * mistakes).
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* full complex storage index for -n <= m <= n: rows of 2n+1 entries */
static int hidx(int n, int m) { return n * n + n + m; }

/* solid layout positions (see header) */
static int pos_re(int n, int m) { return n * (n + 1) + m; }
static int pos_im(int n, int m) { return n * (n + 1) + n + 1 + m; }

static double sgn(int k) { return (k & 1) ? -1.0 : 1.0; }

/*
 * Appendix, "Regular and Singular Harmonics".  Diagonal first:
 *   R_0^0 = 1,      R_n^n = (x+iy)/(2n) R_{n-1}^{n-1}
 *   S_0^0 = 1/|r|,  S_n^n = (2n-1)(x+iy)/|r|^2 S_{n-1}^{n-1}
 * then up each column m (terms with index n-2 < m are absent):
 *   (n^2-m^2) R_n^m = (2n-1) z R_{n-1}^m - |r|^2 R_{n-2}^m
 *   |r|^2 S_n^m     = (2n-1) z S_{n-1}^m - ((n-1)^2-m^2) S_{n-2}^m
 * Negative orders from the symmetry of Sec. 2.1.
 * R and S are arrays of P*P entries (either may be NULL).
 */
static void harmonics(int P, const double r[3], cplx *R, cplx *S)
{
    const double x = r[0], y = r[1], z = r[2];
    const double r2 = x * x + y * y + z * z;
    const cplx w = x + I * y;
    for (int n = 0; n < P; ++n) {
        for (int m = 0; m <= n; ++m) {
            if (R) {
                cplx v;
                if (n == 0) v = 1.0;
                else if (m == n) v = w / (2.0 * n) * R[hidx(n - 1, n - 1)];
                else {
                    cplx rm2 = (n - 2 >= m) ? R[hidx(n - 2, m)] : 0.0;
                    v = ((2.0 * n - 1.0) * z * R[hidx(n - 1, m)] - r2 * rm2)
                        / ((double)n * n - (double)m * m);
                }
                R[hidx(n, m)] = v;
            }
            if (S) {
                cplx v;
                if (n == 0) v = 1.0 / sqrt(r2);
                else if (m == n) v = (2.0 * n - 1.0) * w / r2 * S[hidx(n - 1, n - 1)];
                else {
                    cplx sm2 = (n - 2 >= m) ? S[hidx(n - 2, m)] : 0.0;
                    v = ((2.0 * n - 1.0) * z * S[hidx(n - 1, m)]
                         - ((double)(n - 1) * (n - 1) - (double)m * m) * sm2) / r2;
                }
                S[hidx(n, m)] = v;
            }
        }
        for (int m = 1; m <= n; ++m) {
            if (R) R[hidx(n, -m)] = sgn(m) * conj(R[hidx(n, m)]);
            if (S) S[hidx(n, -m)] = sgn(m) * conj(S[hidx(n, m)]);
        }
    }
}

/* solid (m >= 0, layout above) -> full complex array with negative m */
static void solid_to_full(int P, const double *C, cplx *F)
{
    for (int n = 0; n < P; ++n)
        for (int m = 0; m <= n; ++m) {
            cplx v = C[pos_re(n, m)] + I * C[pos_im(n, m)];
            F[hidx(n, m)] = v;
            F[hidx(n, -m)] = sgn(m) * conj(v);
        }
}

static void full_to_solid(int P, const cplx *F, double *C)
{
    for (int n = 0; n < P; ++n)
        for (int m = 0; m <= n; ++m) {
            C[pos_re(n, m)] = creal(F[hidx(n, m)]);
            C[pos_im(n, m)] = cimag(F[hidx(n, m)]);
        }
}

/* ---------------------------------------------------------------- harmonics */

/* R_n^m(r) and S_n^m(r) for n < P as solids (P(P+1) doubles each). */
void oracle_regular(int P, const double *r, double *Rsolid)
{
    cplx *R = malloc(sizeof(cplx) * P * P);
    harmonics(P, r, R, NULL);
    full_to_solid(P, R, Rsolid);
    free(R);
}

void oracle_singular(int P, const double *r, double *Ssolid)
{
    cplx *S = malloc(sizeof(cplx) * P * P);
    harmonics(P, r, NULL, S);
    full_to_solid(P, S, Ssolid);
    free(S);
}

/* ------------------------------------------------- particles <-> expansions */

/*
 * P2M / P2L.  Forced by eq. MLexpansions together with the addition theorem
 * 1/|x-y| = sum_{n,m} R_n^m(y) conj(S_n^m(x)) for |y| < |x|:
 *   M_n^m = sum_j q_j R_n^m(y_j - x_A),   L_n^m = sum_j q_j S_n^m(y_j - x_B).
 * pos holds nq points as (x,y,z) triples.
 */
void oracle_p2m(int P, long nq, const double *pos, const double *q,
                const double *centre, double *M)
{
    cplx *R = malloc(sizeof(cplx) * P * P);
    cplx *acc = calloc((size_t)P * P, sizeof(cplx));
    for (long j = 0; j < nq; ++j) {
        double d[3] = {pos[3 * j] - centre[0], pos[3 * j + 1] - centre[1],
                       pos[3 * j + 2] - centre[2]};
        harmonics(P, d, R, NULL);
        for (int i = 0; i < P * P; ++i) acc[i] += q[j] * R[i];
    }
    full_to_solid(P, acc, M);
    free(R);
    free(acc);
}

void oracle_p2l(int P, long nq, const double *pos, const double *q,
                const double *centre, double *L)
{
    cplx *S = malloc(sizeof(cplx) * P * P);
    cplx *acc = calloc((size_t)P * P, sizeof(cplx));
    for (long j = 0; j < nq; ++j) {
        double d[3] = {pos[3 * j] - centre[0], pos[3 * j + 1] - centre[1],
                       pos[3 * j + 2] - centre[2]};
        harmonics(P, d, NULL, S);
        for (int i = 0; i < P * P; ++i) acc[i] += q[j] * S[i];
    }
    full_to_solid(P, acc, L);
    free(S);
    free(acc);
}

/* Evaluate the expansions of eq. MLexpansions at x; imag_out (may be NULL)
 * receives the imaginary part of the sum, which must vanish. */
double oracle_eval_m(int P, const double *M, const double *centre,
                     const double *x, double *imag_out)
{
    cplx *S = malloc(sizeof(cplx) * P * P);
    cplx *Mf = malloc(sizeof(cplx) * P * P);
    double d[3] = {x[0] - centre[0], x[1] - centre[1], x[2] - centre[2]};
    harmonics(P, d, NULL, S);
    solid_to_full(P, M, Mf);
    cplx s = 0.0;
    for (int n = 0; n < P; ++n)
        for (int m = -n; m <= n; ++m) s += Mf[hidx(n, m)] * conj(S[hidx(n, m)]);
    free(S);
    free(Mf);
    if (imag_out) *imag_out = cimag(s);
    return creal(s);
}

double oracle_eval_l(int P, const double *L, const double *centre,
                     const double *x, double *imag_out)
{
    cplx *R = malloc(sizeof(cplx) * P * P);
    cplx *Lf = malloc(sizeof(cplx) * P * P);
    double d[3] = {x[0] - centre[0], x[1] - centre[1], x[2] - centre[2]};
    harmonics(P, d, R, NULL);
    solid_to_full(P, L, Lf);
    cplx s = 0.0;
    for (int n = 0; n < P; ++n)
        for (int m = -n; m <= n; ++m) s += Lf[hidx(n, m)] * conj(R[hidx(n, m)]);
    free(R);
    free(Lf);
    if (imag_out) *imag_out = cimag(s);
    return creal(s);
}

/* Direct sum of eq. nbody with G(x,y) = 1/|x-y| at one target point. */
double oracle_direct(long nq, const double *pos, const double *q, const double *x)
{
    double s = 0.0;
    for (long j = 0; j < nq; ++j) {
        double dx = x[0] - pos[3 * j], dy = x[1] - pos[3 * j + 1], dz = x[2] - pos[3 * j + 2];
        s += q[j] / sqrt(dx * dx + dy * dy + dz * dz);
    }
    return s;
}

/* ------------------------------------------------------------ translations */

/*
 * M2L, double-height kernel (Sec. 2.1, eq. m2lkernels, right-hand form),
 * generalised to mixed orders (Sec. 1.1: input order p_in, output order
 * p_out):  for n < p_out, |m| <= n,
 *   L_n^m = (-1)^n sum_{k<p_in} sum_{|l|<=k} conj(M_k^l) S_{n+k}^{m+l}(r),
 * r = x_B - x_A.  S is needed up to order p_in + p_out - 2.
 * Lfull receives p_out^2 complex values (all m), interleaved re/im.
 */
void oracle_m2l_full(int p_in, int p_out, const double *M, const double *r,
                     double *Lfull)
{
    const int Ps = p_in + p_out - 1;
    cplx *S = malloc(sizeof(cplx) * Ps * Ps);
    cplx *Mf = malloc(sizeof(cplx) * p_in * p_in);
    harmonics(Ps, r, NULL, S);
    solid_to_full(p_in, M, Mf);
    for (int n = 0; n < p_out; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx s = 0.0;
            for (int k = 0; k < p_in; ++k)
                for (int l = -k; l <= k; ++l)
                    s += conj(Mf[hidx(k, l)]) * S[hidx(n + k, m + l)];
            s *= sgn(n);
            Lfull[2 * hidx(n, m)] = creal(s);
            Lfull[2 * hidx(n, m) + 1] = cimag(s);
        }
    free(S);
    free(Mf);
}

/*
 * M2M (the paper implements it but omits the formula, Sec. 1.2).  The
 * multipoles about the new centre x_A' = x_A + r follow from eq. MLexpansions,
 * the P2M form M_n^m = sum_j q_j R_n^m(y_j - x_A) and the addition theorem
 * of the regular harmonics, R_n^m(a+b) = sum_{k<=n} sum_l R_k^l(a) R_{n-k}^{m-l}(b):
 *   M'_n^m = sum_{k <= min(n, p_in-1)} sum_{|l|<=k, |m-l|<=n-k} M_k^l R_{n-k}^{m-l}(-r).
 */
void oracle_m2m_full(int p_in, int p_out, const double *M, const double *r,
                     double *Mfull_out)
{
    const double mr[3] = {-r[0], -r[1], -r[2]};
    cplx *R = malloc(sizeof(cplx) * p_out * p_out);
    cplx *Mf = malloc(sizeof(cplx) * p_in * p_in);
    harmonics(p_out, mr, R, NULL);
    solid_to_full(p_in, M, Mf);
    for (int n = 0; n < p_out; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx s = 0.0;
            for (int k = 0; k <= n && k < p_in; ++k)
                for (int l = -k; l <= k; ++l)
                    if (abs(m - l) <= n - k) s += Mf[hidx(k, l)] * R[hidx(n - k, m - l)];
            Mfull_out[2 * hidx(n, m)] = creal(s);
            Mfull_out[2 * hidx(n, m) + 1] = cimag(s);
        }
    free(R);
    free(Mf);
}

/*
 * L2L (implemented but omitted in the paper, Sec. 1.2).  Re-expanding
 * phi_L(x) = sum L_k^l conj(R_k^l(x - x_B)) about x_B' = x_B + r with the same
 * addition theorem gives
 *   L'_n^m = sum_{k=n}^{p_in-1} sum_{|l|<=k, |l-m|<=k-n} L_k^l conj(R_{k-n}^{l-m}(r)).
 */
void oracle_l2l_full(int p_in, int p_out, const double *L, const double *r,
                     double *Lfull_out)
{
    cplx *R = malloc(sizeof(cplx) * p_in * p_in);
    cplx *Lf = malloc(sizeof(cplx) * p_in * p_in);
    harmonics(p_in, r, R, NULL);
    solid_to_full(p_in, L, Lf);
    for (int n = 0; n < p_out; ++n)
        for (int m = -n; m <= n; ++m) {
            cplx s = 0.0;
            for (int k = n; k < p_in; ++k)
                for (int l = -k; l <= k; ++l)
                    if (abs(l - m) <= k - n) s += Lf[hidx(k, l)] * conj(R[hidx(k - n, l - m)]);
            Lfull_out[2 * hidx(n, m)] = creal(s);
            Lfull_out[2 * hidx(n, m) + 1] = cimag(s);
        }
    free(R);
    free(Lf);
}

/* the solid (m >= 0) part of a full result */
static void full_pairs_to_solid(int P, const double *Ffull, double *C)
{
    for (int n = 0; n < P; ++n)
        for (int m = 0; m <= n; ++m) {
            C[pos_re(n, m)] = Ffull[2 * hidx(n, m)];
            C[pos_im(n, m)] = Ffull[2 * hidx(n, m) + 1];
        }
}

enum { ORACLE_M2M = 0, ORACLE_M2L = 1, ORACLE_L2L = 2 };

/* One translation, solid in -> solid out. */
int oracle_translate(int op, int p_in, int p_out, const double *in,
                     const double *r, double *out)
{
    if (p_in < 1 || p_out < 1) return -1;
    double *full = malloc(sizeof(double) * 2 * p_out * p_out);
    if (op == ORACLE_M2M) oracle_m2m_full(p_in, p_out, in, r, full);
    else if (op == ORACLE_M2L) oracle_m2l_full(p_in, p_out, in, r, full);
    else if (op == ORACLE_L2L) oracle_l2l_full(p_in, p_out, in, r, full);
    else { free(full); return -1; }
    full_pairs_to_solid(p_out, full, out);
    free(full);
    return 0;
}

/*
 * Independent translations, out[i] = op(in[i], shift[i]) (or out[i] += ... when
 * accumulate != 0, in which case no two i may share an output row).
 * in/out are dense arrays of solids (count x p_in(p_in+1), count x p_out(p_out+1)).
 * Spread over nthreads host threads with OpenMP; returns the number used.
 */
int oracle_batch(int op, int p_in, int p_out, long count, const double *in,
                 const double *shift, double *out, int accumulate, int nthreads)
{
    const long sin = (long)p_in * (p_in + 1), sout = (long)p_out * (p_out + 1);
    int used = 1;
    if (nthreads < 1) nthreads = 1;
#pragma omp parallel num_threads(nthreads)
    {
#pragma omp single
        {
#ifdef _OPENMP
            used = omp_get_num_threads();
#endif
        }
        double *tmp = malloc(sizeof(double) * sout);
#pragma omp for schedule(dynamic, 16)
        for (long i = 0; i < count; ++i) {
            oracle_translate(op, p_in, p_out, in + i * sin, shift + 3 * i, tmp);
            double *o = out + i * sout;
            if (accumulate)
                for (long j = 0; j < sout; ++j) o[j] += tmp[j];
            else
                memcpy(o, tmp, sizeof(double) * sout);
        }
        free(tmp);
    }
    return used;
}
