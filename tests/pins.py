"""Pins for the oracle: checks against what the paper and the mathematics fix.

Each pin takes an oracle object and returns (error, tolerance).  None of them
re-types the oracle's formulas: they use closed forms, scipy's associated
Legendre functions, finite-difference harmonicity, direct sums over charges,
exact re-expansion identities, composition, symmetry and hand-derived values.
tests/test_oracle_pins.py asserts every pin on the real oracle, and
tests/test_oracle_mutants.py shows that each planted mistake fails at least one.
"""
import os
from fractions import Fraction
from math import factorial

import numpy as np
from scipy.special import lpmv

from paper_2202_02847_gb300 import workloads as W

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def cplx(solid, n, m):
    """Coefficient C_n^m of a solid (any sign of m, Sec. 2.1 symmetry)."""
    b = n * (n + 1)
    if m >= 0:
        return solid[b + m] + 1j * solid[b + n + 1 + m]
    v = solid[b - m] + 1j * solid[b + n + 1 - m]
    return (-1) ** (-m) * np.conj(v)


def wnorm_err(a, b):
    """Relative difference in the plain 2-norm."""
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


# ------------------------------------------------------------ harmonics pins

def pin_golden_low_orders(o):
    """Hand-derived exact values at r = (1,2,2) (tests/golden)."""
    r = np.array([1.0, 2.0, 2.0])
    R, S = o.regular(3, r), o.singular(3, r)
    err = 0.0
    with open(os.path.join(GOLDEN, "harmonics_r122.txt")) as f:
        for line in f:
            if line.startswith("#") or not line.strip():
                continue
            k, n, m, rn, rd, inn, ind = line.split()
            n, m = int(n), int(m)
            want = float(Fraction(int(rn), int(rd))) + 1j * float(Fraction(int(inn), int(ind)))
            got = cplx(R if k == "R" else S, n, m)
            err = max(err, abs(got - want) / abs(want))
    return err, 1e-14


def pin_z_axis(o):
    """S_n^m(0,0,R) = n!/R^{n+1} for m = 0 and 0 otherwise (Sec. 2.3, R > 0;
    for a point below the origin the same with R^{n+1} -> z^n |z|);
    R_n^m(0,0,z) = z^n/n! for m = 0 and 0 otherwise."""
    P = 12
    err = 0.0
    for Rz in (0.7, 2.5, -1.3):
        S = o.singular(P, [0.0, 0.0, Rz])
        Rg = o.regular(P, [0.0, 0.0, Rz])
        for n in range(P):
            for m in range(n + 1):
                s_want = factorial(n) / (Rz ** n * abs(Rz)) if m == 0 else 0.0
                r_want = Rz ** n / factorial(n) if m == 0 else 0.0
                sc_s = factorial(n) / abs(Rz) ** (n + 1)
                sc_r = abs(Rz) ** n / factorial(n)
                err = max(err, abs(cplx(S, n, m) - s_want) / sc_s,
                          abs(cplx(Rg, n, m) - r_want) / sc_r)
    return err, 1e-13


def pin_legendre(o):
    """R_n^m = r^n Pbar_n^m(cos t) e^{i m p}/(n+m)!, S_n^m = (n-m)! Pbar_n^m e^{i m p}/r^{n+1},
    Pbar = associated Legendre function without the Condon-Shortley phase
    (scipy.special.lpmv carries that phase, so Pbar = (-1)^m lpmv)."""
    g = W.rng(11)
    P = 14
    err = 0.0
    for _ in range(5):
        r = g.normal(size=3) * g.uniform(0.3, 3.0)
        R, S = o.regular(P, r), o.singular(P, r)
        rr = np.linalg.norm(r)
        ct, ph = r[2] / rr, np.arctan2(r[1], r[0])
        for n in range(P):
            for m in range(n + 1):
                pb = (-1) ** m * lpmv(m, n, ct)
                fp, fm = float(factorial(n + m)), float(factorial(n - m))
                rv = rr ** n * pb * np.exp(1j * m * ph) / fp
                sv = fm * pb * np.exp(1j * m * ph) / rr ** (n + 1)
                scale_r = rr ** n / np.sqrt(fp * fm)
                scale_s = np.sqrt(fp * fm) / rr ** (n + 1)
                err = max(err, abs(cplx(R, n, m) - rv) / scale_r,
                          abs(cplx(S, n, m) - sv) / scale_s)
    return err, 1e-12


def pin_harmonicity(o):
    """Every R_n^m and S_n^m solves Laplace's equation: the 7-point Laplacian
    (O(h^2) truncation error) is tiny against the size of the second
    differences plus |C|/|r|^2 (the latter covers the linear n <= 1 terms)."""
    P = 7
    h = 1e-3
    r = np.array([0.4, -0.3, 0.8])
    worst = 0.0
    for f in (o.regular, o.singular):
        c = f(P, r)
        lap = -6 * c
        scale = np.zeros_like(c)
        for ax in range(3):
            e = np.zeros(3)
            e[ax] = h
            fp, fm = f(P, r + e), f(P, r - e)
            lap = lap + fp + fm
            scale = scale + np.abs(fp - 2 * c + fm)
        lap /= h * h
        scale /= h * h
        scale += np.abs(c) / float(r @ r)
        live = scale > 0            # Im C_n^0 vanishes identically
        assert live.sum() >= P * P
        worst = max(worst, float(np.max(np.abs(lap[live]) / scale[live])))
    return worst, 1e-4


def pin_addition_theorem(o):
    """1/|x-y| = sum_{n<P,m} R_n^m(y) conj(S_n^m(x)) for |y| < |x| (the expansion
    behind eq. MLexpansions), with error decaying like (|y|/|x|)^P."""
    g = W.rng(12)
    worst = 0.0
    for _ in range(4):
        y = W.unit_directions(g, 1)[0] * 0.5
        x = W.unit_directions(g, 1)[0] * 2.0
        exact = 1.0 / np.linalg.norm(x - y)
        for P in (4, 8, 16, 24):
            R, S = o.regular(P, y), o.singular(P, x)
            s = 0.0
            for n in range(P):
                for m in range(-n, n + 1):
                    s += cplx(R, n, m) * np.conj(cplx(S, n, m))
            bound = 4.0 * (0.25 ** P) / (1 - 0.25) / 2.0 + 1e-14
            worst = max(worst, abs(s - exact) / bound, abs(s.imag) / 1e-13)
    return worst, 1.0


# ----------------------------------------------------------- expansion pins

def _cluster(seed, nq=32):
    g = W.rng(seed)
    pos, q = W.charge_clusters(g, 1, nq)
    return pos[0], q[0]


def pin_p2m_low_moments(o):
    """Monopole = total charge; dipole rows R_1^0 = z, R_1^1 = (x+iy)/2."""
    pos, q = _cluster(21)
    M = o.p2m(6, pos, q, np.zeros(3))
    want = [(0, 0, q.sum()), (1, 0, (q * pos[:, 2]).sum()),
            (1, 1, (q * (pos[:, 0] + 1j * pos[:, 1])).sum() / 2)]
    err = max(abs(cplx(M, n, m) - w) for n, m, w in want)
    L = o.p2l(4, pos, q, np.array([0.0, 0.0, 5.0]))
    d = pos - np.array([0.0, 0.0, 5.0])
    err = max(err, abs(cplx(L, 0, 0) - (q / np.linalg.norm(d, axis=1)).sum()))
    return err, 1e-13


def pin_eval_vs_direct(o):
    """M and L expansions (eq. MLexpansions) of 32 charges reproduce the
    direct sum of eq. nbody; the error decays with P."""
    pos, q = _cluster(22)
    g = W.rng(23)
    pts_far = W.shifts(g, 8, 3.0, 4.0)
    errs = []
    for P in (4, 8, 12, 16):
        M = o.p2m(P, pos, q, np.zeros(3))
        cB = np.array([3.0, 1.0, -1.0])
        L = o.p2l(P, pos, q, cB)
        e = 0.0
        for x in pts_far:
            d = o.direct(pos, q, x)
            v, im = o.eval_m(P, M, np.zeros(3), x, return_imag=True)
            e = max(e, abs(v - d) / abs(d), abs(im) / abs(d))
        for x in cB + W.unit_directions(g, 8) * 0.4:
            d = o.direct(pos, q, x)
            v, im = o.eval_l(P, L, cB, x, return_imag=True)
            e = max(e, abs(v - d) / abs(d), abs(im) / abs(d))
        errs.append(e)
    ok = all(errs[i + 1] < errs[i] for i in range(3)) and errs[-1] < 1e-6
    return (errs[-1] if ok else 1.0), 1e-6


# --------------------------------------------------------- translation pins

def pin_m2l_eval_vs_direct(o):
    """L = M2L(P2M(charges)) evaluated near x_B matches the direct sum, the
    error decaying with P (eq. m2lkernels, double height)."""
    pos, q = _cluster(31)
    g = W.rng(32)
    worst = []
    for P in (4, 8, 12, 16):
        e = 0.0
        for r in W.shifts(g, 3, 3.0, 4.0):
            M = o.p2m(P, pos, q, np.zeros(3))
            L = o.translate("m2l", P, P, M, r)
            for x in r + W.unit_directions(g, 4) * 0.4:
                d = o.direct(pos, q, x)
                e = max(e, abs(o.eval_l(P, L, r, x) - d) / abs(d))
        worst.append(e)
    ok = all(worst[i + 1] < worst[i] for i in range(3)) and worst[-1] < 1e-5
    return (worst[-1] if ok else 1.0), 1e-5


def pin_m2l_z_axis(o):
    """For r = (0,0,R) only m+l = 0 survives (Sec. 2.3):
    L_n^m = (-1)^{n+m} sum_{k>=m} M_k^m (n+k)!/R^{n+k+1}."""
    g = W.rng(33)
    p_in, p_out = 7, 9
    M = W.random_solids(g, 1, p_in)[0]
    err = 0.0
    for Rz in (1.0, 2.7):
        L = o.translate("m2l", p_in, p_out, M, [0.0, 0.0, Rz])
        for n in range(p_out):
            for m in range(n + 1):
                want = 0j
                for k in range(m, p_in):
                    want += cplx(M, k, m) * factorial(n + k) / Rz ** (n + k + 1)
                want *= (-1) ** (n + m)
                err = max(err, abs(cplx(L, n, m) - want) / max(abs(want), 1e-300))
    return err, 1e-13


def pin_m2l_scaling(o):
    """Scaling law (eq. scaling): M2L(M, s r) = s^{-n} M2L(M', r) row-wise with
    M'_k = s^{-(k+1)} M_k."""
    g = W.rng(34)
    P = 8
    M = W.random_solids(g, 1, P)[0]
    r = W.shifts(g, 1)[0]
    s = 1.7
    Ms = M.copy()
    for k in range(P):
        b = k * (k + 1)
        Ms[b:b + 2 * (k + 1)] *= s ** (-(k + 1))
    A = o.translate("m2l", P, P, M, s * r)
    B = o.translate("m2l", P, P, Ms, r)
    for n in range(P):
        b = n * (n + 1)
        B[b:b + 2 * (n + 1)] *= s ** (-n)
    return wnorm_err(A, B), 1e-13


def pin_z_rotation(o):
    """z-rotation law (Sec. 2.4.2): multiplying coefficients by e^{i m a} is a
    rotation about the z axis; M2L/M2M/L2L commute with it.  With the
    Appendix harmonics (R_n^m, S_n^m proportional to e^{i m phi}) the matching
    point map turns the azimuth by +a: (x cos a - y sin a, x sin a + y cos a, z).
    (The map printed in Sec. 2.4.2 turns it by -a; the algorithm of Sec. 3.4,
    cos(alpha) = y/rho, sin(alpha) = x/rho, needs the +a reading.)"""
    g = W.rng(35)
    P = 7
    a = 0.83
    C = W.random_solids(g, 1, P)[0]
    r = W.shifts(g, 1)[0]
    rr = np.array([r[0] * np.cos(a) - r[1] * np.sin(a), r[0] * np.sin(a) + r[1] * np.cos(a), r[2]])

    def rot(S, P):
        out = S.copy()
        for n in range(P):
            for m in range(n + 1):
                v = cplx(S, n, m) * np.exp(1j * m * a)
                b = n * (n + 1)
                out[b + m], out[b + n + 1 + m] = v.real, v.imag
        return out

    err = 0.0
    for op in ("m2l", "m2m", "l2l"):
        A = o.translate(op, P, P, rot(C, P), rr)
        B = rot(o.translate(op, P, P, C, r), P)
        err = max(err, wnorm_err(A, B))
    return err, 1e-13


def pin_conjugate_symmetry(o):
    """C_n^{-m} = (-1)^m conj(C_n^m) for the outputs of all three translations
    computed over every order m (Sec. 2.1)."""
    g = W.rng(36)
    err = 0.0
    for op, (pi, po) in (("m2l", (6, 8)), ("m2m", (6, 6)), ("l2l", (8, 5))):
        C = W.random_solids(g, 1, pi)[0]
        F = o.full(op, pi, po, C, W.shifts(g, 1)[0])
        scale = np.abs(F).max()
        for n in range(po):
            for m in range(1, n + 1):
                a, b = F[n * n + n - m], (-1) ** m * np.conj(F[n * n + n + m])
                err = max(err, abs(a - b) / scale)
            err = max(err, abs(F[n * n + n].imag) / scale)
    return err, 1e-13


def pin_m2m_exact(o):
    """Shifting a multipole expansion (p_in >= p_out) is exact: M2M(P2M about
    x_A, r) = P2M about x_A + r."""
    pos, q = _cluster(41)
    g = W.rng(42)
    err = 0.0
    for r in W.shifts(g, 3, 0.2, 1.0):
        for pi, po in ((8, 8), (10, 7)):
            M = o.p2m(pi, pos, q, np.zeros(3))
            A = o.translate("m2m", pi, po, M, r)
            B = o.p2m(po, pos, q, r)
            err = max(err, wnorm_err(A, B))
    return err, 1e-13


def pin_m2m_composition(o):
    """M2M(a) followed by M2M(b) equals M2M(a+b)."""
    g = W.rng(43)
    P = 9
    M = W.random_solids(g, 1, P)[0]
    a, b = W.shifts(g, 2, 0.5, 1.5)
    A = o.translate("m2m", P, P, o.translate("m2m", P, P, M, a), b)
    B = o.translate("m2m", P, P, M, a + b)
    return wnorm_err(A, B), 1e-13


def pin_l2l_exact(o):
    """A local expansion is a polynomial: re-expanding it (p_out >= p_in)
    evaluates identically at every point."""
    g = W.rng(44)
    err = 0.0
    for pi, po in ((7, 7), (6, 9)):
        L = W.random_solids(g, 1, pi)[0]
        r = W.shifts(g, 1, 0.3, 1.0)[0]
        L2 = o.translate("l2l", pi, po, L, r)
        for x in W.shifts(g, 5, 0.1, 0.8):
            a = o.eval_l(pi, L, np.zeros(3), x)
            b = o.eval_l(po, L2, r, x)
            err = max(err, abs(a - b) / max(abs(a), 1e-12))
    return err, 1e-12


def pin_l2l_composition(o):
    """L2L(a) followed by L2L(b) equals L2L(a+b)."""
    g = W.rng(45)
    P = 9
    L = W.random_solids(g, 1, P)[0]
    a, b = W.shifts(g, 2, 0.2, 0.9)
    A = o.translate("l2l", P, P, o.translate("l2l", P, P, L, a), b)
    B = o.translate("l2l", P, P, L, a + b)
    return wnorm_err(A, B), 1e-13


def pin_m2l_tiny_by_hand(o):
    """P = 1 and P = 2 by hand at r = (1,2,2) with the golden harmonics:
    L_0^0 = M_0^0/|r|; for p_in = 2, p_out = 1,
    L_0^0 = M_0^0 S_0^0 + sum_{l=-1..1} conj(M_1^l) S_1^l."""
    M = np.array([0.7, 0.0, 0.3, -0.2, 0.0, 0.5])   # M_0^0=0.7, M_1^0=0.3, M_1^1=-0.2+0.5i
    r = np.array([1.0, 2.0, 2.0])
    L1 = o.translate("m2l", 1, 1, M[:2], r)
    e1 = abs(L1[0] - 0.7 / 3.0) + abs(L1[1])
    S00, S10, S11 = 1 / 3, 2 / 27, (1 + 2j) / 27
    S1m1 = -np.conj(S11)
    M11 = -0.2 + 0.5j
    M1m1 = -np.conj(M11)
    want = 0.7 * S00 + 0.3 * S10 + np.conj(M11) * S11 + np.conj(M1m1) * S1m1
    L2 = o.translate("m2l", 2, 1, M, r)
    e2 = abs(L2[0] + 1j * L2[1] - want)
    return max(e1, e2), 1e-15


def pin_mixed_orders(o):
    """Mixed orders: M2L(p_in, p_out) is the first rows of M2L(p_in, p_out + 3),
    and equals M2L(P, P) of the zero-padded input truncated to p_out rows."""
    g = W.rng(46)
    pi, po = 5, 8
    M = W.random_solids(g, 1, pi)[0]
    r = W.shifts(g, 1)[0]
    A = o.translate("m2l", pi, po, M, r)
    B = o.translate("m2l", pi, po + 3, M, r)[: po * (po + 1)]
    Mp = np.zeros(po * (po + 1))
    for n in range(pi):
        b = n * (n + 1)
        Mp[b:b + 2 * (n + 1)] = M[b:b + 2 * (n + 1)]
    C = o.translate("m2l", po, po, Mp, r)
    return max(wnorm_err(A, B), wnorm_err(A, C)), 1e-14


ALL_PINS = [
    pin_golden_low_orders, pin_z_axis, pin_legendre, pin_harmonicity,
    pin_addition_theorem, pin_p2m_low_moments, pin_eval_vs_direct,
    pin_m2l_eval_vs_direct, pin_m2l_z_axis, pin_m2l_scaling, pin_z_rotation,
    pin_conjugate_symmetry, pin_m2m_exact, pin_m2m_composition, pin_l2l_exact,
    pin_l2l_composition, pin_m2l_tiny_by_hand, pin_mixed_orders,
]
