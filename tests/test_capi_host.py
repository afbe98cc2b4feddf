"""C-ABI library on the CPU: exported symbols, status strings, host tables.

No kernel is launched here.  The swap and z-translation tables the kernels
apply are checked against the oracle's harmonics and translations."""
import os
import re
from math import factorial

import numpy as np
import pytest

import pins
from paper_2202_02847_gb300 import workloads as W

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def sf():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300 import sfmm
    return sfmm


def declared_functions():
    names = []
    inc = os.path.join(ROOT, "include")
    for fn in sorted(os.listdir(inc)):
        if fn.endswith(".h"):
            src = open(os.path.join(inc, fn)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names += re.findall(r"\b(sfmm_\w+)\s*\(", src)
    return sorted(set(names))


def test_every_declared_symbol_is_exported(sf):
    names = declared_functions()
    assert len(names) >= 13
    for n in names:
        assert hasattr(sf._lib, n), f"{n} declared in include/ but not exported"


def test_unrolled_orders_match_the_compiled_units(sf):
    """sfmm.UNROLLED_ORDERS (what bench, autotuner and tests take as the
    orders with unrolled kernels) is the registry's list of compiled orders,
    and each of them has a translation unit per real type."""
    csrc = os.path.join(ROOT, "paper_2202_02847_gb300", "csrc")
    reg = open(os.path.join(csrc, "sfmm_unrolled_registry.cu")).read()
    line = re.search(r"#define SFMM_UNROLLED_ORDERS\(X\)(.*)", reg).group(1)
    orders = tuple(int(v) for v in re.findall(r"X\((\d+)\)", line))
    assert orders == sf.UNROLLED_ORDERS
    units = os.listdir(csrc)
    for P in orders:
        for t in ("f64", "f32"):
            assert f"sfmm_unrolled_p{P}_{t}.cu" in units, (P, t)


def test_status_strings(sf):
    for code, name in sf.STATUS.items():
        assert sf.status_string(code).startswith(name)
    assert sf.status_string(99).startswith("SFMM_ERR_?")


def test_create_rejects_bad_arguments_without_touching_the_gpu(sf):
    import ctypes
    h = ctypes.c_void_p()
    assert sf._lib.sfmm_create(0, 1, ctypes.byref(h)) == 2        # order
    assert sf._lib.sfmm_create(65, 1, ctypes.byref(h)) == 2
    assert sf._lib.sfmm_create(31, 0, ctypes.byref(h)) == 2       # FP32 limit
    assert sf._lib.sfmm_create(8, 7, ctypes.byref(h)) == 1        # dtype
    assert sf._lib.sfmm_create(8, 1, None) == 1
    assert sf._lib.sfmm_m2l_batch(None, None, None, None, 4, 4, 1, 0, None) == 1
    assert sf._lib.sfmm_destroy(None) == 0


def test_create_without_gpu_reports_cuda_error(sf):
    import ctypes
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    h = ctypes.c_void_p()
    assert sf._lib.sfmm_create(8, 1, ctypes.byref(h)) == 4
    assert not h.value


def test_chequerboard_golden(sf):
    """Fig. 2 caption: pattern of F_7, G_7, F_8, G_8 (tests/golden)."""
    rows = {}
    for line in open(os.path.join(pins.GOLDEN, "chequerboard_n7_n8.txt")):
        if line.startswith("#") or not line.strip():
            continue
        k, *bits = line.split()
        rows.setdefault(k, []).append([int(b) for b in bits])
    for n in (7, 8):
        F, G = sf.host_swap_matrices(n)
        for key, M in (("F%d" % n, F), ("G%d" % n, G)):
            for i, want in enumerate(rows[key]):
                got = (np.abs(M[i]) > 1e-300).astype(int).tolist()
                assert got == want, (key, i)


@pytest.mark.parametrize("n", [0, 1, 2, 5, 10, 17, 29, 40, 63])
def test_swap_structure_and_involution(sf, n):
    """Chequerboard rule, zero first row/column of G, and the swap is its own
    inverse (Sec. 2.4.3, item 1): F^2 = I, G^2 = diag(0, 1, ..., 1)."""
    F, G = sf.host_swap_matrices(n)
    m, l = np.indices(F.shape)
    assert np.all(F[(n + m + l) % 2 == 1] == 0)
    assert np.all(G[(n + m + l) % 2 == 0] == 0)
    assert np.all(G[0] == 0) and np.all(G[:, 0] == 0)
    I = np.eye(n + 1)
    assert np.abs(F @ F - I).max() < 1e-13
    I[0, 0] = 0
    assert np.abs(G @ G - I).max() < 1e-13
    # entries of the orthogonal Bhat are <= 1; F, G add two of them
    assert np.abs(F).max() <= 2.0 and np.abs(G).max() <= 2.0


@pytest.mark.parametrize("n", [1, 2, 3, 7, 12, 20])
def test_swap_maps_harmonics_at_swapped_point(sf, orc, n):
    """In the orthonormal basis (Rhat = R c, Shat = S / c, c = sqrt((n-m)!(n+m)!))
    the reduced swap turns the harmonics at (x,y,z) into those at (z,y,x)
    (eq. swaptransform with eq. FGmappings), for R and S alike."""
    F, G = sf.host_swap_matrices(n)
    g = W.rng(100 + n)
    P = n + 1
    c = np.array([np.sqrt(float(factorial(n - m)) * float(factorial(n + m))) for m in range(n + 1)])
    worst = 0.0
    for _ in range(3):
        r = g.normal(size=3)
        rs = r[::-1].copy()
        for f, scale in ((orc.regular, c), (orc.singular, 1.0 / c)):
            a, b = f(P, r), f(P, rs)
            o = n * (n + 1)
            are, aim = a[o:o + n + 1] * scale, a[o + n + 1:o + 2 * n + 2] * scale
            bre, bim = b[o:o + n + 1] * scale, b[o + n + 1:o + 2 * n + 2] * scale
            nrm = np.linalg.norm(np.concatenate([are, aim]))
            worst = max(worst, np.abs(F @ are - bre).max() / nrm, np.abs(G @ aim - bim).max() / nrm)
    assert worst < 1e-13


@pytest.mark.parametrize("op", ["m2l", "m2m", "l2l"])
def test_ztranslate_blocks_match_oracle_on_axis(sf, orc, op):
    """The z-axis translation blocks reproduce the oracle's translation for a
    unit shift along +z, column by column (eq. zm2lkernels for M2L)."""
    P = 9
    g = W.rng(7)
    C = W.random_solids(g, 1, P)[0]
    out = orc.translate(op, P, P, C, [0.0, 0.0, 1.0])
    cfac = lambda n, m: np.sqrt(float(factorial(n - m)) * float(factorial(n + m)))
    inb = (lambda n, m: 1 / cfac(n, m)) if op == "l2l" else cfac    # to orthonormal
    outb = (lambda n, m: 1 / cfac(n, m)) if op == "m2m" else cfac   # back
    for m in range(P):
        T = sf.host_ztranslate(op, P, m)
        x = np.array([pins.cplx(C, k, m) * inb(k, m) for k in range(m, P)])
        y = T @ x
        want = np.array([pins.cplx(out, n, m) for n in range(m, P)])
        got = y * np.array([outb(n, m) for n in range(m, P)])
        assert np.abs(got - want).max() <= 1e-13 * np.abs(want).max(), m
