"""ctypes wrapper around the C oracle (test infrastructure only).

The oracle is the plain O(P^4) FP64 definition of the solid-harmonic
translations (Kirchhart, solidfmm, Sec. 2.1, eq. m2lkernels; M2M/L2L from the
addition theorem of the regular harmonics).  Only the test suite, the smoke
check and the CPU-baseline leg of the benchmark import this package; the
product library never does.

Solids are numpy float64 arrays of P(P+1) reals in the row layout
[Re C_n^0..Re C_n^n, Im C_n^0..Im C_n^n] for n = 0..P-1.
"""
import ctypes
import os

import numpy as np

from . import build as _build

M2M, M2L, L2L = 0, 1, 2
OPS = {"m2m": M2M, "m2l": M2L, "l2l": L2L}

_dp = ctypes.POINTER(ctypes.c_double)


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class Oracle:
    def __init__(self, path=None):
        path = path or _build.build()
        self.path = path
        lib = ctypes.CDLL(path)
        self.lib = lib
        i, l, d = ctypes.c_int, ctypes.c_long, ctypes.c_double
        sig = {
            "oracle_regular": (None, [i, _dp, _dp]),
            "oracle_singular": (None, [i, _dp, _dp]),
            "oracle_p2m": (None, [i, l, _dp, _dp, _dp, _dp]),
            "oracle_p2l": (None, [i, l, _dp, _dp, _dp, _dp]),
            "oracle_eval_m": (d, [i, _dp, _dp, _dp, _dp]),
            "oracle_eval_l": (d, [i, _dp, _dp, _dp, _dp]),
            "oracle_direct": (d, [l, _dp, _dp, _dp]),
            "oracle_m2l_full": (None, [i, i, _dp, _dp, _dp]),
            "oracle_m2m_full": (None, [i, i, _dp, _dp, _dp]),
            "oracle_l2l_full": (None, [i, i, _dp, _dp, _dp]),
            "oracle_translate": (i, [i, i, i, _dp, _dp, _dp]),
            "oracle_batch": (i, [i, i, i, l, _dp, _dp, _dp, i, i]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args

    # harmonics -----------------------------------------------------------
    def regular(self, P, r):
        out = np.zeros(P * (P + 1))
        self.lib.oracle_regular(P, _ptr(_f64(r)), _ptr(out))
        return out

    def singular(self, P, r):
        out = np.zeros(P * (P + 1))
        self.lib.oracle_singular(P, _ptr(_f64(r)), _ptr(out))
        return out

    # particles -------------------------------------------------------------
    def p2m(self, P, pos, q, centre):
        pos, q = _f64(pos), _f64(q)
        out = np.zeros(P * (P + 1))
        self.lib.oracle_p2m(P, len(q), _ptr(pos), _ptr(q), _ptr(_f64(centre)), _ptr(out))
        return out

    def p2l(self, P, pos, q, centre):
        pos, q = _f64(pos), _f64(q)
        out = np.zeros(P * (P + 1))
        self.lib.oracle_p2l(P, len(q), _ptr(pos), _ptr(q), _ptr(_f64(centre)), _ptr(out))
        return out

    def eval_m(self, P, M, centre, x, return_imag=False):
        im = np.zeros(1)
        v = self.lib.oracle_eval_m(P, _ptr(_f64(M)), _ptr(_f64(centre)), _ptr(_f64(x)), _ptr(im))
        return (v, im[0]) if return_imag else v

    def eval_l(self, P, L, centre, x, return_imag=False):
        im = np.zeros(1)
        v = self.lib.oracle_eval_l(P, _ptr(_f64(L)), _ptr(_f64(centre)), _ptr(_f64(x)), _ptr(im))
        return (v, im[0]) if return_imag else v

    def direct(self, pos, q, x):
        pos, q = _f64(pos), _f64(q)
        return self.lib.oracle_direct(len(q), _ptr(pos), _ptr(q), _ptr(_f64(x)))

    # translations ----------------------------------------------------------
    def full(self, op, p_in, p_out, C, r):
        """All orders -n..n of the result, complex array indexed [n*n+n+m]."""
        out = np.zeros(2 * p_out * p_out)
        f = {M2M: self.lib.oracle_m2m_full, M2L: self.lib.oracle_m2l_full,
             L2L: self.lib.oracle_l2l_full}[OPS.get(op, op)]
        f(p_in, p_out, _ptr(_f64(C)), _ptr(_f64(r)), _ptr(out))
        return out[0::2] + 1j * out[1::2]

    def translate(self, op, p_in, p_out, C, r):
        out = np.zeros(p_out * (p_out + 1))
        rc = self.lib.oracle_translate(OPS.get(op, op), p_in, p_out, _ptr(_f64(C)),
                                       _ptr(_f64(r)), _ptr(out))
        if rc != 0:
            raise ValueError("oracle_translate rejected its arguments")
        return out

    def batch(self, op, p_in, p_out, inp, shift, out=None, accumulate=False,
              nthreads=None):
        """out[i] (+)= op(inp[i], shift[i]); returns (out, threads used)."""
        inp = _f64(inp).reshape(-1, p_in * (p_in + 1))
        shift = _f64(shift).reshape(-1, 3)
        count = inp.shape[0]
        if out is None:
            out = np.zeros((count, p_out * (p_out + 1)))
        nthreads = nthreads or os.cpu_count() or 1
        used = self.lib.oracle_batch(OPS.get(op, op), p_in, p_out, count, _ptr(inp),
                                     _ptr(shift), _ptr(out), int(bool(accumulate)),
                                     int(nthreads))
        return out, used


_DEFAULT = None


def get():
    global _DEFAULT
    if _DEFAULT is None:
        _DEFAULT = Oracle()
    return _DEFAULT
