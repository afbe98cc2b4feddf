"""Helpers for the GPU parity tests: device buffers, launches, error metrics.

Error metric (the evaluation-weighted relative coefficient error): a local
coefficient L_n^m of a box of circumradius a changes the potential inside the
box by about |dL_n^m| a^n / c_n^m, a multipole coefficient M_n^m the potential
outside it by about |dM_n^m| c_n^m / a^n (c_n^m = sqrt((n-m)!(n+m)!); the
bounds |R_n^m(x)| <= |x|^n / c_n^m and |S_n^m(x)| <= c_n^m / |x|^(n+1) of the
Appendix harmonics).  Every parity test asserts the error of EACH expansion,
||w (got_i - want_i)|| / ||w want_i||, with a the circumradius of that
expansion's own box (sqrt(3)/2 times the edge length)."""
from math import factorial

import numpy as np

BOX_RADIUS = np.sqrt(3.0) / 2.0   # circumradius of the unit source/target box


def box_radius(edge):
    """Circumradius of a cubic box of the given edge length."""
    return BOX_RADIUS * edge


def out_radius(op, sh, a=BOX_RADIUS):
    """Circumradius of the box an output expansion describes, per
    translation: M2M re-expands a multipole about a centre |r| away, so the
    new expansion's box (which must contain the old one) has circumradius
    a + |r|; M2L and L2L outputs are locals of a box of the input's size."""
    sh = np.asarray(sh, dtype=np.float64).reshape(-1, 3)
    if op == "m2m":
        return a + np.linalg.norm(sh, axis=1)
    return np.full(sh.shape[0], a)


def cfac(n, m):
    return np.sqrt(float(factorial(n - m)) * float(factorial(n + m)))


def weights(P, kind, a=BOX_RADIUS):
    """Evaluation weights of the coefficient error metric: a local coefficient
    L_n^m contributes about |L_n^m| a^n / c_n^m to the potential in a box of
    circumradius a, a multipole coefficient M_n^m about |M_n^m| c_n^m / a^n
    (c_n^m = sqrt((n-m)!(n+m)!))."""
    w = np.zeros(P * (P + 1))
    for n in range(P):
        for m in range(n + 1):
            v = (a ** n / cfac(n, m)) if kind == "L" else (cfac(n, m) / a ** n)
            o = n * (n + 1)
            w[o + m] = v
            w[o + n + 1 + m] = v
    return w


def _rows(x, P):
    return np.asarray(x, dtype=np.float64).reshape(-1, P * (P + 1))


def rel_err_rows(got, want, P, kind, a=BOX_RADIUS):
    """Weighted relative coefficient error of every expansion (row i):
    ||w (got_i - want_i)|| / ||w want_i||.  A row whose expected value is
    exactly zero scores 0 if the result is zero too and inf otherwise.
    `a` is a scalar or one circumradius per row."""
    got, want = _rows(got, P), _rows(want, P)
    a = np.broadcast_to(np.asarray(a, dtype=np.float64), (got.shape[0],))
    num = np.empty(got.shape[0])
    den = np.empty(got.shape[0])
    for av in np.unique(a):
        sel = a == av
        w = weights(P, kind, av)
        num[sel] = np.linalg.norm((got[sel] - want[sel]) * w, axis=1)
        den[sel] = np.linalg.norm(want[sel] * w, axis=1)
    out = np.zeros_like(num)
    pos = den > 0
    out[pos] = num[pos] / den[pos]
    out[~pos & (num > 0)] = np.inf
    return out


def rel_err(got, want, P, kind, a=BOX_RADIUS):
    """Weighted relative error of the whole batch in one norm (reported beside
    the per-expansion maximum; no test asserts it alone)."""
    got, want = _rows(got, P), _rows(want, P)
    w = weights(P, kind, a)
    return float(np.linalg.norm((got - want) * w) / np.linalg.norm(want * w))


def check_rows(got, want, P, kind, tol, a=BOX_RADIUS, what=""):
    """Assert the per-expansion error of every row against `tol`; return the
    worst error (the message names the worst row and the aggregate)."""
    e = rel_err_rows(got, want, P, kind, a)
    i = int(np.argmax(e)) if e.size else 0
    worst = float(e[i]) if e.size else 0.0
    assert worst <= tol, (f"{what}: expansion {i} has weighted error {worst:.3e} > {tol:.0e} "
                          f"(batch aggregate {rel_err(got, want, P, kind, a):.3e}, "
                          f"{int((e > tol).sum())} of {e.size} over)")
    return worst


def plain_rel_err(got, want):
    return float(np.linalg.norm(np.asarray(got) - want) / np.linalg.norm(want))


def out_kind(op):
    return "M" if op == "m2m" else "L"


def run_batch(sf, h, op, C, sh, p_in, p_out, dtype, accumulate=False, init=None, device="cuda"):
    """Upload solids and shifts, run one batch call, return the outputs (numpy)."""
    import torch
    tdt = torch.float64 if dtype == "f64" else torch.float32
    count = len(C)
    cin = torch.tensor(np.asarray(C), dtype=tdt, device=device).reshape(count, -1)
    if init is None:
        cout = torch.zeros(count, p_out * (p_out + 1), dtype=tdt, device=device)
    else:
        cout = torch.tensor(np.asarray(init), dtype=tdt, device=device).reshape(count, -1)
    shift = torch.tensor(np.asarray(sh), dtype=tdt, device=device).reshape(count, 3)
    idx = torch.arange(count)
    pin = sf.pointer_array(cin, p_in * (p_in + 1), idx)
    pout = sf.pointer_array(cout, p_out * (p_out + 1), idx)
    sf.translate_batch(op, h, pin, pout, shift, p_in, p_out, count, accumulate=accumulate)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    return cout.double().cpu().numpy()
