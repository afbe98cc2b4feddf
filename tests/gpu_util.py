"""Helpers for the GPU parity tests: device buffers, launches, error metrics."""
from math import factorial

import numpy as np

BOX_RADIUS = np.sqrt(3.0) / 2.0   # circumradius of the unit source/target box


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


def rel_err(got, want, P, kind):
    """Weighted relative coefficient error ||w (got - want)|| / ||w want||."""
    w = weights(P, kind)
    got = np.asarray(got).reshape(-1, P * (P + 1))
    want = np.asarray(want).reshape(-1, P * (P + 1))
    return float(np.linalg.norm((got - want) * w) / np.linalg.norm(want * w))


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
