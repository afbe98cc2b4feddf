"""Autotuner for the launch policy of each (op, p_in, p_out, dtype).

The paper picks its register-block sizes (mu, nu) per CPU (Sec. 3.2); here the
choice is which kernel variant serves an order pair on this GPU (fixed-order
unrolled kernel, generic kernel with the working set in shared memory, or
generic kernel with the rotated solid in global scratch) and how many warps a
block has.  Each candidate is timed with CUDA events on a batch of synthetic
translations; the fastest is installed on the handle with sfmm_set_policy and
remembered in a JSON cache keyed by GPU name, dtype and order pair.
"""
import json
import os

import torch

from . import sfmm
from . import workloads as W


def _key(dtype, op, p_in, p_out):
    name = torch.cuda.get_device_name().replace(" ", "_")
    return f"{name}|{dtype}|{op}|{p_in}|{p_out}"


class Autotuner:
    def __init__(self, handle, dtype="f64", cache_path=None):
        self.h, self.dtype = handle, dtype
        self.cache_path = cache_path
        self.cache = {}
        if cache_path and os.path.exists(cache_path):
            with open(cache_path) as f:
                self.cache = json.load(f)

    def candidates(self, p_in, p_out):
        c = [("unrolled", 0)] if (p_in == p_out and p_in in sfmm.UNROLLED_ORDERS) else []
        c += [("shared", w) for w in (1, 2, 4, 8)]
        c += [("global", w) for w in (1, 2, 4)]
        return c

    def _time(self, op, p_in, p_out, n, reps):
        g = W.rng(1234 + 7 * p_in + p_out)
        tdt = torch.float64 if self.dtype == "f64" else torch.float32
        C = torch.tensor(W.random_solids(g, 512, p_in), dtype=tdt, device="cuda")
        out = torch.empty(n, p_out * (p_out + 1), dtype=tdt, device="cuda")
        idx = torch.arange(n, device="cuda")
        pin = sfmm.pointer_array(C, p_in * (p_in + 1), idx % 512)
        pout = sfmm.pointer_array(out, p_out * (p_out + 1), idx)
        sh = torch.tensor(W.shifts(g, n), dtype=tdt, device="cuda")
        sfmm.translate_batch(op, self.h, pin, pout, sh, p_in, p_out, n)     # warm-up
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for _ in range(reps):
            sfmm.translate_batch(op, self.h, pin, pout, sh, p_in, p_out, n)
        e1.record()
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / reps

    def tune(self, op, p_in, p_out, n=None, reps=3):
        """Pick and install the fastest policy; returns (policy, warps, ms per n).
        The sample (default: two full waves of 4 warps per SM) fills the GPU, so
        that variants are compared at the occupancy they reach in production."""
        if n is None:
            n = max(8192, 2 * 4 * 32 * torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count)
        key = _key(self.dtype, op, p_in, p_out)
        if key in self.cache:
            pol, w, ms = self.cache[key]
            sfmm.set_policy(self.h, op, p_in, p_out, pol, w)
            return pol, w, ms
        best = None
        for pol, w in self.candidates(p_in, p_out):
            try:
                sfmm.set_policy(self.h, op, p_in, p_out, pol, w)
            except sfmm.SfmmError:
                continue
            ms = self._time(op, p_in, p_out, n, reps)
            if best is None or ms < best[2]:
                best = (pol, w, ms)
        sfmm.set_policy(self.h, op, p_in, p_out, best[0], best[1])
        self.cache[key] = list(best)
        return best

    def save(self):
        if self.cache_path:
            os.makedirs(os.path.dirname(os.path.abspath(self.cache_path)), exist_ok=True)
            with open(self.cache_path, "w") as f:
                json.dump(self.cache, f, indent=1, sort_keys=True)
