"""Continuous-batching serving loop for translation requests on one GPU.

A request asks for `count` translations of one op (M2M, M2L or L2L) from
order p_in to order p_out in FP32 or FP64: translation i reads solid
(src_start + i) mod pool_size of the device-resident expansion pool of order
p_in and shift (shift_start + i) mod n_shifts of the device-resident shift pool
(unit directions x U[2,4]).  The
server keeps the tables (one handle per dtype) and the pool resident on the
device, admits requests by device memory (their output, pointer and shift
buffers come from one preallocated arena), cuts every admitted request into
chunks and deals the chunks of all admitted requests round-robin onto several
CUDA streams, so a request that arrives while others run starts as soon as
memory and a stream slot free up and its work overlaps theirs.  Each chunk is
one C-ABI batch call; a translation's result depends only on its own input
and shift, so it is the same alone and in any mix.

Arrival and completion are taken on the host clock (completion = when the
host loop sees the request's last chunk done); latency = completion - arrival.
Admission is first-fit with an ageing bound, chunks are sized by work, and
free stream slots serve the request with the least remaining work first.
FP32 requests are computed by the FP32 handles at every order (the rotation
path in FP32 keeps every translation of the mix within the 1e-5 FP32
tolerance up to order 30), FP64 requests by the FP64 handles.
"""
import math
import time
from dataclasses import dataclass

import numpy as np
import torch

from . import sfmm
from . import workloads as W

OPS = ("m2m", "m2l", "l2l")


@dataclass
class Request:
    rid: int
    op: str
    dtype: str               # "f32" or "f64"
    p_in: int
    p_out: int
    count: int
    src_start: int           # first pool solid (wraps around)
    shift_start: int         # first pool shift (wraps around)
    arrival: float = 0.0     # seconds after the start of the run
    # filled by the server
    done_ms: float = None
    out: torch.Tensor = None
    chunks_left: int = 0
    rejected: str = None     # why the request was not served (None: served)

    def out_bytes(self):
        w = 8 if self.dtype == "f64" else 4
        return self.count * self.p_out * (self.p_out + 1) * w


def translation_flop(p_in, p_out):
    """Algorithmic FLOP of one rotation-based translation (order max(p_in, p_out))."""
    P = max(p_in, p_out)
    return 2 * P * (P + 1) * (2 * P + 1) + 14 * P * (P + 1)


class Arena:
    """First-fit allocator over one preallocated device buffer (bytes)."""

    def __init__(self, nbytes, device):
        self.buf = torch.empty(nbytes, dtype=torch.uint8, device=device)
        self.size = nbytes
        self.free = [(0, nbytes)]          # sorted (offset, size)

    @staticmethod
    def _round(n):
        return (n + 255) // 256 * 256

    def alloc(self, n):
        n = self._round(n)
        for i, (o, s) in enumerate(self.free):
            if s >= n:
                if s == n:
                    self.free.pop(i)
                else:
                    self.free[i] = (o + n, s - n)
                return o, n
        return None

    def release(self, o, n):
        self.free.append((o, n))
        self.free.sort()
        merged = []
        for off, sz in self.free:
            if merged and merged[-1][0] + merged[-1][1] == off:
                merged[-1] = (merged[-1][0], merged[-1][1] + sz)
            else:
                merged.append((off, sz))
        self.free = merged

    def view(self, o, n, dtype):
        return self.buf[o:o + n].view(dtype)


class TranslationServer:
    def __init__(self, P_max=30, pool_size=4096, n_shifts=1 << 20, arena_bytes=8 << 30,
                 n_streams=4, chunk=1 << 20, inflight_per_stream=2, device="cuda", seed=5,
                 chunk_flop=1e9, age_limit_s=0.25):
        self.device = torch.device(device)
        self.P_max = P_max
        self.streams = [torch.cuda.Stream(self.device) for _ in range(n_streams)]
        # Two streams of the highest priority: `fast` runs the requests whose
        # remaining work fits in one chunk, so that a small request does not
        # queue behind the chunks of large ones (its blocks are scheduled
        # before theirs as SMs free up), and `prep` runs the marshalling of
        # newly admitted requests (a few small kernels each).
        self.fast = torch.cuda.Stream(self.device, priority=-100)
        self.prep = torch.cuda.Stream(self.device, priority=-100)
        lanes = self.streams + [self.fast]
        # one handle per stream and dtype: launches that use a handle's global
        # scratch run one after another, so streams with their own handles overlap
        self.hs = {"f64": [sfmm.Handle(P_max, "f64") for _ in lanes],
                   "f32": [sfmm.Handle(P_max, "f32") for _ in lanes]}
        self.h = {k: v[0] for k, v in self.hs.items()}
        self._sidx = {id(s): i for i, s in enumerate(lanes)}
        self.chunk = chunk                   # most translations in one chunk
        self.chunk_flop = chunk_flop         # target work of one chunk
        self.age_limit_s = age_limit_s       # ageing bound of admission and dealing
        nsm = torch.cuda.get_device_properties(self.device).multi_processor_count
        self.wave = nsm * 8 * 32             # translations of one wave of the batch kernel
        self.inflight = inflight_per_stream
        self.arena = Arena(arena_bytes, self.device)
        self.pool = {}
        self.pool_size = pool_size
        self._build_pool(pool_size, seed)
        g = W.rng(seed + 1)
        sh = torch.tensor(W.shifts(g, n_shifts, 2.0, 4.0), device=self.device)
        self.shift_pool = {"f64": sh, "f32": sh.float()}
        self.n_shifts = n_shifts

    # ---------------------------------------------------------------- pool
    def _build_pool(self, n, seed):
        """Resident expansions: P2M of 32 charges per cluster (unit box), every
        order 1..P_max, built on the device by the library's P2M."""
        g = W.rng(seed)
        pos, q = W.charge_clusters(g, n, 32)
        pts = torch.tensor(pos.reshape(-1, 3), device=self.device)
        qq = torch.tensor(q.reshape(-1), device=self.device)
        offs = torch.arange(0, 32 * n + 1, 32, dtype=torch.int64, device=self.device)
        cen = torch.zeros(n, 3, dtype=torch.float64, device=self.device)
        for P in range(1, self.P_max + 1):
            buf = torch.empty(n, P * (P + 1), dtype=torch.float64, device=self.device)
            sfmm.p2m_boxes(self.h["f64"], P, pts, qq, offs, cen, buf, n)
            self.pool[("f64", P)] = buf
            self.pool[("f32", P)] = buf.float()
        torch.cuda.synchronize(self.device)

    # ----------------------------------------------------------- admission
    @staticmethod
    def _need(r):
        """Arena bytes of a request: output, two pointer arrays, shifts."""
        w = 8 if r.dtype == "f64" else 4
        S_out = r.p_out * (r.p_out + 1)
        return [r.count * S_out * w, r.count * 8, r.count * 8, r.count * 3 * w]

    def _reject_reason(self, r):
        """Why a request can never be served (None if it can): an unknown op or
        dtype, orders outside 1..P_max, no translations, or buffers larger than
        the whole arena (it would wait for memory forever)."""
        if r.op not in OPS or r.dtype not in ("f32", "f64"):
            return f"unknown op or dtype ({r.op}, {r.dtype})"
        if not (1 <= r.p_in <= self.P_max and 1 <= r.p_out <= self.P_max):
            return f"orders {r.p_in}->{r.p_out} outside 1..{self.P_max}"
        if r.count < 1:
            return "no translations"
        need = sum(Arena._round(n) for n in self._need(r))
        if need > self.arena.size:
            return f"needs {need} bytes of the {self.arena.size}-byte arena"
        return None

    def _admit(self, r):
        """Reserve arena space for the request's output, pointers and shifts."""
        w = 8 if r.dtype == "f64" else 4
        need = self._need(r)
        got = []
        for n in need:
            a = self.arena.alloc(n)
            if a is None:
                for o, s in got:
                    self.arena.release(o, s)
                return False
            got.append(a)
        r._alloc = got
        r._w = w
        return True

    def _release(self, r):
        for o, s in r._alloc:
            self.arena.release(o, s)
        r._alloc = []

    def _prepare(self, r, stream):
        """Pointer and shift arrays of an admitted request (marshalling only)."""
        tdt = torch.float64 if r._w == 8 else torch.float32
        S_in, S_out = r.p_in * (r.p_in + 1), r.p_out * (r.p_out + 1)
        (oo, on), (io, inn), (po, pn), (so, sn) = r._alloc
        out = self.arena.view(oo, on, tdt)[: r.count * S_out].view(r.count, S_out)
        pool = self.pool[("f64" if r._w == 8 else "f32", r.p_in)]
        with torch.cuda.stream(stream):
            ar = torch.arange(r.count, device=self.device, dtype=torch.int64)
            idx = (ar + r.src_start) % self.pool_size
            pin = self.arena.view(io, inn, torch.int64)[: r.count]
            pin.copy_(idx * (S_in * pool.element_size()) + pool.data_ptr())
            pout = self.arena.view(po, pn, torch.int64)[: r.count]
            pout.copy_(ar * (S_out * out.element_size()) + out.data_ptr())
            sh = self.arena.view(so, sn, tdt)[: r.count * 3].view(r.count, 3)
            spool = self.shift_pool["f64" if r._w == 8 else "f32"]
            torch.index_select(spool, 0, (ar + r.shift_start) % self.n_shifts, out=sh)
            ready = torch.cuda.Event()
            ready.record(stream)
        r.out, r._pin, r._pout, r._sh, r._ready = out, pin, pout, sh, ready
        r._next = 0
        r.chunks_left = 0                # chunks launched and not yet complete

    def _launch_chunk(self, r, stream):
        a = r._next
        b = a + self._chunk_len(r)
        r._next = b
        r._left -= self._work(r, b - a)
        r.chunks_left += 1
        h = self.hs["f64" if r._w == 8 else "f32"][self._sidx[id(stream)]]
        stream.wait_event(r._ready)
        sfmm.translate_batch(r.op, h, r._pin[a:b], r._pout[a:b], r._sh[a:b], r.p_in, r.p_out,
                             b - a, stream=stream)
        ev = torch.cuda.Event()
        ev.record(stream)
        return ev

    # ----------------------------------------------------------------- run
    def _work(self, r, n=None):
        """FLOP of n translations of the request (all of them by default)."""
        return translation_flop(r.p_in, r.p_out) * (r.count if n is None else n)

    def _chunk_len(self, r):
        """Translations in the request's next chunk: about chunk_flop of work,
        but at least a quarter wave of the batch kernel (chunks of the four
        streams overlap on the device, so four such chunks keep every SM
        busy), and at most `chunk`."""
        per = translation_flop(r.p_in, r.p_out)
        n = max(self.wave // 4, int(self.chunk_flop // per))
        return max(1, min(n, self.chunk, r.count - r._next))

    def run(self, requests, keep_outputs=False):
        """Serve the requests at their arrival times (seconds after start).

        Admission is first-fit in arrival order: a request whose output does not
        fit in the arena yet is skipped in favour of later ones that fit, until
        it has waited `age_limit_s`; from then on nothing is admitted past it.
        Free stream slots take the next chunk of the admitted request with the
        least remaining work (shortest remaining work first), except that a
        request older than `age_limit_s` goes first.  Arrival and completion are
        both taken on the host clock: done_ms = when the host loop saw the
        request's last chunk complete, in ms after the start of the run.
        A request that can never be served (orders outside 1..P_max, no
        translations, buffers larger than the whole arena) is answered at its
        arrival with `rejected` set and no output, and queues nothing.
        Returns the finished requests, rejected ones included; with keep_outputs
        the results are copied out of the arena before its space is reused."""
        reqs = sorted(requests, key=lambda r: r.arrival)
        torch.cuda.synchronize(self.device)
        t0 = time.perf_counter()
        pending = list(reqs)[::-1]     # not yet arrived (pop from the end)
        queue = []                     # arrived, waiting for memory
        active = []                    # admitted, chunks left to launch
        lanes = self.streams + [self.fast]
        FAST = len(self.streams)
        inflight = {i: [] for i in range(len(lanes))}          # stream -> [(ev, req)]
        finished = []
        while pending or queue or active or any(inflight.values()):
            now = time.perf_counter() - t0
            while pending and pending[-1].arrival <= now:
                r = pending.pop()
                why = self._reject_reason(r)
                if why is None:
                    queue.append(r)
                else:                      # answered at once, never queued
                    r.rejected = why
                    r.done_ms = 1e3 * (time.perf_counter() - t0)
                    r.out = None
                    finished.append(r)
            # admission: first fit, bounded by age
            i = 0
            while i < len(queue):
                r = queue[i]
                if self._admit(r):
                    queue.pop(i)
                    self._prepare(r, self.prep)
                    r._left = self._work(r)
                    active.append(r)
                    continue
                if now - r.arrival > self.age_limit_s:
                    break
                i += 1
            # retire finished chunks (host clock)
            for si, lst in inflight.items():
                keep = []
                for ev, r in lst:
                    if ev.query():
                        r.chunks_left -= 1
                        if r.chunks_left == 0 and r._next >= r.count:
                            r.done_ms = 1e3 * (time.perf_counter() - t0)
                            if keep_outputs:
                                cur = torch.cuda.current_stream(self.device)
                                cur.wait_event(ev)
                                # always a copy: the arena space is reused at once
                                r.out = r.out.clone()
                                cur.synchronize()
                            else:
                                r.out = None
                            self._release(r)
                            finished.append(r)
                    else:
                        keep.append((ev, r))
                inflight[si] = keep
            # deal chunks onto free stream slots: first the fast stream (the
            # request with the least remaining work, if that fits in one chunk)
            launched = False
            if active and len(inflight[FAST]) < self.inflight:
                r = min(active, key=lambda x: (x._left, x.arrival))
                if r._left <= self.chunk_flop:
                    ev = self._launch_chunk(r, self.fast)
                    inflight[FAST].append((ev, r))
                    if r._next >= r.count:
                        active.remove(r)
                    launched = True
            for si, s in enumerate(self.streams):
                if len(inflight[si]) >= self.inflight or not active:
                    continue
                now = time.perf_counter() - t0
                old = [r for r in active if now - r.arrival > self.age_limit_s]
                r = min(old, key=lambda x: x.arrival) if old else min(active, key=lambda x: (x._left, x.arrival))
                ev = self._launch_chunk(r, s)
                inflight[si].append((ev, r))
                if r._next >= r.count:
                    active.remove(r)
                launched = True
            if not launched:
                busy = active or queue or any(inflight.values())
                wait = 5e-5 if busy else 1e-3
                if pending:
                    wait = min(wait, max(0.0, pending[-1].arrival - (time.perf_counter() - t0)))
                time.sleep(wait)
        torch.cuda.synchronize(self.device)
        return finished

    def run_alone(self, r):
        """One request on its own (for the same-result check)."""
        r2 = Request(r.rid, r.op, r.dtype, r.p_in, r.p_out, r.count, r.src_start,
                     r.shift_start, 0.0)
        return self.run([r2], keep_outputs=True)[0]

    def close(self):
        for hl in self.hs.values():
            for h in hl:
                h.close()


def make_requests(n, seed=5, P_lo=3, P_hi=30, count_lo=1e3, count_hi=1e6, pool_size=4096,
                  n_shifts=1 << 20, mixed_frac=0.1):
    """The serving mix: op ~ U{M2M, M2L, L2L}; P ~ U{P_lo..P_hi} with p_in = p_out,
    a fraction with p_out = p_in +- U{1..4}; count log-uniform in [count_lo, count_hi];
    dtype ~ U{FP32, FP64}; inputs are ranges of the resident pools (shifts are
    unit directions x U[2,4], i.e. |r|/box in [2,4] for unit boxes)."""
    g = W.rng(seed)
    out = []
    for i in range(n):
        op = OPS[g.integers(0, 3)]
        P = int(g.integers(P_lo, P_hi + 1))
        p_in = p_out = P
        if g.uniform() < mixed_frac:
            p_out = int(np.clip(P + g.choice([-1, 1]) * g.integers(1, 5), P_lo, P_hi))
        count = int(math.floor(10 ** g.uniform(math.log10(count_lo), math.log10(count_hi))))
        dtype = "f32" if g.uniform() < 0.5 else "f64"
        out.append(Request(i, op, dtype, p_in, p_out, count, int(g.integers(0, pool_size)),
                           int(g.integers(0, n_shifts))))
    return out


def poisson_arrivals(requests, rate_per_s, seed=55):
    g = W.rng(seed)
    t = 0.0
    for r in requests:
        t += g.exponential(1.0 / rate_per_s)
        r.arrival = t
    return requests


def latency_stats(finished, alone_ms=None):
    """Latency percentiles (host clock, arrival to completion), and the
    percentiles of latency per GFLOP of the request's work.  The workload's
    service times span five orders of magnitude (counts 1e3..1e6 times a
    per-translation cost that grows as P^3), so the latency percentiles mostly
    rank request sizes; `alone_ms` (request id -> latency of the same request
    served alone on an idle device) adds the slowdown percentiles, latency in
    the mix over latency alone, which compare each request with itself."""
    finished = [r for r in finished if r.rejected is None]
    lat = np.array([r.done_ms - 1e3 * r.arrival for r in finished])
    work = np.array([translation_flop(r.p_in, r.p_out) * r.count for r in finished]) * 1e-9
    per = lat / work
    st = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
          "mean_ms": float(lat.mean()), "n": len(lat),
          "p50_ms_per_gflop": float(np.percentile(per, 50)),
          "p99_ms_per_gflop": float(np.percentile(per, 99))}
    if alone_ms:
        slow = np.array([(r.done_ms - 1e3 * r.arrival) / max(alone_ms[r.rid], 1e-3) for r in finished])
        st["p50_slowdown"] = float(np.percentile(slow, 50))
        st["p99_slowdown"] = float(np.percentile(slow, 99))
    return st
