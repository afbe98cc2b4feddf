"""Serving loop on the GPU: results are the same alone and in a mix of
concurrently admitted requests, and agree with the oracle."""
import numpy as np
import pytest

import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def server():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300.serve import TranslationServer
    s = TranslationServer(P_max=30, pool_size=512, n_shifts=1 << 16, arena_bytes=1 << 30,
                          n_streams=4, chunk=4096)
    yield s
    s.close()


def _mix():
    from paper_2202_02847_gb300.serve import make_requests
    reqs = make_requests(14, seed=9, count_lo=100, count_hi=20000, pool_size=512,
                         n_shifts=1 << 16, mixed_frac=0.3)
    # make sure the mix covers both dtypes, an unrolled order, a large order and mixed orders
    from dataclasses import replace
    reqs[0] = replace(reqs[0], op="m2l", dtype="f64", p_in=10, p_out=10)
    reqs[1] = replace(reqs[1], op="m2m", dtype="f32", p_in=6, p_out=6)
    reqs[2] = replace(reqs[2], op="l2l", dtype="f64", p_in=28, p_out=28)
    reqs[3] = replace(reqs[3], op="m2l", dtype="f32", p_in=30, p_out=27)
    return reqs


def test_same_result_alone_and_in_the_mix(server):
    reqs = _mix()
    alone = {r.rid: server.run_alone(r).out.cpu().numpy() for r in reqs}
    from paper_2202_02847_gb300.serve import poisson_arrivals
    mixed = poisson_arrivals(_mix(), rate_per_s=2000.0, seed=3)
    done = server.run(mixed, keep_outputs=True)
    assert len(done) == len(reqs)
    for r in done:
        assert np.array_equal(r.out.cpu().numpy(), alone[r.rid]), r.rid
        assert r.done_ms is not None and r.done_ms >= 0


def test_served_results_match_oracle(server, orc):
    import torch
    reqs = _mix()[:6]
    done = server.run(reqs, keep_outputs=True)
    for r in done:
        S_in = r.p_in * (r.p_in + 1)
        i = np.arange(0, r.count, max(1, r.count // 7))[:8]
        pool = server.pool[("f64", r.p_in)].cpu().numpy()
        shp = server.shift_pool["f64"].cpu().numpy()
        src = pool[(r.src_start + i) % server.pool_size]
        sh = shp[(r.shift_start + i) % server.n_shifts]
        if r.dtype == "f32":
            # FP32 requests are computed in FP32 from the FP32 pool and shifts
            src = src.astype(np.float32).astype(np.float64)
            sh = sh.astype(np.float32).astype(np.float64)
        want, _ = orc.batch(r.op, r.p_in, r.p_out, src, sh)
        got = r.out.double().cpu().numpy()[i]
        tol = 1e-12 if r.dtype == "f64" else 1e-5
        U.check_rows(got, want, r.p_out, U.out_kind(r.op), tol, a=U.out_radius(r.op, sh),
                     what=f"request {r.rid} {r.op} {r.dtype} {r.p_in}->{r.p_out}")


def test_requests_that_can_never_be_served_are_rejected(server):
    """A request larger than the whole arena, or with an order above P_max,
    is answered at arrival with a reason and no output (instead of waiting
    for memory forever); the others in the same run are served."""
    from dataclasses import replace
    reqs = _mix()[:4]
    big = replace(reqs[0], rid=100, op="m2l", dtype="f64", p_in=30, p_out=30, count=1_000_000)
    high = replace(reqs[1], rid=101, p_in=31, p_out=31)
    done = server.run(reqs + [big, high])
    by = {r.rid: r for r in done}
    assert len(done) == 6
    assert by[100].rejected and "arena" in by[100].rejected and by[100].out is None
    assert by[101].rejected and "outside" in by[101].rejected
    for r in reqs:
        assert by[r.rid].rejected is None and by[r.rid].done_ms is not None
    from paper_2202_02847_gb300.serve import latency_stats
    assert latency_stats(done)["n"] == 4
