"""sfmm_translate_batch_noalloc against the regular batch entry point and the
oracle.

The entry point serves callers that cannot allocate device memory where they
translate (plug-ins inside a host framework's fixed memory budget, real-time
loops that forbid cudaMalloc/cudaFree and their synchronisation); its scratch
is a fixed array inside the library.  Calls in a row, with different ops,
orders, dtypes and inputs, must each agree with sfmm_*_batch and with the
oracle within the tolerance of the parity tests (FP64 1e-12, FP32 1e-5, per
expansion).  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2202_02847_gb300 import workloads as W
import gpu_util as U

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


def _inputs(orc, g, dtype, op, count, p_in):
    """FP64: random solids; FP32: expansions of charge clusters in a unit box
    (P2M, or P2L about a centre at distance 3 for L2L), rounded to FP32."""
    sh = W.shifts(g, count, 2.0, 4.0)
    if dtype == "f64":
        return W.random_solids(g, count, p_in), sh
    pos, q = W.charge_clusters(g, count, 32)
    if op == "l2l":
        cen = W.unit_directions(g, count) * 3.0
        C = np.stack([orc.p2l(p_in, pos[i], q[i], cen[i]) for i in range(count)])
    else:
        C = np.stack([orc.p2m(p_in, pos[i], q[i], np.zeros(3)) for i in range(count)])
    return (C.astype(np.float32).astype(np.float64), sh.astype(np.float32).astype(np.float64))


def test_noalloc_matches_batch_and_oracle_on_calls_in_a_row(orc):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300 import sfmm
    hs = {"f64": sfmm.Handle(14, "f64"), "f32": sfmm.Handle(20, "f32")}
    g = W.rng(777)
    calls = [("f64", "m2l", 12, 12, 20000), ("f64", "l2l", 14, 9, 3000),
             ("f64", "m2m", 9, 14, 5000), ("f32", "m2m", 10, 13, 4000),
             ("f32", "m2l", 20, 20, 6000)]
    for dtype, op, p_in, p_out, count in calls:
        h = hs[dtype]
        tdt = torch.float64 if dtype == "f64" else torch.float32
        Ch, shh = _inputs(orc, g, dtype, op, count, p_in)
        C = torch.tensor(Ch, dtype=tdt, device="cuda")
        sh = torch.tensor(shh, dtype=tdt, device="cuda")
        ref = torch.zeros(count, p_out * (p_out + 1), dtype=tdt, device="cuda")
        got = torch.full_like(ref, float("nan"))
        idx = torch.arange(count)
        pin = sfmm.pointer_array(C, p_in * (p_in + 1), idx)
        sfmm.translate_batch(op, h, pin, sfmm.pointer_array(ref, p_out * (p_out + 1), idx),
                             sh, p_in, p_out, count)
        sfmm.translate_batch_noalloc(h, op, pin, sfmm.pointer_array(got, p_out * (p_out + 1), idx),
                                     sh, p_in, p_out, count)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        a, b = got.double().cpu().numpy(), ref.double().cpu().numpy()
        assert np.isfinite(a).all()
        rad = U.out_radius(op, shh)
        what = f"{dtype} {op} {p_in}->{p_out}"
        U.check_rows(a, b, p_out, U.out_kind(op), TOL[dtype], a=rad, what=what + " vs batch")
        pick = g.choice(count, size=48, replace=False)
        want, _ = orc.batch(op, p_in, p_out, Ch[pick], shh[pick])
        U.check_rows(a[pick], want, p_out, U.out_kind(op), TOL[dtype], a=rad[pick],
                     what=what + " vs oracle")
    with pytest.raises(sfmm.SfmmError) as e:
        sfmm.translate_batch_noalloc(hs["f64"], "m2l", 1, 1, 1, 15, 4, 1)
    assert e.value.code == 2
    for h in hs.values():
        h.close()
