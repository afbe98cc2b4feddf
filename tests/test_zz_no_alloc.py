"""sfmm_translate_batch_noalloc against the regular batch entry point.

The entry point serves callers that cannot allocate device memory where they
translate (plug-ins inside a host framework's fixed memory budget, real-time
loops that forbid cudaMalloc/cudaFree and their synchronisation); its scratch
is a fixed array inside the library.  Two calls in a row, with different ops,
orders and inputs, must each agree with sfmm_*_batch within the FP64
tolerance of the parity tests.  This file is collected last on purpose."""
import numpy as np
import pytest

from paper_2202_02847_gb300 import workloads as W
import gpu_util as U

pytestmark = pytest.mark.gpu


def test_noalloc_matches_batch_on_two_calls_in_a_row():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300 import sfmm
    h = sfmm.Handle(14, "f64")
    g = W.rng(777)
    calls = [("m2l", 12, 12, 20000), ("l2l", 14, 9, 3000)]
    for op, p_in, p_out, count in calls:
        C = torch.tensor(W.random_solids(g, count, p_in), device="cuda")
        sh = torch.tensor(W.shifts(g, count, 2.0, 4.0), device="cuda")
        ref = torch.zeros(count, p_out * (p_out + 1), dtype=torch.float64, device="cuda")
        got = torch.full_like(ref, float("nan"))
        idx = torch.arange(count)
        pin = sfmm.pointer_array(C, p_in * (p_in + 1), idx)
        sfmm.translate_batch(op, h, pin, sfmm.pointer_array(ref, p_out * (p_out + 1), idx),
                             sh, p_in, p_out, count)
        sfmm.translate_batch_noalloc(h, op, pin, sfmm.pointer_array(got, p_out * (p_out + 1), idx),
                                     sh, p_in, p_out, count)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        a, b = got.cpu().numpy(), ref.cpu().numpy()
        assert np.isfinite(a).all()
        assert U.rel_err(a, b, p_out, U.out_kind(op)) <= 1e-12
    with pytest.raises(sfmm.SfmmError) as e:
        sfmm.translate_batch_noalloc(h, "m2l", 1, 1, 1, 15, 4, 1)
    assert e.value.code == 2
    h.close()
