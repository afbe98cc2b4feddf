"""Tensor-core shift-grouped M2L on a uniform octree level (P = 16) against
the FP64 rotation path on the same interaction lists and against the oracle."""
import numpy as np
import pytest

from paper_2202_02847_gb300 import workloads as W
import gpu_util as U

pytestmark = pytest.mark.gpu

P = 16
TOL = 1e-5     # FP32-class: two-part FP16 split, float-float target sums


@pytest.fixture(scope="module")
def env():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300 import sfmm
    h = sfmm.Handle(P, "f64")
    yield sfmm, h
    h.close()


# sides 8 (64-target tiles, 8 tiles on all SMs), 16 (128-target tiles) and
# 24 (64-target tiles, 216 tiles: CTA ranges split tiles between CTAs)
@pytest.mark.parametrize("ns", [8, 16, 24])
def test_grid_m2l_matches_rotation_path_and_oracle(env, orc, ns):
    import torch
    sfmm, h = env
    lv = W.grid_level(ns)
    g = W.rng(300 + ns)
    # multipoles of a level from P2M of 16 random charges per box (on the device)
    nb = ns ** 3
    pos = lv.centres[:, None, :] + g.uniform(-0.5, 0.5, size=(nb, 16, 3)) * lv.h
    q = g.uniform(-1, 1, size=(nb, 16))
    M = torch.zeros(nb, P * (P + 1), dtype=torch.float64, device="cuda")
    sfmm.p2m_boxes(h, P, torch.tensor(pos.reshape(-1, 3), device="cuda"),
                   torch.tensor(q.reshape(-1), device="cuda"),
                   torch.arange(0, 16 * nb + 1, 16, dtype=torch.int64, device="cuda"),
                   torch.tensor(lv.centres, device="cuda"), M, nb)
    grid = sfmm.Grid(h, P, ns)
    Lg = torch.zeros_like(M)
    grid.m2l(lv.h, M, Lg)
    # the FP64 rotation path on the same lists
    Lr = torch.zeros_like(M)
    S = P * (P + 1)
    src = sfmm.pointer_array(M, S, torch.as_tensor(lv.m2l_sources))
    out = sfmm.pointer_array(Lr, S, torch.arange(nb))
    sfmm.translate_lists(h, "m2l", src, torch.tensor(lv.m2l_shift, device="cuda"),
                         torch.tensor(lv.m2l_offsets, device="cuda"), out, P, P, nb)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    a, b = Lg.cpu().numpy(), Lr.cpu().numpy()
    rad = U.box_radius(lv.h)
    # every target against the FP64 rotation path
    U.check_rows(a, b, P, "L", TOL, a=rad, what=f"grid vs FP64 rotation, side {ns}")
    # the result is the same on every run (each target's sum has a fixed order)
    Lg2 = torch.zeros_like(M)
    grid.m2l(lv.h, M, Lg2)
    torch.cuda.synchronize()
    assert torch.equal(Lg2, Lg)
    # accumulate mode adds
    grid.m2l(lv.h, M, Lg, accumulate=True)
    torch.cuda.synchronize()
    U.check_rows(Lg.cpu().numpy(), 2 * b, P, "L", TOL, a=rad, what="grid accumulate")
    # 32 targets against the oracle (its own multipoles from the charges)
    Mh = {}
    picks = g.choice(nb, size=32, replace=False)
    want = np.zeros((len(picks), S))
    for i, t in enumerate(picks):
        for j in range(lv.m2l_offsets[t], lv.m2l_offsets[t + 1]):
            s_ = int(lv.m2l_sources[j])
            if s_ not in Mh:
                Mh[s_] = orc.p2m(P, pos[s_], q[s_], lv.centres[s_])
            want[i] += orc.translate("m2l", P, P, Mh[s_], lv.m2l_shift[j])
    U.check_rows(a[picks], want, P, "L", TOL, a=rad, what="grid vs oracle")
    grid.close()


def test_grid_rejects_bad_arguments(env):
    sfmm, h = env
    with pytest.raises(sfmm.SfmmError) as e:
        sfmm.Grid(h, 12, 16)
    assert e.value.code == 6
    with pytest.raises(sfmm.SfmmError) as e:
        sfmm.Grid(h, 16, 12)
    assert e.value.code == 1


def test_grid_timeout_path_reports_and_recovers(env):
    """Fault injection from the host into the time-out path: every CTA's copy
    thread acts as if its wait for a free stage had timed out after 40 chunks
    (MMAs and copies still in flight), as on a hung pipeline; the call must
    return, the status word must carry bit 4 (and not bit 8: the work in
    flight drained), and the next call on the same grid and handle must give
    the normal result bitwise."""
    import torch
    sfmm, h = env
    ns = 16
    lv = W.grid_level(ns)
    g = W.rng(399)
    nb = ns ** 3
    pos = lv.centres[:, None, :] + g.uniform(-0.5, 0.5, size=(nb, 16, 3)) * lv.h
    q = g.uniform(-1, 1, size=(nb, 16))
    M = torch.zeros(nb, P * (P + 1), dtype=torch.float64, device="cuda")
    sfmm.p2m_boxes(h, P, torch.tensor(pos.reshape(-1, 3), device="cuda"),
                   torch.tensor(q.reshape(-1), device="cuda"),
                   torch.arange(0, 16 * nb + 1, 16, dtype=torch.int64, device="cuda"),
                   torch.tensor(lv.centres, device="cuda"), M, nb)
    grid = sfmm.Grid(h, P, ns)
    ref = torch.zeros_like(M)
    grid.m2l(lv.h, M, ref)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    grid.inject_timeout(40)
    bad = torch.zeros_like(M)
    grid.m2l(lv.h, M, bad)
    torch.cuda.synchronize()
    st = h.sync_status()
    assert st & 4 and not st & 8, st
    grid.inject_timeout(0)
    again = torch.zeros_like(M)
    grid.m2l(lv.h, M, again)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    assert torch.equal(again, ref)
    with pytest.raises(sfmm.SfmmError):
        grid.inject_timeout(-1)
    grid.close()
