"""CUDA path against the oracle, element by element, through the C ABI.

Tolerances: the weighted relative coefficient error of EVERY expansion
(tests/gpu_util.py: per output solid, normalised by that solid's own weighted
norm) must be <= 1e-12 in FP64 and <= 1e-5 in FP32."""
import numpy as np
import pytest

from paper_2202_02847_gb300 import workloads as W
import gpu_util as U

pytestmark = pytest.mark.gpu

TOL = {"f64": 1e-12, "f32": 1e-5}


@pytest.fixture(scope="module")
def sf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300 import sfmm
    return sfmm


@pytest.fixture(scope="module")
def h64(sf):
    h = sf.Handle(32, "f64")
    yield h
    h.close()


@pytest.fixture(scope="module")
def h32(sf):
    h = sf.Handle(16, "f32")
    yield h
    h.close()


def _charge_expansions(orc, g, count, P, op):
    """The paper's inputs (config 1 recipe): 32 charges uniform in a unit box
    at the origin, q ~ U[-1,1]; M by P2M about the origin (M2M, M2L), L by P2L
    about a centre at distance 3 (L2L); shifts = unit direction x U[2,4]."""
    pos, q = W.charge_clusters(g, count, 32)
    sh = W.shifts(g, count, 2.0, 4.0)
    if op == "l2l":
        cen = W.unit_directions(g, count) * 3.0
        C = np.stack([orc.p2l(P, pos[i], q[i], cen[i]) for i in range(count)])
    else:
        C = np.stack([orc.p2m(P, pos[i], q[i], np.zeros(3)) for i in range(count)])
    return C, sh


def _config1_inputs(orc, sf, count, P, seed, op):
    """32 charges uniform in a unit box at the origin, q ~ U[-1,1]; multipoles
    by P2M about the origin, locals by P2L about a centre at distance 3.
    Each side forms its own expansions from the same charges."""
    import torch
    g = W.rng(seed)
    pos, q = W.charge_clusters(g, count, 32)
    sh = W.shifts(g, count, 2.0, 4.0)
    far = W.unit_directions(g, count) * 3.0
    centres = np.zeros((count, 3)) if op != "l2l" else far
    C = np.stack([(orc.p2m if op != "l2l" else orc.p2l)(P, pos[i], q[i], centres[i])
                  for i in range(count)])
    # the same expansions formed on the device by the library's own P2M / P2L
    h = sf.Handle(P, "f64")
    dev = "cuda"
    pts = torch.tensor(pos.reshape(-1, 3), device=dev)
    qq = torch.tensor(q.reshape(-1), device=dev)
    offs = torch.arange(0, 32 * count + 1, 32, dtype=torch.int64, device=dev)
    cen = torch.tensor(centres, device=dev)
    out = torch.zeros(count, P * (P + 1), dtype=torch.float64, device=dev)
    (sf.p2m_boxes if op != "l2l" else sf.p2l_boxes)(h, P, pts, qq, offs, cen, out, count)
    torch.cuda.synchronize()
    Cg = out.cpu().numpy()
    h.close()
    return C, Cg, sh


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
def test_config1_p6_4096(sf, orc, h64, op):
    """plain FP64, P = 6: 4096 translations of each kind from P2M/P2L of 32
    charges, shift = random unit direction x U[2,4]."""
    P, count = 6, 4096
    C, Cg, sh = _config1_inputs(orc, sf, count, P, 1, op)
    kind_in = "L" if op == "l2l" else "M"
    U.check_rows(Cg, C, P, kind_in, TOL["f64"], what="device P2M / P2L")
    got = U.run_batch(sf, h64, op, Cg, sh, P, P, "f64")
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, want, P, U.out_kind(op), TOL["f64"], what=op)


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("p_in,p_out", [(1, 1), (1, 4), (4, 1), (2, 2), (5, 8), (8, 5),
                                        (10, 10), (13, 7)])
def test_mixed_orders(sf, orc, h64, op, p_in, p_out):
    g = W.rng(1000 + 17 * p_in + p_out)
    count = 77
    C = W.random_solids(g, count, p_in)
    sh = W.shifts(g, count, 2.0, 4.0)
    got = U.run_batch(sf, h64, op, C, sh, p_in, p_out, "f64")
    want, _ = orc.batch(op, p_in, p_out, C, sh)
    U.check_rows(got, want, p_out, U.out_kind(op), TOL["f64"], what=f"{op} {p_in}->{p_out}")


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("P", [16, 20, 27, 32])
def test_high_orders(sf, orc, h64, op, P):
    """M2M and L2L on random solids; M2L on the expansions of charge
    clusters.  Random solids with row decay 0.4^n are not the multipole of
    any charge distribution in the unit box (their weighted top row exceeds
    the monopole by 1e12 and more): their M2L output is a cancellation of
    terms ~1e7 larger than itself, so two exact-in-FP64 evaluations (the
    oracle's naive sum and the rotation path) differ by up to 4e-9 per
    expansion at P = 32, whereas on charge expansions they agree to ~1e-15."""
    g = W.rng(2000 + P)
    count = 40
    if op == "m2l":
        C, sh = _charge_expansions(orc, g, count, P, op)
    else:
        C = W.random_solids(g, count, P, decay=0.4)
        sh = W.shifts(g, count, 2.0, 4.0)
    got = U.run_batch(sf, h64, op, C, sh, P, P, "f64")
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, want, P, U.out_kind(op), TOL["f64"], a=U.out_radius(op, sh),
                 what=f"{op} P={P}")


@pytest.mark.parametrize("P", [7, 10, 12])
@pytest.mark.parametrize("count", [1, 31, 33, 257])
def test_ragged_counts(sf, orc, h64, count, P):
    g = W.rng(3000 + count)
    C = W.random_solids(g, count, P)
    sh = W.shifts(g, count)
    got = U.run_batch(sf, h64, "m2l", C, sh, P, P, "f64")
    want, _ = orc.batch("m2l", P, P, C, sh)
    U.check_rows(got, want, P, "L", TOL["f64"], what=f"m2l count={count}")


@pytest.mark.parametrize("policy", ["shared", "global"])
@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("P", [3, 8, 11])
def test_generic_kernels_at_unrolled_orders(sf, orc, dtype, op, P, policy):
    """The generic batch kernels at equal orders <= 12, where AUTO takes the
    unrolled ones (reached by sfmm_set_policy, as the autotuner does): each
    expansion against the oracle on charge-cluster inputs, 70 translations."""
    g = W.rng(5700 + 10 * P + len(op))
    C, sh = _charge_expansions(orc, g, 70, P, op)
    if dtype == "f32":
        C, sh = (a.astype(np.float32).astype(np.float64) for a in (C, sh))
    h = sf.Handle(P, dtype)
    sf.set_policy(h, op, P, P, policy)
    got = U.run_batch(sf, h, op, C, sh, P, P, dtype)
    h.close()
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, want, P, U.out_kind(op), TOL[dtype], a=U.out_radius(op, sh),
                 what=f"{dtype} {op} P={P} {policy}")


def test_count_zero_is_noop(sf, h64):
    sf.m2l_batch(h64, 0, 0, 0, 4, 4, 0)


@pytest.mark.parametrize("P", [9, 10, 12])
@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
def test_special_shifts(sf, orc, h64, op, P):
    """Shifts along +z and -z (rho = 0, cos(alpha) = 1 by the special case of
    Sec. 3.4 step 1), nearly axial shifts, and axis-aligned shifts."""
    sh = np.array([[0, 0, 3.0], [0, 0, -2.5], [1e-170, 0, 3.0], [0, 1e-9, -2.2],
                   [3.0, 0, 0], [0, -2.4, 0], [2.0, 2.0, 0], [-1.5, 0, 1.5]])
    g = W.rng(4000)
    C = W.random_solids(g, len(sh), P)
    got = U.run_batch(sf, h64, op, C, sh, P, P, "f64")
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, want, P, U.out_kind(op), TOL["f64"], what=f"{op} special shifts")


@pytest.mark.parametrize("op", ["m2m", "l2l"])
def test_zero_shift_is_identity(sf, h64, op):
    P = 6
    g = W.rng(4100)
    C = W.random_solids(g, 5, P)
    got = U.run_batch(sf, h64, op, C, np.zeros((5, 3)), P, P, "f64")
    assert np.array_equal(got, C)
    got = U.run_batch(sf, h64, op, C, np.zeros((5, 3)), P, P + 2, "f64")
    assert np.array_equal(got[:, :P * (P + 1)], C) and not got[:, P * (P + 1):].any()


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
def test_accumulate(sf, orc, h64, op):
    P = 8
    g = W.rng(4200)
    C = W.random_solids(g, 50, P)
    sh = W.shifts(g, 50)
    init = W.random_solids(g, 50, P)
    got = U.run_batch(sf, h64, op, C, sh, P, P, "f64", accumulate=True, init=init)
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, init + want, P, U.out_kind(op), TOL["f64"], what=f"{op} accumulate")


def test_result_independent_of_batch(sf, h64):
    """Each translation gives bitwise the same result alone and inside a mix."""
    P = 8
    g = W.rng(4300)
    C = W.random_solids(g, 300, P)
    sh = W.shifts(g, 300)
    full = U.run_batch(sf, h64, "m2l", C, sh, P, P, "f64")
    for i in (0, 123, 299):
        one = U.run_batch(sf, h64, "m2l", C[i:i + 1], sh[i:i + 1], P, P, "f64")
        assert np.array_equal(one[0], full[i])


@pytest.fixture(scope="module")
def h32_30(sf):
    h = sf.Handle(30, "f32")
    yield h
    h.close()


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("P", [6, 12, 16, 20, 24, 30])
def test_fp32(sf, orc, h32_30, op, P):
    """FP32 rotation path at every order of the paper's workloads, each
    expansion within 1e-5 of the FP64 oracle applied to the same FP32-rounded
    inputs (P = 6, 12: unrolled kernels; above: generic kernels)."""
    g = W.rng(5000 + P)
    count = 200 if P <= 20 else 96
    C, sh = _charge_expansions(orc, g, count, P, op)
    C32, sh32 = C.astype(np.float32), sh.astype(np.float32)
    got = U.run_batch(sf, h32_30, op, C32, sh32, P, P, "f32")
    want, _ = orc.batch(op, P, P, C32.astype(np.float64), sh32.astype(np.float64))
    U.check_rows(got, want, P, U.out_kind(op), TOL["f32"], a=U.out_radius(op, sh32),
                 what=f"fp32 {op} P={P}")


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 7, 9, 11])
def test_unrolled_batch_orders(sf, orc, h64, h32_30, dtype, op, P):
    """Batch calls at the low and odd orders with unrolled kernels (AUTO takes
    them), on the expansions of charge clusters in both precisions, each
    expansion within the tolerance of the FP64 oracle applied to the same
    (for FP32, FP32-rounded) inputs; 100 translations (a ragged last warp)."""
    g = W.rng(5500 + 10 * P + len(op))
    C, sh = _charge_expansions(orc, g, 100, P, op)
    h = h64 if dtype == "f64" else h32_30
    if dtype == "f32":
        C, sh = (a.astype(np.float32).astype(np.float64) for a in (C, sh))
    got = U.run_batch(sf, h, op, C, sh, P, P, dtype)
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, want, P, U.out_kind(op), TOL[dtype], a=U.out_radius(op, sh),
                 what=f"{dtype} {op} P={P}")


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("p_in,p_out", [(30, 27), (24, 30), (7, 18)])
def test_fp32_mixed_orders(sf, orc, h32_30, op, p_in, p_out):
    g = W.rng(5100 + p_in + 31 * p_out)
    C, sh = _charge_expansions(orc, g, 64, p_in, op)
    C32, sh32 = C.astype(np.float32), sh.astype(np.float32)
    got = U.run_batch(sf, h32_30, op, C32, sh32, p_in, p_out, "f32")
    want, _ = orc.batch(op, p_in, p_out, C32.astype(np.float64), sh32.astype(np.float64))
    U.check_rows(got, want, p_out, U.out_kind(op), TOL["f32"], a=U.out_radius(op, sh32),
                 what=f"fp32 {op} {p_in}->{p_out}")


def _run_lists(sf, orc, h, op, P_in, P_out, accumulate, seed, dtype="f64", maxlen=40, nt=70):
    """Target-major lists of lengths 0..maxlen; FP64 runs use random solids,
    FP32 runs the paper's inputs (expansions of charge clusters, the form whose
    FP32 rounding the 1e-5 tolerance is stated for)."""
    import torch
    g = W.rng(seed)
    lens = g.integers(0, maxlen + 1, size=nt)
    lens[3] = 0
    offs = np.zeros(nt + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    nnz = int(offs[-1])
    nsrc = 90
    if dtype == "f32":
        S, _ = _charge_expansions(orc, g, nsrc, P_in, op)
    else:
        S = W.random_solids(g, nsrc, P_in)
    src_idx = g.integers(0, nsrc, size=nnz)
    sh = W.shifts(g, nnz)
    init = W.random_solids(g, nt, P_out)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        S, sh, init = (a.astype(np.float32).astype(np.float64) for a in (S, sh, init))
    dev = "cuda"
    dS = torch.tensor(S, device=dev, dtype=tdt)
    dO = torch.tensor(init, device=dev, dtype=tdt)
    psrc = sf.pointer_array(dS, P_in * (P_in + 1), torch.tensor(src_idx))
    pout = sf.pointer_array(dO, P_out * (P_out + 1), torch.arange(nt))
    sf.translate_lists(h, op, psrc, torch.tensor(sh, device=dev, dtype=tdt),
                       torch.tensor(offs, device=dev), pout, P_in, P_out, nt,
                       accumulate=accumulate)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    got = dO.double().cpu().numpy()
    each, _ = orc.batch(op, P_in, P_out, S[src_idx], sh)
    want = init.copy() if accumulate else np.zeros_like(init)
    for t in range(nt):
        for j in range(offs[t], offs[t + 1]):
            want[t] += each[j]
    return U.rel_err_rows(got, want, P_out, U.out_kind(op))


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("accumulate", [False, True])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
def test_lists_fixed_orders(sf, orc, h64, op, accumulate, P):
    """Lists at the orders with fully unrolled kernels (groups of 8 or 32 lanes
    per target, lengths 0..70 so that targets take several rounds)."""
    err = _run_lists(sf, orc, h64, op, P, P, accumulate, 6100 + P, maxlen=70)
    assert err.max() <= TOL["f64"], (int(err.argmax()), err.max())


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
def test_lists_fixed_orders_fp32(sf, orc, h32, op, P):
    err = _run_lists(sf, orc, h32, op, P, P, False, 6200 + P, dtype="f32")
    assert err.max() <= TOL["f32"], (int(err.argmax()), err.max())


@pytest.mark.parametrize("dtype", ["f64", "f32"])
@pytest.mark.parametrize("P", [1, 2, 3, 4, 5, 6, 7, 8, 9, 10, 11, 12])
def test_lists_m2l_special_shifts(sf, orc, h64, h32, dtype, P):
    """The interaction-list M2L kernel (paired row and column steps, basis
    factors folded into its swap tables) on shifts along +z and -z (rho = 0,
    Sec. 3.4 step 1), nearly axial and axis-aligned shifts, each target
    summing a list of all of them."""
    import torch
    h = h64 if dtype == "f64" else h32
    tdt = torch.float64 if dtype == "f64" else torch.float32
    base = np.array([[0, 0, 3.0], [0, 0, -2.5], [1e-170, 0, 3.0], [0, 1e-9, -2.2],
                     [3.0, 0, 0], [0, -2.4, 0], [2.0, 2.0, 0], [-1.5, 0, 1.5]])
    if dtype == "f32":
        base[2, 0] = 1e-30                          # representable in FP32
    g = W.rng(6300 + P)
    nt, per = 40, len(base)
    if dtype == "f32":
        S, _ = _charge_expansions(orc, g, nt * per, P, "m2l")
    else:
        S = W.random_solids(g, nt * per, P)
    sh = np.tile(base, (nt, 1))
    if dtype == "f32":
        S, sh = (a.astype(np.float32).astype(np.float64) for a in (S, sh))
    offs = np.arange(0, nt * per + 1, per, dtype=np.int64)
    dS = torch.tensor(S, device="cuda", dtype=tdt)
    dO = torch.zeros(nt, P * (P + 1), device="cuda", dtype=tdt)
    psrc = sf.pointer_array(dS, P * (P + 1), torch.arange(nt * per))
    pout = sf.pointer_array(dO, P * (P + 1), torch.arange(nt))
    sf.translate_lists(h, "m2l", psrc, torch.tensor(sh, device="cuda", dtype=tdt),
                       torch.tensor(offs, device="cuda"), pout, P, P, nt)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    got = dO.double().cpu().numpy()
    each, _ = orc.batch("m2l", P, P, S, sh)
    want = each.reshape(nt, per, -1).sum(axis=1)
    U.check_rows(got, want, P, "L", TOL[dtype], what=f"{dtype} lists special shifts")


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("accumulate", [False, True])
def test_lists(sf, orc, h64, op, accumulate):
    """Target-major CSR lists with lengths 0..40 (sum in list order)."""
    import torch
    P_in, P_out = 7, 6
    g = W.rng(6000 + accumulate)
    nt = 70
    lens = g.integers(0, 41, size=nt)
    lens[3] = 0
    offs = np.zeros(nt + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    nnz = int(offs[-1])
    nsrc = 90
    S = W.random_solids(g, nsrc, P_in)
    src_idx = g.integers(0, nsrc, size=nnz)
    sh = W.shifts(g, nnz)
    init = W.random_solids(g, nt, P_out)
    dev = "cuda"
    dS = torch.tensor(S, device=dev)
    dO = torch.tensor(init, device=dev)
    psrc = sf.pointer_array(dS, P_in * (P_in + 1), torch.tensor(src_idx))
    pout = sf.pointer_array(dO, P_out * (P_out + 1), torch.arange(nt))
    sf.translate_lists(h64, op, psrc, torch.tensor(sh, device=dev),
                       torch.tensor(offs, device=dev), pout, P_in, P_out, nt,
                       accumulate=accumulate)
    torch.cuda.synchronize()
    assert h64.sync_status() == 0
    got = dO.cpu().numpy()
    each, _ = orc.batch(op, P_in, P_out, S[src_idx], sh)
    want = init.copy() if accumulate else np.zeros_like(init)
    for t in range(nt):
        for j in range(offs[t], offs[t + 1]):
            want[t] += each[j]
    U.check_rows(got, want, P_out, U.out_kind(op), TOL["f64"], what=f"{op} lists")


@pytest.mark.parametrize("P", [4, 6])
def test_device_status_reports_null_pointer(sf, h64, P):
    import torch
    cin = torch.zeros(2, P * (P + 1), dtype=torch.float64, device="cuda")
    cout = torch.zeros_like(cin)
    pin = sf.pointer_array(cin, P * (P + 1), torch.arange(2))
    pin[1] = 0
    pout = sf.pointer_array(cout, P * (P + 1), torch.arange(2))
    shift = torch.ones(2, 3, dtype=torch.float64, device="cuda")
    sf.m2l_batch(h64, pin, pout, shift, P, P, 2)
    torch.cuda.synchronize()
    assert h64.sync_status() == 1
    assert h64.sync_status() == 0          # cleared by the read


def test_host_errors(sf, h64):
    with pytest.raises(sf.SfmmError) as e:
        sf.m2l_batch(h64, 1, 1, 1, 0, 4, 1)
    assert e.value.code == 2
    with pytest.raises(sf.SfmmError) as e:
        sf.m2l_batch(h64, 1, 1, 1, 4, 33, 1)
    assert e.value.code == 2
    with pytest.raises(sf.SfmmError) as e:
        sf.m2l_batch(h64, 0, 0, 0, 4, 4, 5)
    assert e.value.code == 1


@pytest.mark.parametrize("lanes", [1, 2, 8, 32])
def test_lists_multi_lanes_per_target(sf, orc, h64, lanes):
    """Two mixed-order M2L classes and one M2M class in one launch, lists of
    0..70 sources, each class spread over `lanes` lanes per target (1: one
    thread walks the list); every variant agrees with the oracle's sums, and
    a second run gives bitwise the same result."""
    import torch
    g = W.rng(6100 + lanes)
    spec = [("m2l", 9, 7, 40), ("m2l", 5, 11, 33), ("m2m", 8, 8, 21)]
    nt = sum(c[3] for c in spec)
    lens = g.integers(0, 71, size=nt)
    lens[5] = 0
    offs = np.zeros(nt + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    pmax = 11
    S = pmax * (pmax + 1)
    nsrc = 64
    src_solids = {p: W.random_solids(g, nsrc, p) for p in (5, 8, 9)}
    dS = {p: torch.tensor(v, device="cuda") for p, v in src_solids.items()}
    dO = torch.zeros(nt, S, dtype=torch.float64, device="cuda")
    ptrs = torch.zeros(int(offs[-1]), dtype=torch.int64)
    shifts = W.shifts(g, int(offs[-1]))
    classes, t0, want, picks = [], 0, [], []
    for op, pi, po, n in spec:
        for t in range(t0, t0 + n):
            idx = g.integers(0, nsrc, size=lens[t])
            picks.append(idx)
            ptrs[offs[t]:offs[t + 1]] = sf.pointer_array(dS[pi], pi * (pi + 1), torch.tensor(idx)).cpu()
        classes.append((op, pi, po, t0, t0 + n, lanes))
        t0 += n
    pout = torch.tensor([dO.data_ptr() + 8 * S * t for t in range(nt)], dtype=torch.int64, device="cuda")
    args = (ptrs.cuda(), torch.tensor(shifts, device="cuda"), torch.tensor(offs, device="cuda"), pout)
    sf.translate_lists_multi(h64, classes, *args)
    torch.cuda.synchronize()
    assert h64.sync_status() == 0
    first = dO.clone()
    sf.translate_lists_multi(h64, classes, *args)
    torch.cuda.synchronize()
    assert torch.equal(first, dO)
    got = dO.cpu().numpy()
    t = 0
    for op, pi, po, n in spec:
        for _ in range(n):
            w = np.zeros(po * (po + 1))
            for k, j in enumerate(range(offs[t], offs[t + 1])):
                w += orc.translate(op, pi, po, src_solids[pi][picks[t][k]], shifts[j])
            if lens[t] == 0:
                assert not got[t].any(), t          # an empty list gives zeros
            else:
                U.check_rows(got[t, :po * (po + 1)], w, po, U.out_kind(op), TOL["f64"], what=f"{op} target {t}")
            t += 1


def test_lists_multi_rejects_bad_lanes(sf, h64):
    import torch
    z = torch.zeros(2, dtype=torch.int64, device="cuda")
    with pytest.raises(sf.SfmmError):
        sf.translate_lists_multi(h64, [("m2l", 4, 4, 0, 1, 3)], z, z, z, z)


def test_lists_on_two_streams_share_one_handle(sf, h64):
    """Group-lists launches of one handle on two streams use its one scratch
    and chunk counter; the handle orders them, so each result is bitwise the
    one computed alone."""
    import torch
    g = W.rng(6200)
    P = 14
    S = P * (P + 1)
    res = []
    cases = []
    for k in range(2):
        nt = 300
        lens = g.integers(1, 60, size=nt)
        offs = np.zeros(nt + 1, np.int64)
        np.cumsum(lens, out=offs[1:])
        C = torch.tensor(W.random_solids(g, 128, P), device="cuda")
        src = sf.pointer_array(C, S, torch.tensor(g.integers(0, 128, size=int(offs[-1]))))
        sh = torch.tensor(W.shifts(g, int(offs[-1])), device="cuda")
        cases.append((C, src, sh, torch.tensor(offs, device="cuda"), nt))
    for C, src, sh, offs, nt in cases:                  # alone, one after the other
        out = torch.zeros(nt, S, dtype=torch.float64, device="cuda")
        sf.translate_lists(h64, "m2l", src, sh, offs, sf.pointer_array(out, S, torch.arange(nt)), P, P, nt)
        torch.cuda.synchronize()
        res.append(out)
    streams = [torch.cuda.Stream() for _ in cases]
    outs = [torch.zeros(nt, S, dtype=torch.float64, device="cuda") for *_, nt in cases]
    ptrs = [sf.pointer_array(o, S, torch.arange(o.shape[0])) for o in outs]
    torch.cuda.synchronize()                            # inputs ready before either stream starts
    for (C, src, sh, offs, nt), s, po in zip(cases, streams, ptrs):
        sf.translate_lists(h64, "m2l", src, sh, offs, po, P, P, nt, stream=s)
    torch.cuda.synchronize()
    assert h64.sync_status() == 0
    for a, b in zip(outs, res):
        assert torch.equal(a, b)


@pytest.mark.parametrize("accumulate", [False, True])
@pytest.mark.parametrize("dtype,P", [("f64", 6), ("f64", 10), ("f64", 12), ("f32", 10)])
def test_lists_m2l_packed_rounds(sf, orc, h64, h32, accumulate, dtype, P):
    """M2L lists with more targets than warps (every warp takes several lists
    in turn), lengths 0..80 with many just above and below multiples of 32, so
    that the kernels pack the next list's first sources into the last round of
    a list (FP64 up to order 10: lane sums in tensor memory, handed over around
    that round; FP64 order 12 and FP32: the round's sum split between the two
    targets).  Every target within the dtype's tolerance of the oracle's sum
    of its list, and the same bits on a second run."""
    import torch
    g = W.rng(7700 + P + (100 if dtype == "f32" else 0))
    nt = 5000
    lens = g.choice([0, 1, 5, 31, 32, 33, 37, 40, 63, 64, 65, 80], size=nt)
    offs = np.zeros(nt + 1, np.int64)
    np.cumsum(lens, out=offs[1:])
    nnz = int(offs[-1])
    nsrc = 64
    if dtype == "f32":
        S, _ = _charge_expansions(orc, g, nsrc, P, "m2l")
    else:
        S = W.random_solids(g, nsrc, P)
    src_idx = g.integers(0, nsrc, size=nnz)
    sh = W.shifts(g, nnz)
    init = W.random_solids(g, nt, P)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        S, sh, init = (a.astype(np.float32).astype(np.float64) for a in (S, sh, init))
    h = h64 if dtype == "f64" else h32
    dS = torch.tensor(S, device="cuda", dtype=tdt)
    psrc = sf.pointer_array(dS, P * (P + 1), torch.tensor(src_idx))
    dsh = torch.tensor(sh, device="cuda", dtype=tdt)
    doffs = torch.tensor(offs, device="cuda")
    runs = []
    for _ in range(2):
        dO = torch.tensor(init, device="cuda", dtype=tdt)
        pout = sf.pointer_array(dO, P * (P + 1), torch.arange(nt))
        sf.translate_lists(h, "m2l", psrc, dsh, doffs, pout, P, P, nt, accumulate=accumulate)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        runs.append(dO.double().cpu().numpy())
    assert np.array_equal(runs[0], runs[1])
    pick = np.sort(g.choice(nt, size=96, replace=False))
    pick[:4] = [0, 1, nt - 2, nt - 1]
    pick = np.unique(pick)
    want = init[pick].copy() if accumulate else np.zeros((len(pick), P * (P + 1)))
    for i, t in enumerate(pick):
        a, b = offs[t], offs[t + 1]
        if b > a:
            each, _ = orc.batch("m2l", P, P, S[src_idx[a:b]], sh[a:b])
            want[i] += each.sum(axis=0)
    U.check_rows(runs[0][pick], want, P, "L", TOL[dtype], what=f"packed lists {dtype} P={P}")


@pytest.fixture(scope="module")
def h64_max(sf):
    h = sf.Handle(64, "f64")
    yield h
    h.close()


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("P", [48, 64])
def test_largest_orders(sf, orc, h64_max, op, P):
    """The largest orders an FP64 handle takes (P_max = 64): the generic kernel
    with the rotated solid in the global scratch and the powers regenerated
    per row (three-term recurrence up to m = 63).  M2M / L2L on random solids,
    M2L on charge expansions (see test_high_orders); every expansion within
    1e-12 of the oracle."""
    g = W.rng(2100 + P)
    count = 6
    if op == "m2l":
        C, sh = _charge_expansions(orc, g, count, P, op)
    else:
        C = W.random_solids(g, count, P, decay=0.4)
        sh = W.shifts(g, count, 2.0, 4.0)
    got = U.run_batch(sf, h64_max, op, C, sh, P, P, "f64")
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, want, P, U.out_kind(op), TOL["f64"], a=U.out_radius(op, sh),
                 what=f"{op} P={P}")
