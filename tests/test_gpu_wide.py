"""The warp-cooperative batch kernel (csrc/sfmm_wide.cuh: a warp translates 4
FP32 or 2 FP64 solids together, lanes split by coefficient index) against the
oracle, per expansion, through the C ABI.  FP32 batch calls take it by
default for M2L of orders 16..31 and M2M / L2L of orders 22..31 (the FP32
tests of test_gpu_parity.py at orders 16..30 run through it); the FP64 handle
here selects it with sfmm_set_policy(WIDE) for every order pair.

Tolerances as in test_gpu_parity.py: every expansion within 1e-12 (FP64) and
1e-5 (FP32) in the evaluation-weighted coefficient norm."""
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
def hw64(sf):
    """FP64 handle with the wide kernel selected for every (op, p_in, p_out)
    the tests use."""
    h = sf.Handle(32, "f64")
    for op in ("m2m", "m2l", "l2l"):
        for p_in in range(1, 32):
            for p_out in range(1, 32):
                sf.set_policy(h, op, p_in, p_out, "wide")
    yield h
    h.close()


@pytest.fixture(scope="module")
def h64(sf):
    h = sf.Handle(32, "f64")
    yield h
    h.close()


@pytest.fixture(scope="module")
def h32(sf):
    h = sf.Handle(30, "f32")
    yield h
    h.close()


def _inputs(orc, g, count, P, op):
    """M2L: expansions of 32 charges in a unit box (P2M about the origin);
    M2M and L2L: random solids with row decay 0.4^n (see test_high_orders);
    shifts = unit direction x U[2,4]."""
    if op == "m2l":
        pos, q = W.charge_clusters(g, count, 32)
        C = np.stack([orc.p2m(P, pos[i], q[i], np.zeros(3)) for i in range(count)])
    else:
        C = W.random_solids(g, count, P, decay=0.4)
    return C, W.shifts(g, count, 2.0, 4.0)


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("P", [13, 16, 24, 31])
def test_fp64_orders(sf, orc, hw64, op, P):
    g = W.rng(9000 + P)
    C, sh = _inputs(orc, g, 37, P, op)
    got = U.run_batch(sf, hw64, op, C, sh, P, P, "f64")
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, want, P, U.out_kind(op), TOL["f64"], a=U.out_radius(op, sh),
                 what=f"wide f64 {op} P={P}")


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
@pytest.mark.parametrize("p_in,p_out", [(20, 13), (13, 25), (31, 28), (3, 17)])
def test_fp64_mixed_orders(sf, orc, hw64, op, p_in, p_out):
    g = W.rng(9100 + p_in + 37 * p_out)
    C, sh = _inputs(orc, g, 21, p_in, op)
    got = U.run_batch(sf, hw64, op, C, sh, p_in, p_out, "f64")
    want, _ = orc.batch(op, p_in, p_out, C, sh)
    U.check_rows(got, want, p_out, U.out_kind(op), TOL["f64"], a=U.out_radius(op, sh),
                 what=f"wide f64 {op} {p_in}->{p_out}")


@pytest.mark.parametrize("dtype,count", [("f64", 1), ("f64", 3), ("f64", 129),
                                         ("f32", 1), ("f32", 2), ("f32", 5), ("f32", 258)])
def test_ragged_counts(sf, orc, hw64, h32, dtype, count):
    """Counts that leave the last warp's group of 2 (FP64) or 4 (FP32) solids
    part-filled, and groups spread over more warps than one block holds."""
    P = 17
    g = W.rng(9200 + count)
    C, sh = _inputs(orc, g, count, P, "m2l")
    h = hw64 if dtype == "f64" else h32
    if dtype == "f32":
        C, sh = C.astype(np.float32), sh.astype(np.float32)
    got = U.run_batch(sf, h, "m2l", C, sh, P, P, dtype)
    want, _ = orc.batch("m2l", P, P, np.asarray(C, np.float64), np.asarray(sh, np.float64))
    U.check_rows(got, want, P, "L", TOL[dtype], what=f"wide {dtype} count={count}")


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
def test_special_shifts(sf, orc, hw64, op):
    """Shifts along +z and -z (rho = 0), nearly axial, axis-aligned."""
    P = 14
    sh = np.array([[0, 0, 3.0], [0, 0, -2.5], [1e-170, 0, 3.0], [0, 1e-9, -2.2],
                   [3.0, 0, 0], [0, -2.4, 0], [2.0, 2.0, 0], [-1.5, 0, 1.5]])
    g = W.rng(9300)
    C = W.random_solids(g, len(sh), P, decay=0.4) if op != "m2l" else \
        _inputs(orc, g, len(sh), P, "m2l")[0]
    got = U.run_batch(sf, hw64, op, C, sh, P, P, "f64")
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, want, P, U.out_kind(op), TOL["f64"], a=U.out_radius(op, sh),
                 what=f"wide {op} special shifts")


@pytest.mark.parametrize("op", ["m2m", "l2l"])
@pytest.mark.parametrize("p_out", [13, 15, 18, 24])
def test_zero_shift_is_identity(sf, hw64, h32, op, p_out):
    """M2M / L2L by a zero shift copy the input (truncated or zero-padded),
    bitwise, in a batch that mixes zero and non-zero shifts."""
    P = 15
    g = W.rng(9400 + p_out)
    C = W.random_solids(g, 6, P)
    sh = W.shifts(g, 6, 2.0, 4.0)
    sh[1] = 0.0
    sh[4] = 0.0
    k = min(P, p_out)
    for h, dt in ((hw64, "f64"), (h32, "f32")):
        Cd = C if dt == "f64" else C.astype(np.float32)
        got = U.run_batch(sf, h, op, Cd, sh, P, p_out, dt)
        for i in (1, 4):
            assert np.array_equal(got[i, :k * (k + 1)], np.asarray(Cd, np.float64)[i, :k * (k + 1)])
            assert not got[i, k * (k + 1):].any()


@pytest.mark.parametrize("op", ["m2m", "m2l", "l2l"])
def test_accumulate(sf, orc, hw64, op):
    P = 19
    g = W.rng(9500)
    C, sh = _inputs(orc, g, 23, P, op)
    init = W.random_solids(g, 23, P, decay=0.4)
    got = U.run_batch(sf, hw64, op, C, sh, P, P, "f64", accumulate=True, init=init)
    want, _ = orc.batch(op, P, P, C, sh)
    U.check_rows(got, init + want, P, U.out_kind(op), TOL["f64"], a=U.out_radius(op, sh),
                 what=f"wide {op} accumulate")


def test_null_pointer_sets_status_and_skips(sf, orc, hw64):
    import torch
    P, count = 16, 6
    g = W.rng(9600)
    C, sh = _inputs(orc, g, count, P, "m2l")
    cin = torch.tensor(C, device="cuda")
    cout = torch.full((count, P * (P + 1)), 7.0, dtype=torch.float64, device="cuda")
    pin = sf.pointer_array(cin, P * (P + 1), torch.arange(count))
    pin[2] = 0
    pout = sf.pointer_array(cout, P * (P + 1), torch.arange(count))
    shift = torch.tensor(sh, device="cuda")
    sf.m2l_batch(hw64, pin, pout, shift, P, P, count)
    torch.cuda.synchronize()
    assert hw64.sync_status() == 1
    got = cout.cpu().numpy()
    assert (got[2] == 7.0).all()                   # skipped, untouched
    keep = [0, 1, 3, 4, 5]
    want, _ = orc.batch("m2l", P, P, C[keep], sh[keep])
    U.check_rows(got[keep], want, P, "L", TOL["f64"], what="wide null pointer")


def test_agrees_with_the_per_thread_kernel(sf, orc, hw64, h64):
    """The same inputs through the wide and the per-thread generic kernels."""
    P = 22
    g = W.rng(9700)
    C, sh = _inputs(orc, g, 40, P, "m2l")
    a = U.run_batch(sf, hw64, "m2l", C, sh, P, P, "f64")
    b = U.run_batch(sf, h64, "m2l", C, sh, P, P, "f64")
    U.check_rows(a, b, P, "L", 1e-13, what="wide vs per-thread")


def test_policy_rejects_order_32(sf, hw64):
    with pytest.raises(sf.SfmmError):
        sf.set_policy(hw64, "m2l", 32, 32, "wide")
    with pytest.raises(sf.SfmmError):
        sf.set_policy(hw64, "m2l", 10, 32, "wide")
