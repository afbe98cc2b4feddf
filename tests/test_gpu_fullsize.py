"""Full-size workloads in the launch configuration the benchmark times, checked
on sampled outputs against the oracle (which forms every source multipole
directly from the particles in the source box: P2M of a box's particles equals
the M2M-combined multipoles of its children at the same order).

* Uniform octree, level 5 (32^3 leaves, 2^20 uniform points, q ~ U[-1, 1],
  seed 2), P = 10, FP64: the upward pass and the pass's single M2L lists launch
  (levels 2-5) as the benchmark runs them; 10 sampled level-5 targets and 2
  level-3 targets.  A second run of the same launches gives bitwise the same
  locals (the lists kernels add in a fixed order).
* The same tree at P = 16 through the tensor-core grid M2L of level 5
  (two-part FP16 split, float-float target sums): 8 sampled targets at the FP32-class
  tolerance.
* The largest serving request (10^6 M2L at order 30, FP64 and FP32).
* The mixed-order pass on the 2 M-point Plummer sphere: 3 sampled targets."""
import numpy as np
import pytest

from paper_2202_02847_gb300 import workloads as W
import gpu_util as U

pytestmark = pytest.mark.gpu

NPOINTS = 1 << 20
DEPTH = 5


@pytest.fixture(scope="module")
def tree():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return W.uniform_octree(DEPTH, NPOINTS, seed=2)


@pytest.fixture(scope="module")
def sf():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300 import sfmm
    return sfmm


def _box_points(tree, level):
    """Point indices of every box of a level (boxes of level l contain the
    leaves whose index, read in octal digits, starts with the box's)."""
    ijk = np.floor(tree.points * (1 << level)).astype(np.int64).clip(0, (1 << level) - 1)
    box = W.box_index(ijk[:, 0], ijk[:, 1], ijk[:, 2], 1 << level)
    order = np.argsort(box, kind="stable")
    offs = np.concatenate([[0], np.cumsum(np.bincount(box, minlength=8 ** level))])
    return order, offs


def _oracle_m2l(orc, tree, level, t, P, cache):
    lv = tree.levels[level]
    if level not in cache:
        cache[level] = _box_points(tree, level)
    order, offs = cache[level]
    want = np.zeros(P * (P + 1))
    for j in range(lv.m2l_offsets[t], lv.m2l_offsets[t + 1]):
        s = lv.m2l_sources[j]
        sel = order[offs[s]:offs[s + 1]]
        Ms = orc.p2m(P, tree.points[sel], tree.charges[sel], lv.centres[s])
        want += orc.translate("m2l", P, P, Ms, lv.m2l_shift[j])
    return want


def test_octree_level5_p10_sampled_against_oracle(sf, orc, tree):
    import torch
    from paper_2202_02847_gb300.fmm import UniformPass
    P = 10
    h = sf.Handle(P, "f64")
    fp = UniformPass(tree, P, h)
    fp.p2m_leaves(tree.points, tree.charges, tree.leaf_of_point)
    fp.upward()
    fp.m2l_all()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    L1 = fp.L.clone()
    fp.upward()
    fp.m2l_all()
    torch.cuda.synchronize()
    assert torch.equal(fp.L, L1)
    L = L1.cpu().numpy()
    g = W.rng(77)
    cache = {}
    for level, k in ((5, 10), (3, 2)):
        for t in g.choice(8 ** level, size=k, replace=False):
            want = _oracle_m2l(orc, tree, level, t, P, cache)
            got = L[int(fp.level_base[level]) + t]
            U.check_rows(got, want, P, "L", 1e-12, a=U.box_radius(tree.levels[level].h),
                         what=f"level {level} target {t}")
    h.close()


def test_grid_level5_p16_sampled_against_oracle(sf, orc, tree):
    import torch
    P = 16
    h = sf.Handle(P, "f64")
    lv = tree.levels[DEPTH]
    nb = 8 ** DEPTH
    order = np.argsort(tree.leaf_of_point, kind="stable")
    offs = np.concatenate([[0], np.cumsum(np.bincount(tree.leaf_of_point, minlength=nb))])
    M = torch.zeros(nb, P * (P + 1), dtype=torch.float64, device="cuda")
    sf.p2m_boxes(h, P, torch.tensor(tree.points[order], device="cuda"),
                 torch.tensor(tree.charges[order], device="cuda"), torch.tensor(offs, device="cuda"),
                 torch.tensor(lv.centres, device="cuda"), M, nb)
    grid = sf.Grid(h, P, 1 << DEPTH)
    L = torch.zeros_like(M)
    grid.m2l(lv.h, M, L)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    got = L.cpu().numpy()
    g = W.rng(78)
    cache = {}
    picks = g.choice(nb, size=8, replace=False)
    want = np.stack([_oracle_m2l(orc, tree, DEPTH, t, P, cache) for t in picks])
    U.check_rows(got[picks], want, P, "L", 1e-5, a=U.box_radius(lv.h), what="grid level 5")
    grid.close()
    h.close()


@pytest.mark.parametrize("dtype,P", [("f64", 30), ("f32", 30)])
def test_batch_m2l_one_million_sampled_against_oracle(sf, orc, dtype, P):
    """The largest request of the serving mix: 10^6 M2L of the highest order,
    in FP64 and in FP32, from a resident pool of 4,096 P2M solids and 2^16
    shifts."""
    import torch
    g = W.rng(500 + P)
    n, pool = 1_000_000, 4096
    S = P * (P + 1)
    pos, q = W.charge_clusters(g, pool, 32)
    C = np.stack([orc.p2m(P, pos[i], q[i], np.zeros(3)) for i in range(pool)])
    sh = W.shifts(g, 1 << 16, 2.0, 4.0)
    tdt = torch.float64 if dtype == "f64" else torch.float32
    if dtype == "f32":
        C, sh = C.astype(np.float32).astype(np.float64), sh.astype(np.float32).astype(np.float64)
    h = sf.Handle(P, dtype)
    dC = torch.tensor(C, dtype=tdt, device="cuda")
    dsh = torch.tensor(sh, dtype=tdt, device="cuda")
    out = torch.empty(n, S, dtype=tdt, device="cuda")
    idx = torch.arange(n)
    pin = sf.pointer_array(dC, S, idx % pool)
    pout = sf.pointer_array(out, S, idx)
    shifts = dsh[torch.arange(n, device="cuda") % (1 << 16)].contiguous()
    sf.m2l_batch(h, pin, pout, shifts, P, P, n)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    picks = np.sort(g.choice(n, size=6, replace=False))
    got = out[torch.tensor(picks, device="cuda")].double().cpu().numpy()
    want, _ = orc.batch("m2l", P, P, C[picks % pool], sh[picks % (1 << 16)])
    tol = 1e-12 if dtype == "f64" else 1e-5
    U.check_rows(got, want, P, "L", tol, what=f"10^6 M2L {dtype} P={P}")
    h.close()


def test_adaptive_plummer_2m_sampled_against_oracle(sf, orc):
    """The mixed-order pass on the 2 M-point Plummer sphere (orders 4-24 rising
    with the level, dual-tree M2L): upward pass and all M2L waves as fused
    multi-class launches with the default policies; 3 sampled targets of the
    largest wave, summed over every wave, against the oracle (each source's
    multipole by P2M of its own points at its own order)."""
    import torch
    from paper_2202_02847_gb300.fmm import AdaptivePass
    pts, q = W.plummer(1 << 21, seed=4)
    tree = W.adaptive_octree(pts, leaf_size=64)
    P_node = np.asarray(W.order_by_level(tree, lo=4, span=20))
    h = sf.Handle(int(P_node.max()), "f64")
    ap = AdaptivePass(tree, P_node, h)
    ap.p2m_leaves(pts, q)
    ap.upward()
    ap.L.zero_()
    ap.m2l_all()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    L = ap.L.cpu().numpy()
    big = max(range(len(ap.waves)), key=lambda w: len(ap.waves[w]["host"]["src"]))
    g = W.rng(79)
    rows = ap.waves[big]["host"]
    lens = np.diff(rows["offs"])
    cand = rows["row_tgt"][lens >= 32]
    Mcache = {}
    for t in g.choice(cand, size=3, replace=False):
        Po = int(P_node[t])
        want = np.zeros(Po * (Po + 1))
        for d in ap.waves:
            hst = d["host"]
            for r in np.nonzero(hst["row_tgt"] == t)[0]:
                for j in range(hst["offs"][r], hst["offs"][r + 1]):
                    s = int(hst["src"][j])
                    if s not in Mcache:
                        sel = tree.order[tree.pt_begin[s]:tree.pt_end[s]]
                        Mcache[s] = orc.p2m(int(P_node[s]), pts[sel], q[sel], tree.centre[s])
                    want += orc.translate("m2l", int(P_node[s]), Po, Mcache[s], tree.centre[t] - tree.centre[s])
        got = L[ap.off[t]:ap.off[t + 1]]
        U.check_rows(got, want, Po, "L", 1e-12, a=float(np.sqrt(3.0) * tree.half[t]),
                     what=f"target {t}")
    # the upward pass and the M2L waves as one persistent launch: every target
    # agrees with the separate launches checked above
    ap.L.zero_()
    ap.run_pass(("m2m", "m2l"))
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    L1 = ap.L.cpu().numpy()
    for P in np.unique(P_node):
        nodes = np.nonzero(P_node == P)[0]
        idx = ap.off[nodes][:, None] + np.arange(int(P) * (int(P) + 1))[None, :]
        U.check_rows(L1[idx], L[idx], int(P), "L", 1e-12, a=np.sqrt(3.0) * tree.half[nodes],
                     what=f"one-launch pass, order {P}")
    h.close()
