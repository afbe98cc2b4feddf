"""Host logic of the adaptive pass: the M2L waves and their classes (CPU only)."""
import numpy as np
import pytest

from paper_2202_02847_gb300 import workloads as W


def test_lanes_for_length():
    from paper_2202_02847_gb300.fmm import lanes_for_length
    got = lanes_for_length([0, 1, 2, 3, 4, 5, 8, 9, 16, 17, 31, 32, 33, 800])
    assert list(got) == [1, 1, 2, 4, 4, 8, 8, 16, 16, 32, 32, 32, 32, 32]


@pytest.fixture(scope="module")
def plan():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300.fmm import AdaptivePass
    pts, q = W.plummer(20000, seed=7)
    tree = W.adaptive_octree(pts, leaf_size=16)
    P = W.order_by_level(tree, lo=4, span=12)
    pairs = W.dual_tree_m2l(tree, 0.5)
    return tree, P, pairs, AdaptivePass(tree, P, None, device="cpu", pairs=pairs)


def test_waves_hold_every_pair_once(plan):
    tree, P, (src, tgt), ap = plan
    got = sorted((int(t), int(s)) for d in ap.waves
                 for t, s in zip(d["host"]["tgt"], d["host"]["src"]))
    assert got == sorted(zip(tgt.tolist(), src.tolist()))


def test_classes_partition_rows_with_uniform_orders_and_lanes(plan):
    from paper_2202_02847_gb300.fmm import lanes_for_length, translation_cost
    tree, P, _, ap = plan
    P = np.asarray(P)
    for d in ap.waves:
        h = d["host"]
        offs, row_tgt = h["offs"], h["row_tgt"]
        assert len(set(row_tgt.tolist())) == len(row_tgt)        # a target once per wave
        lens = np.diff(offs)
        covered = np.zeros(len(row_tgt), int)
        cost = []
        for op, pi, po, tb, te, lanes in d["classes"]:
            assert op == "m2l" and te > tb
            covered[tb:te] += 1
            cost.append(-(-lens[tb] // lanes) * translation_cost(pi, po))
            for r in range(tb, te):
                srcs = h["src"][offs[r]:offs[r + 1]]
                assert np.all(P[srcs] == pi) and P[row_tgt[r]] == po
            assert np.all(np.diff(lens[tb:te]) <= 0)              # longest lists first
            assert np.all(lanes_for_length(lens[tb:te]) == lanes)
        assert np.all(covered == 1)                               # classes partition the rows
        assert cost == sorted(cost, reverse=True)                 # costliest first chunk first
        assert len(d["classes"]) <= 256


@pytest.mark.parametrize("min_lanes", [1, 2, 4, 8, 16, 32])
def test_coarsened_lane_classes_still_partition_rows(plan, min_lanes):
    """coarsen_lanes (used when a one-launch pass would exceed the launch's
    class limit): the merged classes still partition every wave's rows, keep
    one order pair each, give every list at least the lanes its length needs
    and at least min_lanes, and never add classes."""
    from paper_2202_02847_gb300.fmm import coarsen_lanes, lanes_for_length
    tree, P, _, ap = plan
    P = np.asarray(P)
    for d in ap.waves:
        h = d["host"]
        lens = np.diff(h["offs"])
        cc = coarsen_lanes(d["classes"], min_lanes)
        assert len(cc) <= len(d["classes"])
        covered = np.zeros(len(lens), int)
        for op, pi, po, tb, te, lanes in cc:
            covered[tb:te] += 1
            assert lanes >= min_lanes and np.all(lanes_for_length(lens[tb:te]) <= lanes)
            for r in range(tb, te):
                assert np.all(P[h["src"][h["offs"][r]:h["offs"][r + 1]]] == pi)
                assert P[h["row_tgt"][r]] == po
        assert np.all(covered == 1)
    if min_lanes == 1:
        assert all(coarsen_lanes(d["classes"], 1) == d["classes"] for d in ap.waves)


def test_pass_plan_fits_the_class_limit():
    """A tree whose waves hold more lane classes than one pass launch takes
    (262,144-point Plummer sphere: 389) gets a plan within the limit."""
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300 import sfmm
    from paper_2202_02847_gb300.fmm import AdaptivePass
    pts, q = W.plummer(262144, seed=4)
    tree = W.adaptive_octree(pts, leaf_size=64)
    P = W.order_by_level(tree, lo=4, span=20)
    ap = AdaptivePass(tree, P, None, device="cpu")
    assert sum(len(d["classes"]) for d in ap.waves) + len(ap.m2m) + len(ap.l2l) > sfmm.MAX_PASS_CLASSES
    cls, _, phases = ap.pass_plan()
    assert len(cls) <= sfmm.MAX_PASS_CLASSES and phases <= 64
    assert sum(c.n_targets for c in cls if c.op == sfmm.OPS["m2l"]) == \
        sum(d["n"] for d in ap.waves)
