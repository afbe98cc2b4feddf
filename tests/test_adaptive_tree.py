"""Host logic of the adaptive octree and its dual-tree interaction lists (CPU)."""
import numpy as np

from paper_2202_02847_gb300 import workloads as W


def _tree(n=3000, leaf=16):
    pts, q = W.plummer(n, seed=4)
    return pts, q, W.adaptive_octree(pts, leaf_size=leaf)


def test_plummer_distribution():
    pts, q = W.plummer(200000, seed=4)
    r = np.linalg.norm(pts, axis=1)
    # Plummer half-mass radius (r_h = 1/sqrt(2^{2/3}-1) = 1.305 for the untruncated profile)
    assert abs(np.median(r) - 1.305) < 0.02
    assert np.isclose(q.sum(), 1.0)
    assert abs(pts.mean(axis=0)).max() < 0.05


def test_octree_structure():
    pts, q, t = _tree()
    nn = len(t.level)
    assert t.parent[0] == -1 and t.level[0] == 0
    for i in range(1, nn):
        p = t.parent[i]
        assert t.level[i] == t.level[p] + 1
        assert t.first_child[p] <= i < t.first_child[p] + t.n_children[p]
        assert np.isclose(t.half[i], t.half[p] / 2)
        assert np.all(np.abs(t.centre[i] - t.centre[p]) <= t.half[p] + 1e-12)
        assert t.pt_begin[p] <= t.pt_begin[i] and t.pt_end[i] <= t.pt_end[p]
    leaves = t.is_leaf
    assert np.all(t.pt_end[leaves] - t.pt_begin[leaves] <= 16)
    # leaves partition the points, every point inside its leaf's box
    assert (t.pt_end[leaves] - t.pt_begin[leaves]).sum() == len(pts)
    for i in np.nonzero(leaves)[0]:
        p = pts[t.order[t.pt_begin[i]:t.pt_end[i]]]
        assert np.all(np.abs(p - t.centre[i]) <= t.half[i] * (1 + 1e-9))


def test_dual_tree_covers_every_far_leaf_pair_once():
    pts, q, t = _tree(1500, 12)
    src, tgt = W.dual_tree_m2l(t, 0.5)
    rad = np.sqrt(3) * t.half
    d = np.linalg.norm(t.centre[src] - t.centre[tgt], axis=1)
    assert np.all(rad[src] + rad[tgt] < 0.5 * d)             # acceptance criterion
    assert len(set(zip(src.tolist(), tgt.tolist()))) == len(src)
    anc = []
    for i in range(len(t.level)):
        a, s = i, set()
        while a >= 0:
            s.add(a)
            a = t.parent[a]
        anc.append(s)
    pairs = set(zip(src.tolist(), tgt.tolist()))
    leaves = np.nonzero(t.is_leaf)[0]
    far = 0
    for a in leaves:
        for b in leaves:
            c = sum((x, y) in pairs for x in anc[a] for y in anc[b])
            assert c <= 1, (a, b)
            if a == b:
                assert c == 0
            elif rad[a] + rad[b] < 0.5 * np.linalg.norm(t.centre[a] - t.centre[b]) * (1 - 1e-9):
                # well separated leaves are always translated (pairs exactly on the
                # acceptance boundary may go either way by rounding)
                assert c == 1, (a, b)
            far += c
    assert far > 0


def test_orders_rise_with_level():
    pts, q, t = _tree()
    P = W.order_by_level(t)
    assert P[0] == 4 and P.max() == 24
    assert np.all(np.diff([P[t.level == l].max() for l in range(t.max_level + 1)]) >= 0)
