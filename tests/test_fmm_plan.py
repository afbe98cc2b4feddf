"""Host logic of the uniform-octree pass: the launch plan (CPU only)."""
import numpy as np
import pytest
import torch

from paper_2202_02847_gb300 import workloads as W


@pytest.fixture(scope="module")
def plan():
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300.fmm import UniformPass
    tree = W.uniform_octree(3)
    return tree, UniformPass(tree, 4, None, device="cpu")


def test_counts(plan):
    tree, fp = plan
    assert fp.counts["m2m"] == 8 + 64 + 512
    assert fp.counts["l2l"] == 512
    assert fp.counts["m2l"] == 3096 + 53352
    assert fp.launches_per_step() == 3 + 1 + 1


def test_m2l_plan_is_a_permutation_of_the_lists(plan):
    """The length-sorted CSR holds exactly every (target, source, shift) of the
    interaction lists of levels 2..3, each target's sources in list order."""
    tree, fp = plan
    lens = np.diff(fp.m2l_offsets_host)
    assert np.all(np.diff(lens) <= 0)                       # long lists first
    seen = {}
    for pos, t in enumerate(fp.m2l_targets):
        j0, j1 = fp.m2l_offsets_host[pos], fp.m2l_offsets_host[pos + 1]
        seen[int(t)] = (fp.m2l_src_host[j0:j1], fp.m2l_shift_host[j0:j1])
    for l in (2, 3):
        lv = tree.levels[l]
        base = fp.level_base[l]
        for b in range(8 ** l):
            src, sh = seen[int(base + b)]
            j0, j1 = lv.m2l_offsets[b], lv.m2l_offsets[b + 1]
            assert np.array_equal(src, base + lv.m2l_sources[j0:j1])
            assert np.allclose(sh, lv.m2l_shift[j0:j1])
            # shift = target centre - source centre, at least 2 boxes apart
            assert np.all(np.abs(sh).max(axis=1) >= 2 * lv.h - 1e-12)


def test_pointer_arrays_address_the_right_solids(plan):
    tree, fp = plan
    S = fp.S
    base = fp.M.data_ptr()
    src = fp.m2l["src"].numpy()
    assert np.array_equal((src - base) // (8 * S), fp.m2l_src_host)
    out = fp.m2l["out"].numpy()
    assert np.array_equal((out - fp.L.data_ptr()) // (8 * S), fp.m2l_targets)


def test_m2m_groups_children_under_parents(plan):
    tree, fp = plan
    for i, l in enumerate(range(3, 0, -1)):
        d = fp.m2m[i]
        src = (d["src"].numpy() - fp.M.data_ptr()) // (8 * fp.S) - fp.level_base[l]
        par = W.parent_map(l)
        assert np.array_equal(par[src], np.repeat(np.arange(8 ** (l - 1)), 8))
        # shift = parent centre - child centre, length sqrt(3) h / 2
        h = tree.levels[l].h
        assert np.allclose(np.linalg.norm(d["shift"].numpy(), axis=1), np.sqrt(3) * h / 2)


def test_l2l_maps_children_to_parents(plan):
    tree, fp = plan
    d = fp.l2l[0]
    inp = (d["inp"].numpy() - fp.L.data_ptr()) // (8 * fp.S) - fp.level_base[2]
    assert np.array_equal(inp, W.parent_map(3))
