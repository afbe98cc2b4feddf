"""Mixed-order batching on an adaptive octree (Plummer sphere): the fused
multi-class launch, the per-class launches, the policies and the autotuner
against each other and against the oracle."""
import numpy as np
import pytest

from paper_2202_02847_gb300 import workloads as W
import gpu_util as U

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def setup():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__
    __graft_entry__.build_library()
    from paper_2202_02847_gb300 import sfmm
    from paper_2202_02847_gb300.fmm import AdaptivePass
    pts, q = W.plummer(6000, seed=4)
    tree = W.adaptive_octree(pts, leaf_size=24)
    P_node = W.order_by_level(tree, lo=4, span=10)
    h = sfmm.Handle(int(P_node.max()), "f64")
    ap = AdaptivePass(tree, P_node, h)
    ap.p2m_leaves(pts, q)
    yield sfmm, ap, pts, q, tree, P_node, h
    h.close()


def _radius(tree, node):
    """Circumradius of an adaptive-tree box (half edge times sqrt(3))."""
    return float(np.sqrt(3.0) * tree.half[node])


def _oracle_M(orc, pts, q, tree, P_node, node):
    sel = tree.order[tree.pt_begin[node]:tree.pt_end[node]]
    return orc.p2m(int(P_node[node]), pts[sel], q[sel], tree.centre[node])


def test_m2l_waves_fused_and_per_class_agree_with_oracle(setup, orc):
    import torch
    sfmm, ap, pts, q, tree, P_node, h = setup
    ap.upward()
    assert len(ap.waves) >= 2 and any(len(d["classes"]) > 1 for d in ap.waves)
    results = {}
    for fused in (True, False):
        ap.L.zero_()
        for w in range(len(ap.waves)):
            ap.m2l_wave(w, fused)
        torch.cuda.synchronize()
        assert h.sync_status() == 0
        results[fused] = ap.L.cpu().numpy()
    g = W.rng(77)
    d0 = ap.waves[0]["host"]
    cand = np.unique(d0["row_tgt"])
    picks = g.choice(cand, size=min(12, len(cand)), replace=False)
    # all sources of the picked targets, over every wave
    for t in picks:
        Po = int(P_node[t])
        want = np.zeros(Po * (Po + 1))
        for d in ap.waves:
            hst = d["host"]
            for r in np.nonzero(hst["row_tgt"] == t)[0]:
                for j in range(hst["offs"][r], hst["offs"][r + 1]):
                    s = int(hst["src"][j])
                    Ms = _oracle_M(orc, pts, q, tree, P_node, s)
                    want += orc.translate("m2l", int(P_node[s]), Po, Ms, tree.centre[t] - tree.centre[s])
        a, b = ap.off[t], ap.off[t + 1]
        for fused in (True, False):
            U.check_rows(results[fused][a:b], want, Po, "L", 1e-12, a=_radius(tree, t),
                         what=f"target {t} fused={fused}")


def test_upward_pass_matches_p2m_of_subtrees(setup, orc):
    import torch
    sfmm, ap, pts, q, tree, P_node, h = setup
    ap.upward()
    torch.cuda.synchronize()
    M = ap.M.cpu().numpy()
    g = W.rng(78)
    inner = np.nonzero(~tree.is_leaf & (tree.pt_end - tree.pt_begin < 3000))[0]
    for n in g.choice(inner, size=min(8, len(inner)), replace=False):
        want = _oracle_M(orc, pts, q, tree, P_node, n)
        P = int(P_node[n])
        U.check_rows(M[ap.off[n]:ap.off[n + 1]], want, P, "M", 1e-12, a=_radius(tree, n),
                     what=f"node {n}")


def test_autotuner_installs_policies_and_keeps_results(setup, tmp_path):
    import torch
    sfmm, ap, pts, q, tree, P_node, h = setup
    from paper_2202_02847_gb300.autotune import Autotuner
    ap.step()
    torch.cuda.synchronize()
    before = ap.L.cpu().numpy()
    tuner = Autotuner(h, "f64", cache_path=str(tmp_path / "tune.json"))
    chosen, waves = ap.autotune(tuner, reps=1)
    tuner.save()
    assert chosen and waves and (tmp_path / "tune.json").exists()
    ap.step()
    torch.cuda.synchronize()
    after = ap.L.cpu().numpy()
    P = int(P_node.max())
    assert np.abs(after - before).max() <= 1e-12 * np.abs(before).max()
    # cached decisions are reused
    t2 = Autotuner(h, "f64", cache_path=str(tmp_path / "tune.json"))
    op, pi, po = "m2l", ap.waves[0]["classes"][0][1], ap.waves[0]["classes"][0][2]
    assert t2.tune(op, pi, po) == tuple(tuner.cache[next(k for k in tuner.cache if k.endswith(f"|m2l|{pi}|{po}"))])


def test_graph_capture_replays_the_pass(setup):
    import torch
    sfmm, ap, pts, q, tree, P_node, h = setup
    ap.step()
    torch.cuda.synchronize()
    ref = ap.L.clone()
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ap.step()                                   # warm-up on the capture stream
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ap.step()
    ap.L.fill_(7.0)
    graph.replay()
    torch.cuda.synchronize()
    assert torch.equal(ap.L, ref)


def test_policy_errors(setup):
    sfmm, ap, pts, q, tree, P_node, h = setup
    with pytest.raises(sfmm.SfmmError) as e:
        sfmm.set_policy(h, "m2l", 13, 13, "unrolled")   # order 13: no unrolled kernels
    assert e.value.code == 6
    with pytest.raises(sfmm.SfmmError) as e:
        sfmm.set_policy(h, "m2l", 7, 99, "shared")
    assert e.value.code == 2


def _check_all_nodes(ap, tree, P_node, got, want, kind, tol, what):
    """Per-expansion check of every node's solid (grouped by order)."""
    for P in np.unique(P_node):
        nodes = np.nonzero(P_node == P)[0]
        S = int(P) * (int(P) + 1)
        idx = (ap.off[nodes][:, None] + np.arange(S)[None, :])
        U.check_rows(got[idx], want[idx], int(P), kind, tol, a=np.sqrt(3.0) * tree.half[nodes],
                     what=f"{what}, order {P}")


def test_one_launch_pass_matches_the_multi_launch_pass(setup):
    """The whole pass (M2M levels, M2L waves, L2L levels) as one persistent
    launch with grid barriers between its phases gives, for every expansion,
    the result of the pass as separate launches (within 1e-12), and bitwise
    the same result on every run and under CUDA-graph replay."""
    import torch
    sfmm, ap, pts, q, tree, P_node, h = setup
    ap.step()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    refL, refM = ap.L.cpu().numpy(), ap.M.cpu().numpy()
    ap.step_one_launch()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    one = ap.L.clone()
    _check_all_nodes(ap, tree, P_node, ap.M.cpu().numpy(), refM, "M", 1e-12, "M after the one-launch pass")
    _check_all_nodes(ap, tree, P_node, one.cpu().numpy(), refL, "L", 1e-12, "L after the one-launch pass")
    ap.step_one_launch()
    torch.cuda.synchronize()
    assert torch.equal(ap.L, one)
    s = torch.cuda.Stream()
    s.wait_stream(torch.cuda.current_stream())
    with torch.cuda.stream(s):
        ap.step_one_launch()
    torch.cuda.current_stream().wait_stream(s)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph):
        ap.step_one_launch()
    ap.L.fill_(3.0)
    graph.replay()
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    assert torch.equal(ap.L, one)


@pytest.mark.parametrize("min_lanes", [4, 32])
def test_one_launch_pass_with_coarsened_lane_classes(setup, min_lanes):
    """The one-launch pass with every list on at least min_lanes lanes (the
    merged classes a pass gets when its lane classes exceed the class limit)
    agrees with the separate-launch pass for every expansion within 1e-12."""
    import torch
    sfmm, ap, pts, q, tree, P_node, h = setup
    ap.step()
    torch.cuda.synchronize()
    refL, refM = ap.L.cpu().numpy(), ap.M.cpu().numpy()
    ap.step_one_launch(min_lanes=min_lanes)
    torch.cuda.synchronize()
    assert h.sync_status() == 0
    _check_all_nodes(ap, tree, P_node, ap.L.cpu().numpy(), refL, "L", 1e-12,
                     f"L after the one-launch pass, lanes >= {min_lanes}")


def test_pass_rejects_bad_classes(setup):
    import torch
    sfmm, ap, pts, q, tree, P_node, h = setup
    z = torch.zeros(4, dtype=torch.int64, device="cuda")
    bad_phase = sfmm.pass_classes([("m2l", 4, 4, 1, 1, True, 1, z, z, z, z),
                                   ("m2l", 4, 4, 1, 0, True, 1, z, z, z, z)])
    with pytest.raises(sfmm.SfmmError) as e:
        sfmm.translate_pass(h, bad_phase)
    assert e.value.code == 1
    bad_lanes = sfmm.pass_classes([("m2l", 4, 4, 3, 0, True, 1, z, z, z, z)])
    with pytest.raises(sfmm.SfmmError) as e:
        sfmm.translate_pass(h, bad_lanes)
    assert e.value.code == 1
    bad_order = sfmm.pass_classes([("m2l", 4, 99, 1, 0, True, 1, z, z, z, z)])
    with pytest.raises(sfmm.SfmmError) as e:
        sfmm.translate_pass(h, bad_order)
    assert e.value.code == 2
