"""Translation pass of a uniform-octree FMM on the device (the hot path).

One pass = M2M from the leaves up to the root (one lists call per level,
each parent gathering its 8 children), all M2L interaction-list translations
of levels 2..depth in one lists call, and L2L from level 2 down to the leaves
(one batch call per level, accumulating onto the M2L results).  Every
translation is a C-ABI call into libsfmm.so; this module only lays out the
device arrays (solids of all levels, pointer and shift arrays, CSR offsets)
once and replays the launches.

Device layout: one array holds the multipole solids of all levels (level l
after levels 0..l-1, box-major, P(P+1) reals per box), one the local solids.
"""
import numpy as np
import torch

from . import sfmm
from . import workloads as W


class UniformPass:
    def __init__(self, tree, P, handle, device="cuda", dtype=torch.float64):
        self.tree, self.P, self.h = tree, P, handle
        self.device, self.dtype = device, dtype
        D = tree.depth
        self.D = D
        S = P * (P + 1)
        self.S = S
        nbox = [8 ** l for l in range(D + 1)]
        self.level_base = np.concatenate([[0], np.cumsum(nbox)])
        total = int(self.level_base[-1])
        self.M = torch.zeros(total, S, dtype=dtype, device=device)
        self.L = torch.zeros(total, S, dtype=dtype, device=device)
        dev = device

        def gidx(level, idx):
            return torch.as_tensor(self.level_base[level] + np.asarray(idx), dtype=torch.int64)

        # ---- M2M: parents at level l-1 gather their 8 children at level l
        self.m2m = []
        for l in range(D, 0, -1):
            par = W.parent_map(l)
            child = np.argsort(par, kind="stable")          # children grouped by parent
            npar = nbox[l - 1]
            offs = np.arange(0, 8 * npar + 1, 8, dtype=np.int64)
            cent_c = tree.levels[l].centres[child]
            cent_p = tree.levels[l - 1].centres[par[child]]
            self.m2m.append(dict(
                src=sfmm.pointer_array(self.M, S, gidx(l, child)),
                shift=torch.tensor(cent_p - cent_c, dtype=dtype, device=dev),
                offsets=torch.tensor(offs, device=dev),
                out=sfmm.pointer_array(self.M, S, gidx(l - 1, np.arange(npar))),
                n=npar, count=8 * npar))

        # ---- M2L: all targets of levels 2..D in one CSR, sorted by list length
        tgt, src, sh, lens = [], [], [], []
        for l in range(2, D + 1):
            lv = tree.levels[l]
            cnt = np.diff(lv.m2l_offsets)
            tgt.append(self.level_base[l] + np.arange(nbox[l]))
            lens.append(cnt)
            src.append(self.level_base[l] + lv.m2l_sources)
            sh.append(lv.m2l_shift)
        tgt, lens = np.concatenate(tgt), np.concatenate(lens)
        src_all, sh_all = np.concatenate(src), np.concatenate(sh)
        starts = np.concatenate([[0], np.cumsum(lens)[:-1]])
        order = np.argsort(-lens, kind="stable")              # long lists first
        new_lens = lens[order]
        new_offs = np.zeros(len(order) + 1, np.int64)
        np.cumsum(new_lens, out=new_offs[1:])
        gather = np.concatenate([np.arange(starts[t], starts[t] + lens[t]) for t in order]) \
            if len(order) else np.zeros(0, np.int64)
        self.m2l_targets = tgt[order]                 # global box ids, in kernel order
        self.m2l_offsets_host = new_offs
        self.m2l_src_host = src_all[gather]
        self.m2l_shift_host = sh_all[gather]
        self.m2l = dict(
            src=sfmm.pointer_array(self.M, S, torch.as_tensor(self.m2l_src_host)),
            shift=torch.tensor(self.m2l_shift_host, dtype=dtype, device=dev),
            offsets=torch.tensor(new_offs, device=dev),
            out=sfmm.pointer_array(self.L, S, torch.as_tensor(self.m2l_targets)),
            n=len(order), count=int(new_offs[-1]))

        # ---- L2L: each child at level l+1 receives from its parent at level l
        self.l2l = []
        for l in range(2, D):
            par = W.parent_map(l + 1)
            cent_c = tree.levels[l + 1].centres
            cent_p = tree.levels[l].centres[par]
            self.l2l.append(dict(
                inp=sfmm.pointer_array(self.L, S, gidx(l, par)),
                out=sfmm.pointer_array(self.L, S, gidx(l + 1, np.arange(nbox[l + 1]))),
                shift=torch.tensor(cent_c - cent_p, dtype=dtype, device=dev),
                count=nbox[l + 1]))

        self.counts = dict(m2m=sum(d["count"] for d in self.m2m), m2l=self.m2l["count"],
                           l2l=sum(d["count"] for d in self.l2l))

    # ------------------------------------------------------------ inputs
    def leaf_slice(self, which="M"):
        a = self.M if which == "M" else self.L
        return a[int(self.level_base[self.D]):int(self.level_base[self.D + 1])]

    def p2m_leaves(self, points, charges, leaf_of_point):
        """Multipoles of the leaves from the particles (sfmm_p2m_boxes)."""
        order = np.argsort(leaf_of_point, kind="stable")
        nleaf = 8 ** self.D
        counts = np.bincount(leaf_of_point, minlength=nleaf)
        offs = np.zeros(nleaf + 1, np.int64)
        np.cumsum(counts, out=offs[1:])
        dev = self.device
        pts = torch.tensor(points[order], dtype=self.dtype, device=dev)
        q = torch.tensor(charges[order], dtype=self.dtype, device=dev)
        cen = torch.tensor(self.tree.levels[self.D].centres, dtype=self.dtype, device=dev)
        sfmm.p2m_boxes(self.h, self.P, pts, q, torch.tensor(offs, device=dev), cen,
                       self.leaf_slice("M"), nleaf)

    # ------------------------------------------------------------ the pass
    def upward(self, stream=None):
        P = self.P
        for d in self.m2m:
            sfmm.translate_lists(self.h, "m2m", d["src"], d["shift"], d["offsets"], d["out"],
                                 P, P, d["n"], accumulate=False, stream=stream)

    def m2l_all(self, stream=None):
        d, P = self.m2l, self.P
        sfmm.translate_lists(self.h, "m2l", d["src"], d["shift"], d["offsets"], d["out"],
                             P, P, d["n"], accumulate=False, stream=stream)

    def downward(self, stream=None):
        P = self.P
        for d in self.l2l:
            sfmm.l2l_batch(self.h, d["inp"], d["out"], d["shift"], P, P, d["count"],
                           accumulate=True, stream=stream)

    def step(self, stream=None):
        self.upward(stream)
        self.m2l_all(stream)
        self.downward(stream)

    def launches_per_step(self):
        return len(self.m2m) + 1 + len(self.l2l)


def translation_cost(p_in, p_out):
    """Relative cost of one rotation-based translation from order p_in to
    p_out (the swaps of the input and output rows and the z-translation
    coupling them; constant factors dropped)."""
    z = sum((p_out - m) * (p_in - m) for m in range(min(p_in, p_out)))
    return p_in * (p_in + 1) * (2 * p_in + 1) // 6 + p_out * (p_out + 1) * (2 * p_out + 1) // 6 + z


def coarsen_lanes(classes, min_lanes):
    """A wave's classes (op, p_in, p_out, first row, end row, lanes) with at
    least `min_lanes` lanes per target: runs of adjacent rows of one order pair
    that end up with the same lanes are merged into one class.  Rows of one
    order pair are sorted by decreasing list length, so a merged class still
    gives every list at least as many lanes as its length needs (up to 32).
    The merged classes keep the order of the input (most expensive first
    chunk first), each at the place of its earliest part."""
    rank = {c[3]: k for k, c in enumerate(classes)}     # row ranges are disjoint
    out = []
    for c in sorted(classes, key=lambda c: (c[1], c[2], c[3])):
        g = max(c[5], min_lanes)
        if out and out[-1][0][1:3] == c[1:3] and out[-1][0][4] == c[3] and out[-1][0][5] == g:
            m, r = out[-1]
            out[-1] = ((m[0], m[1], m[2], m[3], c[4], g), min(r, rank[c[3]]))
        else:
            out.append(((c[0], c[1], c[2], c[3], c[4], g), rank[c[3]]))
    return [c for c, _ in sorted(out, key=lambda x: x[1])]


def lanes_for_length(lengths):
    """Lanes per target for lists of the given lengths: the smallest power of
    two >= the length, capped at 32 (one warp); 1 for lists of 0 or 1 source.
    A list then costs ceil(length / lanes) translations on the critical path
    and at most half of a group's lanes idle."""
    n = np.maximum(np.asarray(lengths, np.int64), 1)
    return np.minimum(32, 1 << np.ceil(np.log2(n)).astype(np.int64))


class AdaptivePass:
    """Translation pass of an adaptive octree with the expansion order rising
    with the level (mixed p_in != p_out in M2M, M2L and L2L).

    M2L pairs come from a dual-tree traversal.  A target may receive sources
    of several levels, i.e. several p_in; its sources are split by p_in into
    "waves" so that inside one wave every target appears at most once.  Each
    wave runs as one multi-class launch (sfmm_translate_lists_multi) or as one
    lists launch per class, whichever the autotuner measured faster; all waves
    accumulate onto locals zeroed at the start of the step.  M2M runs one lists
    launch per level (parents gather their children), L2L one batch launch per
    level.  Solids of all nodes live in one flat array each for M and L
    (node i at offset off[i], order P[i]).
    """

    def __init__(self, tree, P_node, handle, device="cuda", dtype=torch.float64, theta=0.5,
                 pairs=None):
        self.tree, self.h, self.device, self.dtype = tree, handle, device, dtype
        self.P = np.asarray(P_node, np.int64)
        S = self.P * (self.P + 1)
        self.off = np.concatenate([[0], np.cumsum(S)])
        total = int(self.off[-1])
        self.M = torch.zeros(total, dtype=dtype, device=device)
        self.L = torch.zeros(total, dtype=dtype, device=device)
        esz = self.M.element_size()
        baseM, baseL = self.M.data_ptr(), self.L.data_ptr()
        self.ptrM = lambda idx: torch.as_tensor(baseM + esz * self.off[np.asarray(idx)], dtype=torch.int64, device=device)
        self.ptrL = lambda idx: torch.as_tensor(baseL + esz * self.off[np.asarray(idx)], dtype=torch.int64, device=device)
        lev = tree.level
        cen = tree.centre
        self.launch_count = 0

        # ---- M2M by level (deepest first): parent gathers its children
        self.m2m = []
        for l in range(tree.max_level, 0, -1):
            par = np.nonzero((lev == l - 1) & (tree.first_child >= 0))[0]
            par = par[lev[tree.first_child[par]] == l]
            if len(par) == 0:
                continue
            cnt = tree.n_children[par]
            offs = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
            child = np.concatenate([np.arange(tree.first_child[p], tree.first_child[p] + c)
                                    for p, c in zip(par, cnt)])
            self.m2m.append(dict(
                p_in=int(self.P[child[0]]), p_out=int(self.P[par[0]]),
                src=self.ptrM(child), out=self.ptrM(par),
                shift=torch.tensor(cen[par].repeat(cnt, axis=0) - cen[child], dtype=dtype, device=device),
                offsets=torch.tensor(offs, device=device), n=len(par)))

        # ---- M2L pairs, grouped into waves and classes
        src, tgt = pairs if pairs is not None else W.dual_tree_m2l(tree, theta)
        self.n_m2l = len(src)
        pin, pout = self.P[src], self.P[tgt]
        # rank of p_in among the distinct p_in of the target -> wave
        o = np.lexsort((src, pin, tgt))
        src, tgt, pin, pout = src[o], tgt[o], pin[o], pout[o]
        newgrp = np.ones(len(src), bool)
        newgrp[1:] = (tgt[1:] != tgt[:-1]) | (pin[1:] != pin[:-1])
        grp_id = np.cumsum(newgrp) - 1
        gstart = np.nonzero(newgrp)[0]
        g_tgt = tgt[gstart]
        first_of_tgt = np.ones(len(gstart), bool)
        first_of_tgt[1:] = g_tgt[1:] != g_tgt[:-1]
        tstart = np.maximum.accumulate(np.where(first_of_tgt, np.arange(len(gstart)), 0))
        g_wave = np.arange(len(gstart)) - tstart
        wave = g_wave[grp_id]
        self.waves = []
        for w in range(int(wave.max()) + 1 if len(wave) else 0):
            sel = np.nonzero(wave == w)[0]
            ws, wt, wpi, wpo = src[sel], tgt[sel], pin[sel], pout[sel]
            # classes contiguous; inside a class, targets by decreasing list length
            # (a warp's 32 lanes take 32 consecutive targets and run as long as the
            # longest list), then by target and source
            _, tinv, tcnt = np.unique(wt, return_inverse=True, return_counts=True)
            oo = np.lexsort((ws, wt, -tcnt[tinv], wpo, wpi))
            ws, wt, wpi, wpo = ws[oo], wt[oo], wpi[oo], wpo[oo]
            newt = np.ones(len(ws), bool)
            newt[1:] = wt[1:] != wt[:-1]
            rows = np.nonzero(newt)[0]
            offs = np.concatenate([rows, [len(ws)]]).astype(np.int64)
            row_tgt, row_pi, row_po = wt[rows], wpi[rows], wpo[rows]
            # lanes per target: the power of two >= the list length, at most 32
            # (monotone in the length, so equal values are contiguous in a class)
            row_lanes = lanes_for_length(np.diff(offs))
            classes = []
            cs = 0
            for r in range(1, len(rows) + 1):
                if (r == len(rows) or row_pi[r] != row_pi[cs] or row_po[r] != row_po[cs]
                        or row_lanes[r] != row_lanes[cs]):
                    classes.append(("m2l", int(row_pi[cs]), int(row_po[cs]), cs, r, int(row_lanes[cs])))
                    cs = r
            # the fused launch hands out chunks in class order: most expensive
            # first chunk first (its longest list, ceil(length / lanes) rounds
            # of translations of that order pair)
            row_len = np.diff(offs)
            classes.sort(key=lambda c: -(-(-row_len[c[3]] // c[5]) * translation_cost(c[1], c[2])))
            self.waves.append(dict(
                classes=classes, n=len(rows),
                src=self.ptrM(ws), out=self.ptrL(row_tgt),
                shift=torch.tensor(cen[wt] - cen[ws], dtype=dtype, device=device),
                offsets=torch.tensor(offs, device=device), fused=True,
                host=dict(src=ws, tgt=wt, offs=offs, row_tgt=row_tgt)))

        # ---- L2L by level (top-down): every child receives from its parent
        self.l2l = []
        for l in range(1, tree.max_level + 1):
            child = np.nonzero(lev == l)[0]
            if len(child) == 0:
                continue
            par = tree.parent[child]
            self.l2l.append(dict(
                p_in=int(self.P[par[0]]), p_out=int(self.P[child[0]]),
                inp=self.ptrL(par), out=self.ptrL(child),
                shift=torch.tensor(cen[child] - cen[par], dtype=dtype, device=device),
                count=len(child)))
        self.counts = dict(m2m=int(sum(len(d["src"]) for d in self.m2m)), m2l=self.n_m2l,
                           l2l=int(sum(d["count"] for d in self.l2l)))
        pmax = int(self.P.max())
        self._plans = {}
        if handle is not None:                    # None: build the plan only (host tests)
            sfmm.reserve_scratch(handle, pmax)

    # ------------------------------------------------------------ inputs
    def p2m_leaves(self, points, charges):
        """Leaf multipoles from the particles, one P2M call per leaf level (the
        leaves' points are gathered into one contiguous array per level)."""
        t = self.tree
        pts_sorted = points[t.order]
        q_sorted = charges[t.order]
        leaves = np.nonzero(t.is_leaf)[0]
        for l in np.unique(t.level[leaves]):
            lv = leaves[t.level[leaves] == l]
            P = int(self.P[lv[0]])
            S = P * (P + 1)
            cnt = t.pt_end[lv] - t.pt_begin[lv]
            idx = np.concatenate([np.arange(b, e) for b, e in zip(t.pt_begin[lv], t.pt_end[lv])])
            offs = np.concatenate([[0], np.cumsum(cnt)]).astype(np.int64)
            pts = torch.tensor(pts_sorted[idx], dtype=self.dtype, device=self.device)
            q = torch.tensor(q_sorted[idx], dtype=self.dtype, device=self.device)
            cen = torch.tensor(t.centre[lv], dtype=self.dtype, device=self.device)
            tmp = torch.empty(len(lv), S, dtype=self.dtype, device=self.device)
            sfmm.p2m_boxes(self.h, P, pts, q, torch.tensor(offs, device=self.device), cen, tmp, len(lv))
            pos = torch.as_tensor(self.off[lv], device=self.device)
            cols = torch.arange(S, device=self.device)
            self.M.index_put_(((pos[:, None] + cols[None, :]).reshape(-1),), tmp.reshape(-1))

    # ------------------------------------------------------------ the pass
    def upward(self, stream=None):
        for d in self.m2m:
            sfmm.translate_lists(self.h, "m2m", d["src"], d["shift"], d["offsets"], d["out"],
                                 d["p_in"], d["p_out"], d["n"], stream=stream)

    def m2l_wave(self, w, fused, stream=None):
        d = self.waves[w]
        if fused:
            for a in range(0, len(d["classes"]), sfmm.MAX_CLASSES):
                sfmm.translate_lists_multi(self.h, d["classes"][a:a + sfmm.MAX_CLASSES], d["src"],
                                           d["shift"], d["offsets"], d["out"], accumulate=True,
                                           stream=stream)
        else:
            for op, pi, po, tb, te, _ in d["classes"]:
                sfmm.translate_lists(self.h, op, d["src"], d["shift"], d["offsets"][tb:],
                                     d["out"][tb:], pi, po, te - tb, accumulate=True, stream=stream)

    def m2l_all(self, stream=None):
        for w, d in enumerate(self.waves):
            self.m2l_wave(w, d["fused"], stream)

    def downward(self, stream=None):
        for d in self.l2l:
            sfmm.l2l_batch(self.h, d["inp"], d["out"], d["shift"], d["p_in"], d["p_out"],
                           d["count"], accumulate=True, stream=stream)

    def step(self, stream=None):
        self.L.zero_()
        self.upward(stream)
        self.m2l_all(stream)
        self.downward(stream)

    def pass_plan(self, parts=("m2m", "m2l", "l2l"), min_lanes=1):
        """The pass as phased classes for sfmm_translate_pass: one phase per M2M
        level (deepest first, parents overwritten), one per M2L wave (the
        wave's classes, accumulating), one per L2L level (each child a list of
        its parent, accumulating).  Built once per choice of parts; the
        arrays it points into are held by the pass object."""
        key = (tuple(parts), min_lanes)
        if key in self._plans:
            return self._plans[key]
        # a launch takes at most MAX_PASS_CLASSES classes: raise the fewest lanes
        # per target until the M2L waves' lane classes fit (merged ranges run
        # their shorter lists with idle lanes; the sums are unchanged)
        fixed = (len(self.m2m) if "m2m" in parts else 0) + (len(self.l2l) if "l2l" in parts else 0)
        waves = [coarsen_lanes(d["classes"], min_lanes) for d in self.waves]
        while "m2l" in parts and fixed + sum(len(c) for c in waves) > sfmm.MAX_PASS_CLASSES \
                and min_lanes < 32:
            min_lanes *= 2
            waves = [coarsen_lanes(d["classes"], min_lanes) for d in self.waves]
        cls, keep, ph = [], [], 0
        if "m2m" in parts:
            for d in self.m2m:
                cls.append(("m2m", d["p_in"], d["p_out"], 8, ph, False, d["n"], d["src"], d["shift"],
                            d["offsets"], d["out"]))
                ph += 1
        if "m2l" in parts:
            for d, wcls in zip(self.waves, waves):
                for op, pi, po, tb, te, g in wcls:
                    cls.append((op, pi, po, g, ph, True, te - tb, d["src"], d["shift"],
                                d["offsets"][tb:], d["out"][tb:]))
                ph += 1
        if "l2l" in parts:
            for d in self.l2l:
                offs = torch.arange(d["count"] + 1, dtype=torch.int64, device=self.device)
                keep.append(offs)
                cls.append(("l2l", d["p_in"], d["p_out"], 1, ph, True, d["count"], d["inp"], d["shift"],
                            offs, d["out"]))
                ph += 1
        plan = (sfmm.pass_classes(cls), keep, ph)
        self._plans[key] = plan
        return plan

    def run_pass(self, parts=("m2m", "m2l", "l2l"), stream=None, min_lanes=1):
        """The chosen parts of the pass as one persistent launch."""
        sfmm.translate_pass(self.h, self.pass_plan(parts, min_lanes)[0], stream=stream)

    def step_one_launch(self, stream=None, min_lanes=1):
        """The whole pass (locals zeroed first) as one persistent launch;
        min_lanes > 1 runs every list with at least that many lanes (the form a
        pass takes when its lane classes exceed the launch's class limit)."""
        self.L.zero_()
        self.run_pass(stream=stream, min_lanes=min_lanes)

    def launches_per_step(self):
        m2l = sum((len(d["classes"]) + sfmm.MAX_CLASSES - 1) // sfmm.MAX_CLASSES if d["fused"]
                  else len(d["classes"]) for d in self.waves)
        return len(self.m2m) + m2l + len(self.l2l)

    # ------------------------------------------------------------ tuning
    def autotune(self, tuner, reps=2):
        """Tune every order pair of the pass, then choose per M2L wave between
        the fused multi-class launch and per-class launches by timing both."""
        pairs = set()
        for d in self.m2m:
            pairs.add(("m2m", d["p_in"], d["p_out"]))
        for d in self.l2l:
            pairs.add(("l2l", d["p_in"], d["p_out"]))
        for d in self.waves:
            for op, pi, po, *_ in d["classes"]:
                pairs.add((op, pi, po))
        chosen = {}
        for op, pi, po in sorted(pairs):
            chosen[f"{op}:{pi}->{po}"] = tuner.tune(op, pi, po)
        waves = []
        for w, d in enumerate(self.waves):
            t = {}
            for fused in (True, False):
                self.m2l_wave(w, fused)
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record()
                for _ in range(reps):
                    self.m2l_wave(w, fused)
                e1.record()
                torch.cuda.synchronize()
                t[fused] = e0.elapsed_time(e1) / reps
            d["fused"] = t[True] <= t[False]
            waves.append({"wave": w, "classes": len(d["classes"]), "targets": d["n"],
                          "fused_ms": t[True], "per_class_ms": t[False], "fused": d["fused"]})
        return chosen, waves
