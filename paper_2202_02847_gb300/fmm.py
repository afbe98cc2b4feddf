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
