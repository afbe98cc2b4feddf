"""Seeded synthetic inputs shared by the CUDA path's tests/benchmark and the oracle.

This module holds only input generation: random numbers (numpy PCG64),
geometry of boxes and octrees, and index lists.  It contains none of the
translation arithmetic (no harmonics, no expansions, no rotations), so both
sides of every parity test can draw from it without sharing method code.

Workloads (the paper's workloads are "many translations of order P with
arbitrary shifts", Sec. 4; the FMM structure follows the standard uniform
octree of Sec. 1.2):
  * clusters of charges uniform in a unit box, q ~ U[-1, 1];
  * shift vectors = random unit direction x length U[lo, hi];
  * a uniform octree of given depth over the unit cube with the standard
    M2M / M2L interaction list / L2L structure.
"""
from dataclasses import dataclass, field

import numpy as np
from types import SimpleNamespace


def rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


def unit_directions(g, count):
    v = g.normal(size=(count, 3))
    v /= np.linalg.norm(v, axis=1, keepdims=True)
    return v


def shifts(g, count, lo=2.0, hi=4.0):
    """Random unit directions scaled by U[lo, hi] (count x 3)."""
    return unit_directions(g, count) * g.uniform(lo, hi, size=(count, 1))


def charge_clusters(g, count, nq=32, half=0.5):
    """count clusters of nq charges uniform in [-half, half]^3, q ~ U[-1,1].

    Returns positions (count, nq, 3) and charges (count, nq)."""
    pos = g.uniform(-half, half, size=(count, nq, 3))
    q = g.uniform(-1.0, 1.0, size=(count, nq))
    return pos, q


def random_solids(g, count, P, decay=0.5):
    """Random coefficient solids in the row layout with Im C_n^0 = 0.

    Row n is drawn N(0,1) and multiplied by decay**n, so that higher rows are
    smaller (as in expansions of a source cluster); this is an input
    distribution only."""
    out = np.zeros((count, P * (P + 1)))
    for n in range(P):
        base = n * (n + 1)
        out[:, base:base + 2 * (n + 1)] = g.normal(size=(count, 2 * (n + 1))) * decay ** n
        out[:, base + n + 1] = 0.0  # Im C_n^0
    return out


def solid_size(P):
    return P * (P + 1)


# --------------------------------------------------------------------- octree

@dataclass
class Level:
    depth: int
    nside: int
    h: float                      # box edge length
    centres: np.ndarray           # (nbox, 3)
    # M2L interaction lists in target-major CSR form
    m2l_offsets: np.ndarray = field(default=None)   # (nbox+1,) int64
    m2l_sources: np.ndarray = field(default=None)   # (nnz,) int64 box index at this level
    m2l_shift: np.ndarray = field(default=None)     # (nnz, 3) target centre - source centre
    m2l_code: np.ndarray = field(default=None)      # (nnz,) offset code in [0, 343)


@dataclass
class UniformOctree:
    depth: int
    levels: list                  # levels[0..depth]
    points: np.ndarray = None
    charges: np.ndarray = None
    leaf_of_point: np.ndarray = None


def box_index(ix, iy, iz, nside):
    return (ix * nside + iy) * nside + iz


def _level_geometry(depth, nside=None):
    nside = (1 << depth) if nside is None else nside
    h = 1.0 / nside
    ijk = np.stack(np.meshgrid(np.arange(nside), np.arange(nside), np.arange(nside),
                               indexing="ij"), axis=-1).reshape(-1, 3)
    centres = (ijk + 0.5) * h
    return nside, h, ijk, centres


def _interaction_lists(depth, nside=None):
    """Standard FMM interaction list at a level: children of the parent's
    neighbours (including the parent itself) that are not adjacent to the
    target box.  Returns CSR arrays in target-major order, sources sorted by
    box index within each target.  ``nside`` overrides the side 2^depth (any
    even side: a uniform grid of boxes whose parents form a grid of side/2)."""
    nside, h, ijk, centres = _level_geometry(depth, nside)
    nbox = nside ** 3
    if nside < 4:
        return (np.zeros(nbox + 1, np.int64), np.zeros(0, np.int64),
                np.zeros((0, 3)), np.zeros(0, np.int64))
    par = ijk // 2
    tg, sr, cd = [], [], []
    for dx in range(-3, 4):
        for dy in range(-3, 4):
            for dz in range(-3, 4):
                if max(abs(dx), abs(dy), abs(dz)) <= 1:
                    continue                    # adjacent boxes are near field
                o = np.array([dx, dy, dz])
                s = ijk + o
                ok = np.all((s >= 0) & (s < nside), axis=1)
                ok &= np.all(np.abs(s // 2 - par) <= 1, axis=1)
                t = np.nonzero(ok)[0]
                tg.append(t)
                sr.append(box_index(s[t, 0], s[t, 1], s[t, 2], nside))
                cd.append(np.full(len(t), ((dx + 3) * 7 + (dy + 3)) * 7 + (dz + 3)))
    tg, sr, cd = np.concatenate(tg), np.concatenate(sr), np.concatenate(cd)
    order = np.lexsort((sr, tg))
    tg, sr, cd = tg[order], sr[order], cd[order]
    counts = np.bincount(tg, minlength=nbox)
    offsets = np.zeros(nbox + 1, np.int64)
    np.cumsum(counts, out=offsets[1:])
    shift = centres[tg] - centres[sr]
    return offsets, sr.astype(np.int64), shift, cd.astype(np.int64)


def grid_level(nside):
    """One uniform level of side ``nside`` (even) over the unit cube: box size,
    centres and its M2L interaction lists (``m2l_offsets``, ``m2l_sources``,
    ``m2l_shift``, ``m2l_code``), as for a level of ``uniform_octree``."""
    if nside < 2 or nside % 2:
        raise ValueError("grid side must be even")
    _, h, ijk, centres = _level_geometry(0, nside)
    off, src, shift, code = _interaction_lists(0, nside)
    return SimpleNamespace(nside=nside, h=h, ijk=ijk, centres=centres, m2l_offsets=off,
                           m2l_sources=src, m2l_shift=shift, m2l_code=code)


def uniform_octree(depth, npoints=0, seed=2):
    """Uniform octree over the unit cube down to ``depth`` (level l has 8^l boxes).

    With npoints > 0 the points are uniform in the unit cube with q ~ U[-1,1]
    (seeded) and bucketed into the leaves."""
    levels = []
    for d in range(depth + 1):
        nside, h, ijk, centres = _level_geometry(d)
        lv = Level(depth=d, nside=nside, h=h, centres=centres)
        lv.m2l_offsets, lv.m2l_sources, lv.m2l_shift, lv.m2l_code = _interaction_lists(d)
        levels.append(lv)
    tree = UniformOctree(depth=depth, levels=levels)
    if npoints:
        g = rng(seed)
        tree.points = g.uniform(0.0, 1.0, size=(npoints, 3))
        tree.charges = g.uniform(-1.0, 1.0, size=npoints)
        nside = 1 << depth
        ijk = np.minimum((tree.points * nside).astype(np.int64), nside - 1)
        tree.leaf_of_point = box_index(ijk[:, 0], ijk[:, 1], ijk[:, 2], nside)
    return tree


def children_of(depth, parent_index):
    """The 8 child box indices (level depth+1) of a box at level ``depth``."""
    nside = 1 << depth
    i, rem = divmod(parent_index, nside * nside)
    j, k = divmod(rem, nside)
    out = []
    for a in range(2):
        for b in range(2):
            for c in range(2):
                out.append(box_index(2 * i + a, 2 * j + b, 2 * k + c, 2 * nside))
    return out


def parent_map(depth):
    """For every box at level depth (>= 1), the index of its parent at depth-1."""
    nside = 1 << depth
    _, _, ijk, _ = _level_geometry(depth)
    p = ijk // 2
    return box_index(p[:, 0], p[:, 1], p[:, 2], nside // 2)


# ------------------------------------------------------------ adaptive octree

def plummer(n, seed=4, u_max=0.999):
    """Plummer sphere: radius r = (u^{-2/3} - 1)^{-1/2}, u ~ U(0, u_max) (the cut
    keeps r finite), isotropic directions; masses q = 1/n."""
    g = rng(seed)
    u = g.uniform(0.0, u_max, size=n)
    u = np.maximum(u, 1e-300)
    r = 1.0 / np.sqrt(u ** (-2.0 / 3.0) - 1.0)
    pts = unit_directions(g, n) * r[:, None]
    return pts, np.full(n, 1.0 / n)


@dataclass
class AdaptiveOctree:
    """Nodes in breadth-first order (parents before children)."""
    level: np.ndarray          # (nn,)
    centre: np.ndarray         # (nn, 3)
    half: np.ndarray           # (nn,) half edge length
    parent: np.ndarray         # (nn,) -1 for the root
    first_child: np.ndarray    # (nn,) index of first child, -1 for leaves
    n_children: np.ndarray     # (nn,) number of (non-empty) children
    pt_begin: np.ndarray       # (nn,) range of the node's points in `order`
    pt_end: np.ndarray
    order: np.ndarray          # point permutation (Morton order)
    max_level: int

    @property
    def is_leaf(self):
        return self.first_child < 0


def adaptive_octree(points, leaf_size=64, max_level=21):
    """Octree over the bounding cube of the points, splitting every node with
    more than leaf_size points (empty children are not created)."""
    lo = points.min(axis=0)
    hi = points.max(axis=0)
    span = float((hi - lo).max()) * (1 + 1e-12)
    centre0 = (lo + hi) / 2
    corner = centre0 - span / 2
    B = max_level
    ijk = np.clip(((points - corner) / span * (1 << B)).astype(np.int64), 0, (1 << B) - 1)
    key = np.zeros(len(points), np.int64)
    for b in range(B):                         # interleave bits: x high, then y, then z
        for d in range(3):
            key |= ((ijk[:, d] >> b) & 1) << (3 * b + (2 - d))
    order = np.argsort(key, kind="stable")
    key = key[order]
    # level-by-level construction
    levels, centres, halfs, parents, begins, ends = [], [], [], [], [], []
    cur = [(0, 0, len(points), -1)]            # (prefix, begin, end, parent)
    lvl = 0
    node_prefix = []
    while cur:
        nxt = []
        base = len(levels)
        for i, (pref, b, e, par) in enumerate(cur):
            idx = base + i
            levels.append(lvl)
            h = span / (1 << lvl) / 2
            # centre from the prefix bits
            c = corner.copy()
            for k in range(lvl):
                trip = (pref >> (3 * (lvl - 1 - k))) & 7
                step = span / (1 << (k + 1))
                c = c + np.array([(trip >> 2) & 1, (trip >> 1) & 1, trip & 1]) * step
            centres.append(c + h)
            halfs.append(h)
            parents.append(par)
            begins.append(b)
            ends.append(e)
            if e - b > leaf_size and lvl < B:
                shift = 3 * (B - lvl - 1)
                sub = (key[b:e] >> shift) & 7
                cuts = np.searchsorted(sub, np.arange(9))
                for ch in range(8):
                    cb, ce = b + cuts[ch], b + cuts[ch + 1]
                    if ce > cb:
                        nxt.append(((pref << 3) | ch, cb, ce, idx))
        cur = nxt
        lvl += 1
    nn = len(levels)
    parent = np.array(parents, np.int64)
    first_child = np.full(nn, -1, np.int64)
    n_children = np.zeros(nn, np.int64)
    for i in range(1, nn):
        p = parent[i]
        if first_child[p] < 0:
            first_child[p] = i
        n_children[p] += 1
    return AdaptiveOctree(level=np.array(levels, np.int64), centre=np.array(centres),
                          half=np.array(halfs), parent=parent, first_child=first_child,
                          n_children=n_children, pt_begin=np.array(begins, np.int64),
                          pt_end=np.array(ends, np.int64), order=order,
                          max_level=int(max(levels)))


def order_by_level(tree, lo=4, span=20):
    """Expansion order rising with the level: P(l) = lo + round(span * l / L_max)."""
    L = max(tree.max_level, 1)
    return lo + np.rint(span * tree.level / L).astype(np.int64)


def dual_tree_m2l(tree, theta=0.5):
    """M2L pairs (source A, target B) of a dual-tree traversal with the
    acceptance criterion (rA + rB) < theta |cA - cB| (r = box circumradius).
    Breadth-first over pair arrays, splitting the larger box (or the non-leaf)
    of every rejected pair; leaf-leaf pairs are near field (not translated).
    Returns (src, tgt) arrays sorted by (tgt, src)."""
    rad = np.sqrt(3.0) * tree.half
    leaf = tree.is_leaf
    fc, nc = tree.first_child, tree.n_children
    A = np.array([0], np.int64)
    Bn = np.array([0], np.int64)
    out_a, out_b = [], []

    def children_pairs(keep_side, split_side, split_first):
        # expand split_side nodes into their children, pairing each with keep_side
        cnt = nc[split_side]
        rep_keep = np.repeat(keep_side, cnt)
        starts = np.repeat(fc[split_side], cnt)
        offs = np.arange(cnt.sum()) - np.repeat(np.cumsum(cnt) - cnt, cnt)
        return rep_keep, starts + offs

    while len(A):
        same = A == Bn
        d = np.linalg.norm(tree.centre[A] - tree.centre[Bn], axis=1)
        acc = (~same) & (rad[A] + rad[Bn] < theta * d)
        out_a.append(A[acc])
        out_b.append(Bn[acc])
        rest = ~acc
        A, Bn, same = A[rest], Bn[rest], same[rest]
        la, lb = leaf[A], leaf[Bn]
        near = la & lb
        A, Bn, same, la, lb = A[~near], Bn[~near], same[~near], la[~near], lb[~near]
        # self pairs: all (child, child') pairs of the node
        sA = A[same]
        cnt = nc[sA]
        if len(sA):
            par = np.repeat(sA, cnt * cnt)
            k = np.arange((cnt * cnt).sum()) - np.repeat(np.cumsum(cnt * cnt) - cnt * cnt, cnt * cnt)
            cc = np.repeat(cnt, cnt * cnt)
            sa_new = fc[par] + k // cc
            sb_new = fc[par] + k % cc
        else:
            sa_new = sb_new = np.zeros(0, np.int64)
        A, Bn, la, lb = A[~same], Bn[~same], la[~same], lb[~same]
        split_a = (~la) & (lb | (rad[A] >= rad[Bn]))
        b_keep, a_new = children_pairs(Bn[split_a], A[split_a], True)
        a_keep, b_new = children_pairs(A[~split_a], Bn[~split_a], False)
        A = np.concatenate([sa_new, a_new, a_keep])
        Bn = np.concatenate([sb_new, b_keep, b_new])
    src = np.concatenate(out_a)
    tgt = np.concatenate(out_b)
    o = np.lexsort((src, tgt))
    return src[o], tgt[o]
