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


def _level_geometry(depth):
    nside = 1 << depth
    h = 1.0 / nside
    ijk = np.stack(np.meshgrid(np.arange(nside), np.arange(nside), np.arange(nside),
                               indexing="ij"), axis=-1).reshape(-1, 3)
    centres = (ijk + 0.5) * h
    return nside, h, ijk, centres


def _interaction_lists(depth):
    """Standard FMM interaction list at a level: children of the parent's
    neighbours (including the parent itself) that are not adjacent to the
    target box.  Returns CSR arrays in target-major order, sources sorted by
    box index within each target."""
    nside, h, ijk, centres = _level_geometry(depth)
    nbox = nside ** 3
    if depth < 2:
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
