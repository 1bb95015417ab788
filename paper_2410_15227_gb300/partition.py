"""Spatial split of the mapping over ranks (one process per GPU).

The cells are divided into contiguous ranges of their generators' Morton
order (x, y, z each quantised to 21 bits over the box, bits interleaved x
highest), balanced by count.  A rank maps the pairs of its own cells only,
for the particles whose kernel support, the ball of radius 2h (Section 2.3),
reaches one of the bounding boxes of contiguous groups of those cells: every
pair (i, j) with dist(x_i, V_j) < 2 h_i has x_i within 2 h_i of the box of
V_j's group, so the ranks' pair lists together are the single-rank list,
each pair on exactly one rank.  The inverse mapping's per-particle sums,
sum_j w_ij f_j and sum_j w_ij, are then added over the ranks with one
all-reduce each, the only exchange.

Host logic only: which cells and particles a rank takes, and the reduction.
On the GPU a rank builds its cells with build_voronoi_cells, finds their
pairs with find_pairs_cells (the tree walk from each cell reaches the
particles near it, so every rank may pass all particles), maps them, and adds
the inverse mapping's sums with map_back_sums before reduce_sums.
"""
from __future__ import annotations

import numpy as np

_BITS = 21


def _spread3(q: np.ndarray) -> np.ndarray:
    """Insert two zero bits after each of the low 21 bits of q."""
    q = q.astype(np.uint64) & np.uint64(0x1FFFFF)
    q = (q | (q << np.uint64(32))) & np.uint64(0x1F00000000FFFF)
    q = (q | (q << np.uint64(16))) & np.uint64(0x1F0000FF0000FF)
    q = (q | (q << np.uint64(8))) & np.uint64(0x100F00F00F00F00F)
    q = (q | (q << np.uint64(4))) & np.uint64(0x10C30C30C30C30C3)
    q = (q | (q << np.uint64(2))) & np.uint64(0x1249249249249249)
    return q


def morton_keys(x, y, z, box) -> np.ndarray:
    """63-bit Morton keys of the points in the box [x0, x1, y0, y1, z0, z1]."""
    out = np.zeros(np.shape(x), np.uint64)
    for ax, (c, shift) in enumerate(((x, 2), (y, 1), (z, 0))):
        lo, hi = float(box[2 * ax]), float(box[2 * ax + 1])
        q = np.floor((np.asarray(c, dtype=np.float64) - lo) * ((1 << _BITS) / (hi - lo)))
        q = np.clip(q, 0, (1 << _BITS) - 1).astype(np.uint64)
        out |= _spread3(q) << np.uint64(shift)
    return out


def cell_ranges(gx, gy, gz, box, world: int) -> list[np.ndarray]:
    """Generator indices of each rank: the Morton order (ties by index) cut
    into `world` contiguous ranges whose sizes differ by at most one."""
    if world < 1:
        raise ValueError("world must be at least 1")
    order = np.argsort(morton_keys(gx, gy, gz, box), kind="stable")
    return [np.sort(part) for part in np.array_split(order, world)]


def morton_order(gx, gy, gz, box) -> np.ndarray:
    """The permutation that sorts the generators into Morton order (ties by
    index); with the generators stored in that order, rank r's cells are the
    contiguous range contiguous_ranges(n, world)[r]."""
    return np.argsort(morton_keys(gx, gy, gz, box), kind="stable")


def contiguous_ranges(n: int, world: int) -> list[tuple[int, int]]:
    """[begin, end) of each rank over n items, sizes differing by at most one
    (the ranges cell_ranges cuts from the Morton order)."""
    if world < 1:
        raise ValueError("world must be at least 1")
    edges = np.cumsum([0] + [len(p) for p in np.array_split(np.arange(n), world)])
    return [(int(edges[r]), int(edges[r + 1])) for r in range(world)]


def cell_boxes(cell_face_off, face_vert_off, verts) -> tuple[np.ndarray, np.ndarray]:
    """Axis-aligned bounding box (lo, hi), each (ncell, 3), of every cell of a
    face list in CSR form (cell j: faces cell_face_off[j]:cell_face_off[j+1],
    face f: vertices face_vert_off[f]:face_vert_off[f+1])."""
    cfo = np.asarray(cell_face_off, dtype=np.int64)
    fvo = np.asarray(face_vert_off, dtype=np.int64)
    v = np.asarray(verts, dtype=np.float64).reshape(-1, 3)
    start = fvo[cfo[:-1]]
    if np.any(fvo[cfo[1:]] <= start):
        raise ValueError("every cell needs at least one vertex")
    return np.minimum.reduceat(v, start, axis=0), np.maximum.reduceat(v, start, axis=0)


def group_boxes(lo, hi, order, ngroups: int) -> tuple[np.ndarray, np.ndarray]:
    """Boxes of `ngroups` contiguous groups of the cells taken in `order`
    (a rank's cells in Morton order, so that each group is compact): the
    union box of each group's cell boxes."""
    order = np.asarray(order)
    parts = [p for p in np.array_split(order, max(1, min(ngroups, order.shape[0]))) if p.shape[0]]
    glo = np.array([lo[p].min(axis=0) for p in parts]).reshape(-1, 3)
    ghi = np.array([hi[p].max(axis=0) for p in parts]).reshape(-1, 3)
    return glo, ghi


def reaching(x, y, z, h, lo, hi) -> np.ndarray:
    """Indices of the particles whose ball of radius 2h meets at least one of
    the boxes [lo_k, hi_k] (lo, hi of shape (3,) or (k, 3); closed: a particle
    at distance exactly 2h is kept, and the squared distances are compared
    with a relative margin of 1e-12 above their rounding: a superset of the
    strict pair test)."""
    p = np.stack([np.asarray(x, np.float64), np.asarray(y, np.float64), np.asarray(z, np.float64)], axis=1)
    r2 = (2.0 * np.asarray(h, np.float64)) ** 2
    lo, hi = np.atleast_2d(lo), np.atleast_2d(hi)
    hit = np.zeros(p.shape[0], dtype=bool)
    for k in range(lo.shape[0]):
        d = np.maximum(np.maximum(lo[k] - p, p - hi[k]), 0.0)
        hit |= (d * d).sum(axis=1) <= r2 * (1.0 + 1e-12)
    return np.nonzero(hit)[0]


def reduce_sums(num, den, group=None):
    """Add the ranks' per-particle sums (torch tensors, in place) with one
    all-reduce each; a single process returns them unchanged."""
    import torch.distributed as dist
    if dist.is_available() and dist.is_initialized() and dist.get_world_size(group) > 1:
        dist.all_reduce(num, op=dist.ReduceOp.SUM, group=group)
        dist.all_reduce(den, op=dist.ReduceOp.SUM, group=group)
    return num, den
