"""Plain FP64 CPU oracle for the pseudo-particle Exact mapping.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the CPU
baseline leg of ``bench.py`` may import this package.  It shares no code with
the CUDA library: the arithmetic lives in ``exact.c`` and ``tree.c`` (plain C,
compiled with ``-ffp-contract=off``) and in the numpy code below.

What it computes, by the paper's sections and equations:

* M4 kernel, cumulative G, analytic integral over a right sub-triangle pyramid,
  signed face-pyramid decomposition of a convex cell (Exact mapping, Section 1,
  Section 2.3; the formula is derived from the definition of the weight), and an
  independent ray quadrature of the same weight.
* Brute-force Voronoi cells (Section 2.3), all-pairs particle-cell test,
  cell densities rho_j = sum_i m_i w_ij / V_j.
* Morton octree, node mass / COM / size (Section 2.2.1), adaptive tree-walk
  (Section 2.4.1, Eq. 4), node h-solver (Section 2.4.2, Eqs. 6-11), inverse
  mapping f_i = sum_j w_ij f_j / sum_j w_ij (Section 2.3, ``map_back``) and
  constituent inheritance (Section 2.5, ``inherit``).
* Cell centroids and Lloyd's iteration on the sites (Section 2.3); the
  adaptive refinement of the tree-walk (Section 2.4.1, Eq. 5).

Parity pins live in ``tests/test_oracle_*.py``.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

from .build import build as _build
from .build import build_count as _build_count

_HERE = os.path.dirname(os.path.abspath(__file__))
_lib = None
_count_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build()
        _lib = C.CDLL(path)
        _declare(_lib)
    return _lib


_d = C.c_double
_i64 = C.c_int64
_i32 = C.c_int
_p = C.c_void_p


def _declare(L):
    L.orc_w_shape.restype = _d; L.orc_w_shape.argtypes = [_d]
    L.orc_W.restype = _d; L.orc_W.argtypes = [_d, _d]
    L.orc_dWdh.restype = _d; L.orc_dWdh.argtypes = [_d, _d]
    L.orc_g.restype = _d; L.orc_g.argtypes = [_d]
    L.orc_G.restype = _d; L.orc_G.argtypes = [_d, _d]
    L.orc_K.restype = _d; L.orc_K.argtypes = [_d]
    L.orc_right_triangle.restype = _d; L.orc_right_triangle.argtypes = [_d, _d, _d]
    L.orc_face_pyramid.restype = _d
    L.orc_face_pyramid.argtypes = [_p, _d, _i32, _p, _p]
    L.orc_cell_weight.restype = _d
    L.orc_cell_weight.argtypes = [_p, _d, _i32, _p, _p, _p]
    L.orc_cell_weight_quadrature.restype = _d
    L.orc_cell_weight_quadrature.argtypes = [_p, _d, _i32, _p, _p, _d]
    L.orc_voronoi_cells.restype = _i64
    L.orc_voronoi_cells.argtypes = [_i64, _p, _p, _p, _p, _i64, _p, _i32, _i32,
                                    _p, _p, _p, _p, _p, _p, _p, _i32]
    L.orc_cell_distance.restype = _d
    L.orc_cell_distance.argtypes = [_p, _i32, _p, _p, _p]
    L.orc_find_pairs.restype = None
    L.orc_find_pairs.argtypes = [_i64, _p, _p, _p, _p, _i64, _p, _p, _p, _p, _p, _p, _p,
                                 _p, _p, _p, _p, _i32]
    L.orc_map_exact.restype = None
    L.orc_map_exact.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _i32]
    L.orc_cell_density.restype = None
    L.orc_cell_density.argtypes = [_i64, _p, _p, _p, _p, _p, _p]
    L.orc_morton_keys.restype = None
    L.orc_morton_keys.argtypes = [_i64, _p, _p, _p, _p, _p]
    L.orc_build_tree.restype = _i64
    L.orc_build_tree.argtypes = [_i64, _p, _p, _p, _p, _p, _i32, _i64] + [_p] * 16
    L.orc_select.restype = _i64
    L.orc_select.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _p, _p, _i32, _p, _d, _d, _d,
                             _i64, _p, _p, _p, _p, _p]
    L.orc_h_solve.restype = None
    L.orc_h_solve.argtypes = [_i64, _p, _p, _p, _i64, _p, _p, _p, _p, _d, _d, _i32, _p, _p,
                              _p, _i32]


def _ptr(a: np.ndarray):
    """Pointer to a contiguous array; the returned ctypes object keeps the array
    alive until the call that receives it has returned."""
    assert a.flags["C_CONTIGUOUS"], "arrays passed to the oracle must be contiguous"
    return a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


def _i64a(a):
    return np.ascontiguousarray(a, dtype=np.int64)


def nthreads_default() -> int:
    return max(1, os.cpu_count() or 1)


# ---------------------------------------------------------------------------
# Kernel
# ---------------------------------------------------------------------------

def W(r: float, h: float) -> float:
    return lib().orc_W(float(r), float(h))


def dWdh(r: float, h: float) -> float:
    return lib().orc_dWdh(float(r), float(h))


def G(R: float, h: float) -> float:
    return lib().orc_G(float(R), float(h))


def K(Q: float) -> float:
    return lib().orc_K(float(Q))


def right_triangle(D: float, A: float, T: float) -> float:
    return lib().orc_right_triangle(float(D), float(A), float(T))


# ---------------------------------------------------------------------------
# Cells
# ---------------------------------------------------------------------------

@dataclass
class Cells:
    """Convex cells in CSR form: cell j has faces cell_face_off[j]:cell_face_off[j+1];
    face f has vertices verts[face_vert_off[f]:face_vert_off[f+1]] (counter-clockwise
    seen from outside), unit outward normal normals[f] and neighbour id nbr[f]
    (generator index, or -1-w for box wall w)."""
    cell_face_off: np.ndarray
    face_vert_off: np.ndarray
    verts: np.ndarray
    normals: np.ndarray
    nbr: np.ndarray
    volume: np.ndarray
    gen: np.ndarray            # generator positions (ncell, 3)
    cell_ids: np.ndarray       # generator index of each stored cell

    @property
    def ncell(self) -> int:
        return int(self.cell_face_off.shape[0] - 1)

    def faces(self, j):
        f0, f1 = self.cell_face_off[j], self.cell_face_off[j + 1]
        out = []
        for f in range(f0, f1):
            v0, v1 = self.face_vert_off[f], self.face_vert_off[f + 1]
            out.append((self.verts[v0:v1], self.normals[f], int(self.nbr[f])))
        return out

    def offsets(self):
        """Plane offsets c_f = n_f . v_0 for every face."""
        return np.einsum("ij,ij->i", self.normals, self.verts[self.face_vert_off[:-1]])

    def sub(self, j):
        """A one-cell Cells object for cell j."""
        f0, f1 = int(self.cell_face_off[j]), int(self.cell_face_off[j + 1])
        v0, v1 = int(self.face_vert_off[f0]), int(self.face_vert_off[f1])
        return Cells(np.array([0, f1 - f0], dtype=np.int64),
                     self.face_vert_off[f0:f1 + 1] - v0, self.verts[v0:v1].copy(),
                     self.normals[f0:f1].copy(), self.nbr[f0:f1].copy(),
                     self.volume[j:j + 1].copy(), self.gen[j:j + 1].copy(),
                     self.cell_ids[j:j + 1].copy())


def cells_from_faces(face_lists, gen=None, volume=None) -> Cells:
    """Build Cells from [[(verts (k,3), normal (3,)), ...] per cell]."""
    cfo, fvo, V, N, nb = [0], [0], [], [], []
    for faces in face_lists:
        for item in faces:
            v, n = item[0], item[1]
            V.append(np.asarray(v, dtype=np.float64))
            N.append(np.asarray(n, dtype=np.float64))
            nb.append(item[2] if len(item) > 2 else -1)
            fvo.append(fvo[-1] + len(v))
        cfo.append(len(N))
    nc = len(face_lists)
    return Cells(np.array(cfo, dtype=np.int64), np.array(fvo, dtype=np.int64),
                 np.concatenate(V).reshape(-1, 3), np.array(N).reshape(-1, 3),
                 np.array(nb, dtype=np.int64),
                 np.zeros(nc) if volume is None else np.asarray(volume, dtype=np.float64),
                 np.zeros((nc, 3)) if gen is None else np.asarray(gen, dtype=np.float64),
                 np.arange(nc, dtype=np.int64))


def box_cell(lo, hi) -> list:
    """Faces of an axis-aligned box (for building test cells)."""
    lo = np.asarray(lo, dtype=np.float64)
    hi = np.asarray(hi, dtype=np.float64)
    c = np.array([[hi[0] if i & 1 else lo[0], hi[1] if i & 2 else lo[1],
                   hi[2] if i & 4 else lo[2]] for i in range(8)])
    loops = [(0, 4, 6, 2), (1, 3, 7, 5), (0, 1, 5, 4), (2, 6, 7, 3), (0, 2, 3, 1), (4, 5, 7, 6)]
    normals = [(-1, 0, 0), (1, 0, 0), (0, -1, 0), (0, 1, 0), (0, 0, -1), (0, 0, 1)]
    return [(c[list(l)], np.array(n, dtype=np.float64), -1 - w)
            for w, (l, n) in enumerate(zip(loops, normals))]


def cell_weight(p, h, cells: Cells, j: int = 0) -> float:
    p = _f64(p)
    f0, f1 = int(cells.cell_face_off[j]), int(cells.cell_face_off[j + 1])
    fvo = _i64a(cells.face_vert_off[f0:f1 + 1])
    verts = _f64(cells.verts)
    nrm = _f64(cells.normals[f0:f1])
    return lib().orc_cell_weight(_ptr(p), float(h), f1 - f0, _ptr(fvo), _ptr(verts), _ptr(nrm))


def cell_weight_quadrature(p, h, cells: Cells, j: int = 0, tol: float = 1e-11) -> float:
    p = _f64(p)
    f0, f1 = int(cells.cell_face_off[j]), int(cells.cell_face_off[j + 1])
    nrm = _f64(cells.normals[f0:f1])
    off = _f64(cells.offsets()[f0:f1])
    return lib().orc_cell_weight_quadrature(_ptr(p), float(h), f1 - f0, _ptr(nrm), _ptr(off),
                                            float(tol))


def cell_distance(p, cells: Cells, j: int) -> float:
    p = _f64(p)
    f0, f1 = int(cells.cell_face_off[j]), int(cells.cell_face_off[j + 1])
    fvo = _i64a(cells.face_vert_off[f0:f1 + 1])
    return lib().orc_cell_distance(_ptr(p), f1 - f0, _ptr(fvo), _ptr(_f64(cells.verts)),
                                   _ptr(_f64(cells.normals[f0:f1])))


def voronoi(gx, gy, gz, box, cells=None, nthreads=None, max_faces=96, max_fv=768,
            batch=2048) -> Cells:
    """Brute-force Voronoi cells of the generators, clipped to the box."""
    gx, gy, gz, box = _f64(gx), _f64(gy), _f64(gz), _f64(box)
    ngen = gx.shape[0]
    ids = np.arange(ngen, dtype=np.int64) if cells is None else _i64a(cells)
    nt = nthreads or nthreads_default()
    cfo, fvo, V, N, NB, VOL = [np.zeros(1, np.int64)], [np.zeros(1, np.int64)], [], [], [], []
    nf_tot, nv_tot = 0, 0
    for b0 in range(0, ids.shape[0], batch):
        sub = _i64a(ids[b0:b0 + batch])
        nb = sub.shape[0]
        nface = np.zeros(nb, np.int64)
        nfv = np.zeros(nb, np.int64)
        fnbr = np.zeros(nb * max_faces, np.int64)
        fn = np.zeros((nb * max_faces, 3))
        fnv = np.zeros(nb * max_faces, np.int64)
        vv = np.zeros((nb * max_fv, 3))
        vol = np.zeros(nb)
        nover = lib().orc_voronoi_cells(ngen, _ptr(gx), _ptr(gy), _ptr(gz), _ptr(box), nb,
                                        _ptr(sub), max_faces, max_fv, _ptr(nface), _ptr(nfv),
                                        _ptr(fnbr), _ptr(fn), _ptr(fnv), _ptr(vv), _ptr(vol), nt)
        if nover:
            raise RuntimeError(f"oracle voronoi: {nover} cells overflowed the per-cell limits")
        for c in range(nb):
            k = int(nface[c])
            fs = slice(c * max_faces, c * max_faces + k)
            cfo.append(np.array([nf_tot + k]))
            fvo.append(nv_tot + np.cumsum(fnv[fs]))
            V.append(vv[c * max_fv: c * max_fv + int(nfv[c])])
            N.append(fn[fs])
            NB.append(fnbr[fs])
            nf_tot += k
            nv_tot += int(nfv[c])
        VOL.append(vol)
    gen = np.stack([gx[ids], gy[ids], gz[ids]], axis=1)
    return Cells(np.concatenate(cfo), np.concatenate(fvo), np.concatenate(V),
                 np.concatenate(N), np.concatenate(NB), np.concatenate(VOL), gen, ids)


@dataclass
class Pairs:
    pair_i: np.ndarray         # particle index, sorted by (cell, particle)
    pair_j: np.ndarray         # cell index (row of the Cells object)
    near: np.ndarray           # 1 when |dist - 2h| < 1e-9 h
    cell_pair_off: np.ndarray  # CSR offsets over cells

    @property
    def n(self) -> int:
        return int(self.pair_i.shape[0])


def find_pairs(x, y, z, h, cells: Cells, nthreads=None) -> Pairs:
    """All pairs with dist(x_i, V_j) < 2 h_i (exact predicate, every particle
    against every cell)."""
    x, y, z, h = _f64(x), _f64(y), _f64(z), _f64(h)
    nc = cells.ncell
    g = _f64(cells.gen)
    gx, gy, gz = _f64(g[:, 0]), _f64(g[:, 1]), _f64(g[:, 2])
    cfo, fvo = _i64a(cells.cell_face_off), _i64a(cells.face_vert_off)
    verts, nrm = _f64(cells.verts), _f64(cells.normals)
    count = np.zeros(nc, np.int64)
    nt = nthreads or nthreads_default()
    args = (x.shape[0], _ptr(x), _ptr(y), _ptr(z), _ptr(h), nc, _ptr(gx), _ptr(gy), _ptr(gz),
            _ptr(cfo), _ptr(fvo), _ptr(verts), _ptr(nrm))
    lib().orc_find_pairs(*args, _ptr(count), None, None, None, nt)
    off = np.zeros(nc + 1, np.int64)
    np.cumsum(count, out=off[1:])
    pi = np.zeros(int(off[-1]), np.int64)
    near = np.zeros(int(off[-1]), np.uint8)
    lib().orc_find_pairs(*args, _ptr(count), _ptr(off), _ptr(pi), _ptr(near), nt)
    pj = np.repeat(np.arange(nc, dtype=np.int64), count)
    return Pairs(pi, pj, near, off)


def map_exact(pairs: Pairs, x, y, z, h, cells: Cells, nthreads=None) -> np.ndarray:
    """w_ij for every pair by the signed face-pyramid decomposition."""
    x, y, z, h = _f64(x), _f64(y), _f64(z), _f64(h)
    pi, pj = _i64a(pairs.pair_i), _i64a(pairs.pair_j)
    w = np.zeros(pi.shape[0])
    lib().orc_map_exact(pi.shape[0], _ptr(pi), _ptr(pj), _ptr(x), _ptr(y), _ptr(z), _ptr(h),
                        _ptr(_i64a(cells.cell_face_off)), _ptr(_i64a(cells.face_vert_off)),
                        _ptr(_f64(cells.verts)), _ptr(_f64(cells.normals)), _ptr(w),
                        nthreads or nthreads_default())
    return w


def map_exact_list(pi, pj, x, y, z, h, cells: Cells, nthreads=None) -> np.ndarray:
    pi, pj = _i64a(pi), _i64a(pj)
    return map_exact(Pairs(pi, pj, np.zeros_like(pi, dtype=np.uint8), np.zeros(1, np.int64)),
                     x, y, z, h, cells, nthreads)


WORK_FIELDS = ("right_subtriangles", "add", "mul", "div", "sqrt", "transcendental")


def count_map_exact(pairs: Pairs, x, y, z, h, cells: Cells, nthreads=None):
    """map_exact with its algorithmic work counted per pair (count.cpp): the
    weights (bit-identical to map_exact's) and an (npairs, 6) array of counts
    in the order of WORK_FIELDS -- right sub-triangles evaluated, FP64
    additions/subtractions, multiplications, divisions, square roots and
    transcendental calls (atan2, asinh, pow) of the closed form."""
    global _count_lib
    if _count_lib is None:
        _count_lib = C.CDLL(_build_count())
        _count_lib.orc_count_map_exact.restype = None
        _count_lib.orc_count_map_exact.argtypes = [_i64, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _p, _i32]
    x, y, z, h = _f64(x), _f64(y), _f64(z), _f64(h)
    pi, pj = _i64a(pairs.pair_i), _i64a(pairs.pair_j)
    w = np.zeros(pi.shape[0])
    counts = np.zeros((pi.shape[0], 6), np.uint64)
    _count_lib.orc_count_map_exact(pi.shape[0], _ptr(pi), _ptr(pj), _ptr(x), _ptr(y), _ptr(z), _ptr(h),
                                   _ptr(_i64a(cells.cell_face_off)), _ptr(_i64a(cells.face_vert_off)),
                                   _ptr(_f64(cells.verts)), _ptr(_f64(cells.normals)), _ptr(w), _ptr(counts),
                                   nthreads or nthreads_default())
    return w, counts


def cell_density(pairs: Pairs, w, m, volume) -> np.ndarray:
    """rho_j = sum_i m_i w_ij / V_j, summed in the pair order (ascending i)."""
    nc = pairs.cell_pair_off.shape[0] - 1
    rho = np.zeros(nc)
    lib().orc_cell_density(nc, _ptr(_i64a(pairs.cell_pair_off)), _ptr(_i64a(pairs.pair_i)),
                           _ptr(_f64(w)), _ptr(_f64(m)), _ptr(_f64(volume)), _ptr(rho))
    return rho


def particle_weight_sum(pairs: Pairs, w, n) -> np.ndarray:
    """u_i = sum_j w_ij (partition of unity check), summed in ascending j."""
    order = np.lexsort((pairs.pair_j, pairs.pair_i))
    out = np.zeros(n)
    for k in order:
        out[pairs.pair_i[k]] += w[k]
    return out


def map_back_sums(pairs: Pairs, w, f_cell, n):
    """The two sums of the inverse mapping (Section 2.3) per particle,
    num_i = sum_j w_ij f_j and den_i = sum_j w_ij, over particle i's pairs in
    ascending j, one rounded product and one rounded addition per term
    (np.add.at applies the additions in index order)."""
    order = np.lexsort((pairs.pair_j, pairs.pair_i))
    pi = np.asarray(pairs.pair_i)[order]
    pj = np.asarray(pairs.pair_j)[order]
    wk = np.asarray(w, dtype=np.float64)[order]
    fk = np.asarray(f_cell, dtype=np.float64)[pj]
    num = np.zeros(n)
    den = np.zeros(n)
    np.add.at(num, pi, wk * fk)
    np.add.at(den, pi, wk)
    return num, den


def map_back(pairs: Pairs, w, f_cell, n) -> np.ndarray:
    """Inverse mapping (Section 2.3): f_i = sum_j w_ij f_j / sum_j w_ij, the
    kernel-weighted average of the cell values over particle i's cells
    (map_back_sums); NaN for particles without any pair."""
    num, den = map_back_sums(pairs, w, f_cell, n)
    with np.errstate(invalid="ignore", divide="ignore"):
        return num / den


def inherit(ps: "Pseudo", tree: "Tree", f_pseudo) -> np.ndarray:
    """Constituent inheritance (Section 2.5): the SPH particles a pseudo-particle
    stands for share its value.  Pseudo-particle a covers the Morton positions
    [first_a, first_a + count_a) of the tree's particle order, that is the
    particles perm[first_a .. first_a + count_a - 1] (a node's constituents,
    or the one extracted particle).  Returns one value per particle in the
    input order; raises if a particle is covered twice or not at all (the
    selection tiles the particles exactly once, Section 2.4.1)."""
    n = tree.perm.shape[0]
    f_pseudo = np.asarray(f_pseudo, dtype=np.float64)
    out = np.zeros(n)
    cover = np.zeros(n, np.int64)
    for a in range(ps.n):
        idx = tree.perm[int(ps.first[a]):int(ps.first[a]) + int(ps.count[a])]
        out[idx] = f_pseudo[a]
        cover[idx] += 1
    if np.any(cover != 1):
        raise ValueError(f"inherit: {int(np.sum(cover == 0))} particles uncovered, "
                         f"{int(np.sum(cover > 1))} covered more than once")
    return out


# ---------------------------------------------------------------------------
# Tree, selection, h-solver
# ---------------------------------------------------------------------------

@dataclass
class Tree:
    perm: np.ndarray
    label: np.ndarray
    level: np.ndarray
    parent: np.ndarray
    first: np.ndarray
    count: np.ndarray
    first_child: np.ndarray
    nchild: np.ndarray
    mass: np.ndarray
    msum: np.ndarray           # (nnode, 3) sums of m*x
    com: np.ndarray            # (nnode, 3)
    size: np.ndarray

    @property
    def nnode(self) -> int:
        return int(self.label.shape[0])


def morton_keys(x, y, z, box) -> np.ndarray:
    x, y, z, box = _f64(x), _f64(y), _f64(z), _f64(box)
    k = np.zeros(x.shape[0], np.uint64)
    lib().orc_morton_keys(x.shape[0], _ptr(x), _ptr(y), _ptr(z), _ptr(box), _ptr(k))
    return k


def build_tree(x, y, z, m, box, leaf_max=8) -> Tree:
    x, y, z, m, box = _f64(x), _f64(y), _f64(z), _f64(m), _f64(box)
    n = x.shape[0]
    cap = 4 * n + 64
    while True:
        perm = np.zeros(n, np.int64)
        arr = dict(label=np.zeros(cap, np.uint64), level=np.zeros(cap, np.int32),
                   parent=np.zeros(cap, np.int64), first=np.zeros(cap, np.int64),
                   count=np.zeros(cap, np.int64), first_child=np.zeros(cap, np.int64),
                   nchild=np.zeros(cap, np.int32))
        f = {k: np.zeros(cap) for k in ("mass", "mx", "my", "mz", "cx", "cy", "cz", "size")}
        nn = lib().orc_build_tree(n, _ptr(x), _ptr(y), _ptr(z), _ptr(m), _ptr(box), int(leaf_max),
                                  cap, _ptr(perm), *[_ptr(arr[k]) for k in arr],
                                  *[_ptr(f[k]) for k in f])
        if nn >= 0:
            break
        cap *= 4
    s = slice(0, nn)
    return Tree(perm, arr["label"][s], arr["level"][s], arr["parent"][s], arr["first"][s],
                arr["count"][s], arr["first_child"][s], arr["nchild"][s], f["mass"][s],
                np.stack([f["mx"][s], f["my"][s], f["mz"][s]], 1),
                np.stack([f["cx"][s], f["cy"][s], f["cz"][s]], 1), f["size"][s])


@dataclass
class Selection:
    kind: np.ndarray           # 0 node, 1 particle
    ref: np.ndarray            # node index, or Morton position of the particle
    pop_node: np.ndarray       # h-solver population (node indices)

    @property
    def n(self) -> int:
        return int(self.kind.shape[0])


def select(tree: Tree, sources, r_part, r_leaf, theta, force=None) -> Selection:
    """Adaptive tree-walk (Section 2.4.1, Eq. 4).  force: optional per-node flags
    from the refinement check (refine_fail): a flagged node is opened, a flagged
    leaf has its particles extracted."""
    src = _f64(np.asarray(sources).reshape(-1, 3))
    fz = None if force is None else np.ascontiguousarray(np.asarray(force, dtype=np.uint8))
    if fz is not None and fz.shape[0] != tree.nnode:
        raise ValueError("force: one flag per tree node")
    cap = tree.perm.shape[0] + tree.nnode + 8
    kind = np.zeros(cap, np.int32)
    ref = np.zeros(cap, np.int64)
    pop = np.zeros(cap, np.int64)
    npop = np.zeros(1, np.int64)
    com = tree.com
    nout = lib().orc_select(tree.nnode, _ptr(tree.nchild), _ptr(tree.first_child),
                            _ptr(tree.first), _ptr(tree.count), _ptr(_f64(com[:, 0])),
                            _ptr(_f64(com[:, 1])), _ptr(_f64(com[:, 2])), _ptr(tree.size),
                            src.shape[0], _ptr(src), float(r_part), float(r_leaf), float(theta),
                            cap, _ptr(kind), _ptr(ref), _ptr(pop), _ptr(npop),
                            None if fz is None else _ptr(fz))
    if nout < 0:
        raise RuntimeError("oracle select: output overflow")
    return Selection(kind[:nout].copy(), ref[:nout].copy(), pop[:int(npop[0])].copy())


def h_initial(tree: Tree, nodes, h_particle, h_fact):
    """h_0 = 2 h_fact s_node (Eq. 11); a one-particle node starts from its
    particle's own h."""
    nodes = np.asarray(nodes, dtype=np.int64)
    h0 = 2.0 * h_fact * tree.size[nodes]
    single = (tree.count[nodes] == 1) | (tree.size[nodes] == 0.0)
    if np.any(single):
        part = tree.perm[tree.first[nodes[single]]]
        h0[single] = np.asarray(h_particle)[part]
    return h0


def h_solve(pop_xyz, tgt_xyz, h0, h_fact=1.2, tol=1e-13, max_newton=50, nthreads=None):
    pop_xyz = np.asarray(pop_xyz, dtype=np.float64)
    tgt_xyz = np.asarray(tgt_xyz, dtype=np.float64)
    px, py, pz = (_f64(pop_xyz[:, k]) for k in range(3))
    tx, ty, tz = (_f64(tgt_xyz[:, k]) for k in range(3))
    h0 = _f64(h0)
    nt = tgt_xyz.shape[0]
    h = np.zeros(nt)
    st = np.zeros(nt, np.int32)
    it = np.zeros(nt, np.int32)
    lib().orc_h_solve(px.shape[0], _ptr(px), _ptr(py), _ptr(pz), nt, _ptr(tx), _ptr(ty), _ptr(tz),
                      _ptr(h0), float(h_fact), float(tol), int(max_newton), _ptr(h), _ptr(st),
                      _ptr(it), nthreads or nthreads_default())
    return h, st, it


@dataclass
class Pseudo:
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    h: np.ndarray
    m: np.ndarray
    origin: np.ndarray         # node label (>0) or -(particle index + 1)
    first: np.ndarray          # Morton range of constituents
    count: np.ndarray
    status: np.ndarray         # h-solver status (0 Newton, 1 bisection, 2 fallback, 3 particle)

    @property
    def n(self) -> int:
        return int(self.x.shape[0])


def make_pseudo_particles(x, y, z, m, h_particle, box, sources, r_part, r_leaf, theta,
                          h_fact=1.2, tol=1e-13, max_newton=50, leaf_max=8, nthreads=None,
                          solve=True, force=None, h0_above=0):
    """Tree build, adaptive tree-walk and node h-solver (Sections 2.2, 2.4);
    force: per-node refinement flags (see select).  With h0_above > 0 and
    more pseudo-particles than that (nodes and extracted particles), every
    node takes h_0 of Eq. 11 (status 2) without the neighbour search, as
    Section 2.4.2 does above 10^6 pseudo-particles."""
    t = build_tree(x, y, z, m, box, leaf_max)
    sel = select(t, sources, r_part, r_leaf, theta, force)
    x, y, z, m = (np.asarray(a, dtype=np.float64) for a in (x, y, z, m))
    hp = np.asarray(h_particle, dtype=np.float64)
    n = sel.n
    isn = sel.kind == 0
    nodes = sel.ref[isn]
    parts = t.perm[sel.ref[~isn]]
    px = np.empty(n); py = np.empty(n); pz = np.empty(n); pm = np.empty(n); ph = np.empty(n)
    org = np.empty(n, np.int64); first = np.empty(n, np.int64); cnt = np.empty(n, np.int64)
    st = np.full(n, 3, np.int32)
    px[isn], py[isn], pz[isn] = t.com[nodes, 0], t.com[nodes, 1], t.com[nodes, 2]
    pm[isn] = t.mass[nodes]
    org[isn] = t.label[nodes].astype(np.int64)
    first[isn], cnt[isn] = t.first[nodes], t.count[nodes]
    px[~isn], py[~isn], pz[~isn] = x[parts], y[parts], z[parts]
    pm[~isn] = m[parts]
    ph[~isn] = hp[parts]
    org[~isn] = -(parts + 1)
    first[~isn], cnt[~isn] = sel.ref[~isn], 1
    if h0_above > 0 and n > h0_above and nodes.shape[0]:
        ph[isn] = h_initial(t, nodes, hp, h_fact)
        st[isn] = 2
    elif solve and nodes.shape[0]:
        h0 = h_initial(t, nodes, hp, h_fact)
        hh, s, _ = h_solve(t.com[sel.pop_node], t.com[nodes], h0, h_fact, tol, max_newton,
                           nthreads)
        ph[isn] = hh
        st[isn] = s
    return Pseudo(px, py, pz, ph, pm, org, first, cnt, st), t, sel


# ---------------------------------------------------------------------------
# Lloyd regularisation of the sites (Section 2.3)
# ---------------------------------------------------------------------------

def cell_centroids(cells: Cells):
    """Centroid c_j = (1/V_j) integral over V_j of r d^3r of every stored cell,
    and the volume V_j, from the cell's faces.  Each face is fanned into
    triangles (v_0, v_k, v_k+1); each triangle with the generator g spans a
    tetrahedron of signed volume a.(b x c)/6 (a, b, c its corners relative
    to g) and centroid g + (a + b + c)/4.  The tetrahedra tile the convex
    cell, so the volume-weighted mean of their centroids is the cell's."""
    nc = cells.ncell
    cen = np.zeros((nc, 3))
    vol = np.zeros(nc)
    for j in range(nc):
        g = cells.gen[j]
        m1 = np.zeros(3)
        v6 = 0.0
        for verts, _, _ in cells.faces(j):
            a = verts[0] - g
            for k in range(1, verts.shape[0] - 1):
                b = verts[k] - g
                c = verts[k + 1] - g
                t6 = float(np.dot(a, np.cross(b, c)))
                v6 += t6
                m1 += t6 * (a + b + c)
        vol[j] = v6 / 6.0
        cen[j] = g + m1 / (4.0 * v6)
    return cen, vol


def lloyd(gx, gy, gz, box, iters=5, nthreads=None):
    """Lloyd's iteration (Section 2.3 applies five before the mapping): build
    the Voronoi cells clipped to the box and move every site to its cell's
    centroid, iters times.  Returns the sites after the last move."""
    g = np.stack([_f64(gx), _f64(gy), _f64(gz)], axis=1)
    for _ in range(iters):
        cells = voronoi(g[:, 0], g[:, 1], g[:, 2], box, nthreads=nthreads)
        cen, _ = cell_centroids(cells)
        g = np.empty_like(g)
        g[cells.cell_ids] = cen
    return g[:, 0].copy(), g[:, 1].copy(), g[:, 2].copy()


# ---------------------------------------------------------------------------
# Adaptive refinement (Section 2.4.1, Eq. 5)
# ---------------------------------------------------------------------------

def refine_limit(size, size_root, K):
    """Eq. 5: the neutral-fraction threshold of a node of size s,
    f_neu,limit = (1/K) (K - 1 / (s / s_root)); -inf for a node of size 0."""
    size = np.asarray(size, dtype=np.float64)
    with np.errstate(divide="ignore"):
        return (K - size_root / size) / K


def refine_fail(tree: Tree, nodes, f_neu, K):
    """Mask over nodes: under-resolved when f_neu < f_neu,limit(s_node) (Eq. 5).
    NaN (a pseudo-particle without pairs) does not fail."""
    nodes = np.asarray(nodes, dtype=np.int64)
    return np.asarray(f_neu) < refine_limit(tree.size[nodes], tree.size[0], K)


def refine(x, y, z, m, h_particle, box, sources, r_part, r_leaf, theta, cells: Cells, f_cell, K,
           max_iter=20, leaf_step=0.0, h_fact=1.2, tol=1e-13, leaf_max=8, nthreads=None):
    """The adaptive tree-walk iterations of Section 2.4.1: select, map, map the
    cells' neutral fraction back onto the pseudo-particles, flag the nodes that
    fail Eq. 5, and select again with the flagged internal nodes opened, until
    no node fails.

    A failing leaf cannot be opened.  With leaf_step > 0, as in Section 2.4.1
    and the runs of Section 3.3, r_part and r_leaf both grow by leaf_step for
    the next walk whenever some leaf fails; the leaf itself is not flagged.
    With leaf_step = 0 the failing leaf is flagged and its particles are
    extracted in the next walk, the local form of raising r_part for it.

    Returns (pseudo, tree, selection, force flags, iterations, f_neu per
    pseudo-particle of the last round, (r_part, r_leaf) of the last round)."""
    force = None
    for it in range(1, max_iter + 1):
        ps, t, sel = make_pseudo_particles(x, y, z, m, h_particle, box, sources, r_part, r_leaf, theta,
                                           h_fact=h_fact, tol=tol, leaf_max=leaf_max, nthreads=nthreads,
                                           force=force)
        if force is None:
            force = np.zeros(t.nnode, np.uint8)
        pairs = find_pairs(ps.x, ps.y, ps.z, ps.h, cells, nthreads)
        w = map_exact(pairs, ps.x, ps.y, ps.z, ps.h, cells, nthreads)
        fn = map_back(pairs, w, f_cell, ps.n)
        isn = sel.kind == 0
        nodes = sel.ref[isn]
        bad = nodes[refine_fail(t, nodes, fn[isn], K)]
        leaf = t.nchild[bad] == 0
        if leaf_step > 0:
            grow = bool(np.any(leaf))
            bad = bad[~leaf]
        else:
            grow = False
        new = bad[force[bad] == 0]
        if new.shape[0] == 0 and not grow:
            return ps, t, sel, force, it, fn, (r_part, r_leaf)
        force[new] = 1
        if grow:
            r_part += leaf_step
            r_leaf += leaf_step
    return ps, t, sel, force, max_iter, fn, (r_part, r_leaf)


# ---------------------------------------------------------------------------
# Bounded samples of a workload (the CPU baseline and the work counts)
# ---------------------------------------------------------------------------

def workload_sample(w, theta, ntarget=64, seed=7, pseudo=True, complete=False, nthreads=None):
    """A bounded sample of a workload built by the oracle alone: `ntarget`
    random pseudo-particles of the oracle's own tree and selection on the cloud
    (Sections 2.2, 2.4; nodes get h from the h-solver against the whole
    population) -- or random particles when the workload maps particles
    directly -- with the oracle's brute-force cells and pairs around them.
    complete=False takes the cells whose generators lie within 2h of a sampled
    particle (a subset of its pairs); complete=True takes every cell that can
    reach within 2h, from the bound |g - p| <= 4h + d_p (d_p the distance to
    the nearest generator), so the sampled particles' pair lists are whole.
    Returns ((x, y, z, h) of the sampled particles, cells, pairs)."""
    pr = w.params
    rng = np.random.default_rng(seed)
    if not pseudo:      # the particles themselves
        tg = np.sort(rng.choice(w.n, ntarget, replace=False))
        px, py, pz, h = w.x[tg], w.y[tg], w.z[tg], w.h[tg]
    else:
        ps, tree, sel = make_pseudo_particles(w.x, w.y, w.z, w.m, w.h, w.box, np.zeros((1, 3)), pr["r_part"],
                                              pr["r_leaf"], theta, h_fact=pr["h_fact"], solve=False)
        tg = np.sort(rng.choice(ps.n, ntarget, replace=False))
        h = ps.h[tg].copy()
        node = ps.origin[tg] > 0
        if node.any():
            ids = sel.ref[tg[node]]
            h0 = h_initial(tree, ids, w.h, pr["h_fact"])
            h[node] = h_solve(tree.com[sel.pop_node], tree.com[ids], h0, pr["h_fact"], 1e-13, 50,
                              nthreads)[0]
        px, py, pz = ps.x[tg], ps.y[tg], ps.z[tg]
    gen = np.stack([w.gx, w.gy, w.gz], 1)
    near = np.zeros(w.ngen, bool)
    for a in range(px.shape[0]):
        d2 = np.einsum("ij,ij->i", gen - (px[a], py[a], pz[a]), gen - (px[a], py[a], pz[a]))
        reach = 4.0 * h[a] + np.sqrt(d2.min()) if complete else 2.0 * h[a]
        near |= d2 < reach * reach + (1e-12 if complete else 0.0)
    cells = voronoi(w.gx, w.gy, w.gz, w.box, cells=np.flatnonzero(near), nthreads=nthreads)
    pairs = find_pairs(px, py, pz, h, cells, nthreads)
    return (px, py, pz, h), cells, pairs

