"""Python binding of the C ABI, with the same call names.

PyTorch supplies device memory and the CUDA stream; every computation runs in
``libexactmap.so``.  Inputs are CUDA tensors (float64 for coordinates,
masses, smoothing lengths; int32 for pair indices); outputs are new CUDA
tensors allocated by torch.
"""
from __future__ import annotations

import ctypes as C
from dataclasses import dataclass, fields, replace

import torch

from . import _native as N


@dataclass
class Params:
    """Method parameters (see em_params in include/exactmap.h)."""
    r_part: float = 0.05
    r_leaf: float = 0.1
    theta: float = 0.1
    h_fact: float = 1.2
    h_tol: float = 1e-13
    max_newton: int = 50
    precision: int = 0            # 0 FP64, 1 mixed FP32 / FP64
    fp64_threshold: float = 1e-5
    knn_k: int = 48
    leaf_max: int = 8
    block_pairs: int = 0
    h0_above: int = 0             # > 0: with more pseudo-particles than this, every node takes h_0 (Eq. 11)
    fp32_err_ulps: int = 8        # mixed mode: factor of the FP32 error estimate, in units of 2^-24
    fp32_variant: int = 0         # mixed mode: launch shape of the FP32 pass (map_autotune)

    def native(self) -> N.EmParams:
        p = N.EmParams()
        for f in fields(self):
            setattr(p, f.name, getattr(self, f.name))
        return p


def _ptr(t: torch.Tensor | None, dtype=None, n=None, name="tensor"):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if dtype is not None and t.dtype != dtype:
        raise TypeError(f"{name} must be {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() != n:
        raise ValueError(f"{name} must have {n} elements, got {t.numel()}")
    return C.c_void_p(t.data_ptr())


def _box(box):
    b = (C.c_double * 6)(*[float(v) for v in box])
    return C.cast(b, C.c_void_p), b


class Context:
    """Library context bound to a device and the current torch stream."""

    def __init__(self, device: int = 0, stream: torch.cuda.Stream | None = None):
        self.device = torch.device("cuda", device)
        self.stream = stream or torch.cuda.current_stream(self.device)
        h = C.c_void_p()
        N.call("em_ctx_create", C.byref(h), device, C.c_void_p(self.stream.cuda_stream))
        self.handle = h

    @property
    def launches(self) -> int:
        return int(N.lib().em_ctx_launch_count(self.handle))

    def sync(self):
        N.call("em_ctx_sync", self.handle)

    def set_timing(self, on: bool = True):
        """Record CUDA events around the map_exact kernels (see map_times)."""
        N.call("em_ctx_set_timing", self.handle, int(bool(on)))

    def map_times(self):
        """(main pass ms, FP64 recompute ms) of the last map_exact while timing was on."""
        a, b = C.c_double(), C.c_double()
        N.call("em_ctx_map_times", self.handle, C.byref(a), C.byref(b))
        return a.value, b.value

    def measure_peaks(self) -> dict:
        """Measured FP32 and FP64 FMA rates (TFLOP/s), special-function rate
        (Top/s), SM count and maximum SM clock (MHz) of the device."""
        out = (C.c_double * 5)()
        N.call("em_measure_peaks", self.handle, C.cast(out, C.c_void_p))
        return dict(fp32_tflops=out[0], fp64_tflops=out[1], xu_tops=out[2], sm_count=int(out[3]),
                    sm_clock_mhz=out[4])

    def close(self):
        if getattr(self, "handle", None):
            N.lib().em_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def empty(self, n, dtype=torch.float64):
        return torch.empty(int(n), dtype=dtype, device=self.device)


class _Handle:
    _destroy = ""

    def __init__(self, ctx: Context, handle: C.c_void_p):
        self.ctx = ctx
        self.handle = handle

    def close(self):
        if getattr(self, "handle", None):
            getattr(N.lib(), self._destroy)(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Tree(_Handle):
    """The octree of build_tree (Section 2.2.1): info() gives (particles,
    nodes, depth); get() copies out the Morton permutation and, per node,
    label, level, parent, first particle, count, first child, children, mass,
    centre of mass and size."""
    _destroy = "tree_destroy"

    def info(self):
        n, nn, depth = C.c_int64(), C.c_int64(), C.c_int32()
        N.call("tree_info", self.handle, C.byref(n), C.byref(nn), C.byref(depth))
        return n.value, nn.value, depth.value

    def get(self):
        n, nn, _ = self.info()
        e = self.ctx.empty
        out = dict(perm=e(n, torch.int32), label=e(nn, torch.int64), level=e(nn, torch.int32),
                   parent=e(nn, torch.int32), first=e(nn, torch.int32), count=e(nn, torch.int32),
                   first_child=e(nn, torch.int32), nchild=e(nn, torch.int32), mass=e(nn),
                   com=e(3 * nn), size=e(nn))
        N.call("tree_get", self.ctx.handle, self.handle,
               *[_ptr(out[k]) for k in ("perm", "label", "level", "parent", "first", "count",
                                        "first_child", "nchild", "mass", "com", "size")])
        out["com"] = out["com"].view(nn, 3)
        return out


class Pseudo(_Handle):
    """The pseudo-particles of make_pseudo_particles (Section 2.4): info()
    gives (count, the four solver status counts); get() copies out position,
    h, mass, origin (the node label, > 0, or -(particle index + 1) for an
    extracted particle), the Morton range of the
    constituents (first, count) and the solver status."""
    _destroy = "pseudo_destroy"

    def info(self):
        n = C.c_int64()
        st = (C.c_int64 * 4)()
        N.call("pseudo_info", self.handle, C.byref(n), st)
        return n.value, list(st)

    def get(self):
        n, _ = self.info()
        e = self.ctx.empty
        out = dict(x=e(n), y=e(n), z=e(n), h=e(n), m=e(n), origin=e(n, torch.int64),
                   first=e(n, torch.int32), count=e(n, torch.int32), status=e(n, torch.int32))
        N.call("pseudo_get", self.ctx.handle, self.handle,
               *[_ptr(out[k]) for k in ("x", "y", "z", "h", "m", "origin", "first", "count",
                                        "status")])
        return out


class Voronoi(_Handle):
    """The cells of build_voronoi (Section 2.3), clipped to the box: info()
    gives (cells, faces, face-vertices); get() copies out the CSR offsets,
    vertices (counter-clockwise seen from outside), outward normals,
    neighbours (negative for a box face) and volumes."""
    _destroy = "voronoi_destroy"

    def info(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        N.call("voronoi_info", self.handle, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    def get(self):
        nc, nf, nfv = self.info()
        e = self.ctx.empty
        out = dict(cell_face_off=e(nc + 1, torch.int64), face_vert_off=e(nf + 1, torch.int64),
                   verts=e(3 * nfv), normals=e(3 * nf), nbr=e(nf, torch.int64), volume=e(nc))
        N.call("voronoi_get", self.ctx.handle, self.handle,
               *[_ptr(out[k]) for k in ("cell_face_off", "face_vert_off", "verts", "normals",
                                        "nbr", "volume")])
        out["verts"] = out["verts"].view(nfv, 3)
        out["normals"] = out["normals"].view(nf, 3)
        return out


class Pairs(_Handle):
    """A particle-cell pair list sorted by (cell, particle): info() gives
    (pairs, particles, cells); get() copies out pair_i, pair_j, the near
    flags (within 1e-9 h of the 2h boundary) and the cells' pair offsets."""
    _destroy = "pairs_destroy"

    def info(self):
        a, b, c = C.c_int64(), C.c_int64(), C.c_int64()
        N.call("pairs_info", self.handle, C.byref(a), C.byref(b), C.byref(c))
        return a.value, b.value, c.value

    @property
    def n(self) -> int:
        return self.info()[0]

    def get(self):
        npairs, _, nc = self.info()
        e = self.ctx.empty
        out = dict(pair_i=e(npairs, torch.int32), pair_j=e(npairs, torch.int32),
                   near=e(npairs, torch.uint8), cell_pair_off=e(nc + 1, torch.int64))
        N.call("pairs_get", self.ctx.handle, self.handle,
               *[_ptr(out[k]) for k in ("pair_i", "pair_j", "near", "cell_pair_off")])
        return out


f64 = torch.float64


def build_tree(ctx: Context, x, y, z, m, box, leaf_max: int = 8) -> Tree:
    """Morton octree of the particles (x, y, z, m: FP64 device tensors) in box
    (xlo, xhi, ylo, yhi, zlo, zhi), at most leaf_max particles per leaf, with
    node mass, centre of mass and size (Section 2.2.1)."""
    n = x.numel()
    h = C.c_void_p()
    bp, _keep = _box(box)
    N.call("build_tree", ctx.handle, n, _ptr(x, f64, n, "x"), _ptr(y, f64, n, "y"),
           _ptr(z, f64, n, "z"), _ptr(m, f64, n, "m"), bp, int(leaf_max), C.byref(h))
    return Tree(ctx, h)


def make_pseudo_particles(ctx: Context, tree: Tree, h_particle, sources, params: Params,
                          force: torch.Tensor | None = None) -> Pseudo:
    """force: optional uint8 flags, one per tree node (refine_check), for
    make_pseudo_particles_forced."""
    src = [float(v) for v in torch.as_tensor(sources, dtype=torch.float64).reshape(-1).tolist()]
    arr = (C.c_double * len(src))(*src)
    p = params.native()
    h = C.c_void_p()
    n, nnode, _ = tree.info()
    if force is None:
        N.call("make_pseudo_particles", ctx.handle, tree.handle, _ptr(h_particle, f64, n, "h"),
               len(src) // 3, C.cast(arr, C.c_void_p), C.byref(p), C.byref(h),
               allow=(N.EM_OK, N.EM_ENOTCONV))
    else:
        N.call("make_pseudo_particles_forced", ctx.handle, tree.handle, _ptr(h_particle, f64, n, "h"),
               len(src) // 3, C.cast(arr, C.c_void_p), C.byref(p), _ptr(force, torch.uint8, nnode, "force"),
               C.byref(h), allow=(N.EM_OK, N.EM_ENOTCONV))
    return Pseudo(ctx, h)


def refine_check(ctx: Context, ps: Pseudo, tree: Tree, f_neu, K: float, force: torch.Tensor,
                 flag_leaves: bool = True) -> tuple[int, int]:
    """Flags (in force) the node pseudo-particles that fail Eq. 5, leaves only
    with flag_leaves; returns (newly flagged nodes, failing leaves)."""
    n, _ = ps.info()
    _, nnode, _ = tree.info()
    k, nl = C.c_int64(), C.c_int64()
    N.call("refine_check", ctx.handle, ps.handle, tree.handle, _ptr(f_neu, f64, n, "f_neu"), float(K),
           int(bool(flag_leaves)), _ptr(force, torch.uint8, nnode, "force"), C.byref(k), C.byref(nl))
    return k.value, nl.value


def refine(ctx: Context, tree: Tree, h_particle, sources, params: Params, vor: "Voronoi", f_cell, K: float,
           max_iter: int = 20, leaf_step: float = 0.0):
    """The iteration of Section 2.4.1 as a sequence of library calls:
    make_pseudo_particles(_forced), find_pairs, map_exact, map_back of the
    cells' neutral fraction f_cell, refine_check; until no node fails Eq. 5
    anew.  A failing leaf is flagged for extraction (leaf_step = 0) or, with
    leaf_step > 0, raises r_part and r_leaf by leaf_step for the next walk
    (Sections 2.4.1 and 3.3).  Returns (pseudo, pairs, w, force, iterations,
    f_neu, (r_part, r_leaf) of the last walk)."""
    _, nnode, _ = tree.info()
    force = torch.zeros(nnode, dtype=torch.uint8, device=ctx.device)
    p = replace(params)
    for it in range(1, max_iter + 1):
        ps = make_pseudo_particles(ctx, tree, h_particle, sources, p, force)
        g = ps.get()
        pr = find_pairs(ctx, g["x"], g["y"], g["z"], g["h"], vor)
        w, _, _, _ = map_exact(ctx, pr, g["x"], g["y"], g["z"], g["h"], g["m"], vor, p)
        f_neu, _ = map_back(ctx, pr, w, f_cell)
        nnew, nleaf = refine_check(ctx, ps, tree, f_neu, K, force, flag_leaves=leaf_step <= 0)
        grow = leaf_step > 0 and nleaf > 0
        if nnew == 0 and not grow:
            return ps, pr, w, force, it, f_neu, (p.r_part, p.r_leaf)
        if grow:
            p.r_part += leaf_step
            p.r_leaf += leaf_step
    return ps, pr, w, force, max_iter, f_neu, (p.r_part, p.r_leaf)


def build_voronoi(ctx: Context, gx, gy, gz, box, params: Params | None = None) -> Voronoi:
    """The Voronoi cells of the generators (gx, gy, gz: FP64 device tensors),
    clipped to box, with the derived geometry map_exact uses (Section 2.3).
    Generators outside the box, or two at one position, are rejected."""
    n = gx.numel()
    p = (params or Params()).native()
    h = C.c_void_p()
    bp, _keep = _box(box)
    N.call("build_voronoi", ctx.handle, n, _ptr(gx, f64, n, "gx"), _ptr(gy, f64, n, "gy"),
           _ptr(gz, f64, n, "gz"), bp, C.byref(p), C.byref(h))
    return Voronoi(ctx, h)


def build_voronoi_cells(ctx: Context, gx, gy, gz, box, cell_begin: int, cell_end: int,
                        params: Params | None = None) -> Voronoi:
    """The cells [cell_begin, cell_end) only (one rank of a spatial split)."""
    n = gx.numel()
    p = (params or Params()).native()
    h = C.c_void_p()
    bp, _keep = _box(box)
    N.call("build_voronoi_cells", ctx.handle, n, _ptr(gx, f64, n, "gx"), _ptr(gy, f64, n, "gy"),
           _ptr(gz, f64, n, "gz"), bp, C.byref(p), int(cell_begin), int(cell_end), C.byref(h))
    return Voronoi(ctx, h)


def voronoi_centroids(ctx: Context, vor: Voronoi):
    """Centroid of every cell (Section 2.3, the move of Lloyd's iteration),
    as three device tensors in generator order."""
    nc, _, _ = vor.info()
    cx, cy, cz = ctx.empty(nc), ctx.empty(nc), ctx.empty(nc)
    N.call("voronoi_centroids", ctx.handle, vor.handle, _ptr(cx, f64, nc), _ptr(cy, f64, nc), _ptr(cz, f64, nc))
    return cx, cy, cz


def lloyd(ctx: Context, gx, gy, gz, box, iters: int = 5, params: Params | None = None):
    """Lloyd's iteration on the sites (Section 2.3: five before the mapping),
    in place on the device tensors gx, gy, gz, which are returned."""
    n = gx.numel()
    p = (params or Params()).native()
    bp, _keep = _box(box)
    N.call("lloyd", ctx.handle, n, _ptr(gx, f64, n, "gx"), _ptr(gy, f64, n, "gy"), _ptr(gz, f64, n, "gz"),
           bp, int(iters), C.byref(p))
    return gx, gy, gz


def _snapshot_record(e, sn):
    """Fill the em_snapshot record e from a snapshot dict (see map_batch);
    returns the host source array to keep alive and the output tensors."""
    x = sn["x"]
    np_, ng = x.numel(), sn["gx"].numel()
    dev = x.device
    rho = torch.empty(ng, dtype=f64, device=dev)
    f = torch.empty(np_, dtype=f64, device=dev) if sn.get("f_cell") is not None else None
    src = [float(v) for v in torch.as_tensor(sn["sources"], dtype=f64).reshape(-1).tolist()]
    hsrc = (C.c_double * len(src))(*src)
    e.n, e.ngen = np_, ng
    for name in ("x", "y", "z", "m", "h"):
        setattr(e, "d_" + name, _ptr(sn[name], f64, np_, name))
    for name in ("gx", "gy", "gz"):
        setattr(e, "d_" + name, _ptr(sn[name], f64, ng, name))
    for i, b in enumerate(sn["box"]):
        e.box[i] = float(b)
    e.nsrc = len(src) // 3
    e.h_src = C.cast(hsrc, C.c_void_p)
    e.d_f_cell = _ptr(sn.get("f_cell"), f64, ng, "f_cell")
    e.d_rho = _ptr(rho, f64, ng)
    e.d_f = _ptr(f, f64, np_) if f is not None else None
    return hsrc, (rho, f)


class Batch:
    """The batch as a handle (map_batch_create / add / run / get): snapshots
    added one at a time (dicts as for map_batch), mapped together by run().
    The snapshots' tensors must stay alive until a run that maps them
    returns; the handle keeps references to them."""

    def __init__(self, device: int, params: Params, nworkers: int = 4):
        self._p = params.native()
        h = C.c_void_p()
        N.call("map_batch_create", int(device), C.byref(self._p), int(nworkers), C.byref(h))
        self.handle = h
        self._keep, self._outs = [], []

    def add(self, snapshot) -> int:
        rec = N.EmSnapshot()
        hsrc, out = _snapshot_record(rec, snapshot)
        idx = C.c_int32()
        N.call("map_batch_add", self.handle, C.byref(rec), C.byref(idx))
        self._keep.append((hsrc, snapshot))
        self._outs.append(out)
        return idx.value

    def run(self, tune: bool = False, info: dict | None = None):
        """Map every snapshot added so far; returns the results as map_batch
        does (one dict per snapshot, and the kernel launches)."""
        launches = C.c_int64()
        variant = C.c_int32()
        ms = (C.c_double * 2)()
        rc = N.lib().map_batch_run(self.handle, int(bool(tune)), C.byref(variant), C.cast(ms, C.c_void_p),
                                   C.byref(launches))
        if info is not None:
            info["variant"] = variant.value
            info["map_ms"] = (ms[0], ms[1])
        res = [dict(rho=self._outs[k][0], f=self._outs[k][1], **self.get(k)) for k in range(len(self._outs))]
        if rc != N.EM_OK:
            err = N.NativeError("map_batch_run", rc, N.lib().em_last_error().decode(errors="replace"))
            err.results = res
            raise err
        return res, launches.value

    def get(self, index: int) -> dict:
        rec = N.EmSnapshot()
        N.call("map_batch_get", self.handle, int(index), C.byref(rec))
        return dict(npseudo=rec.npseudo, npairs=rec.npairs, nfp64=rec.nfp64, status=rec.status)

    def __del__(self):
        h = getattr(self, "handle", None)
        if h is not None and h.value:
            N.lib().map_batch_destroy(h)
            self.handle = None


def map_batch(device: int, snapshots, params: Params, nworkers: int = 4, tune: bool = False, info: dict | None = None):
    """Independent snapshots through the whole path: build_tree ...
    find_pairs per snapshot on nworkers host threads with a stream each, then
    one map_exact over all snapshots' pairs, and map_back when a cell field is
    given.  snapshots: dicts with device tensors x, y, z, m, h, gx, gy, gz, box
    (6 numbers), sources ((k, 3) numbers) and optionally f_cell.  tune: pick
    the FP32 pass's launch shape on the batch (map_autotune).  info (optional
    dict) receives the launch shape used ("variant") and the mapping's device
    milliseconds ("map_ms": main pass, FP64 recompute).
    Returns one dict per snapshot: rho, f (or None), npseudo, npairs, nfp64,
    status, and the total kernel launches."""
    n = len(snapshots)
    arr = (N.EmSnapshot * max(n, 1))()
    keep, outs = [], []
    for k, sn in enumerate(snapshots):
        hsrc, out = _snapshot_record(arr[k], sn)
        keep.append(hsrc)
        outs.append(out)
    p = params.native()
    launches = C.c_int64()
    variant = C.c_int32()
    ms = (C.c_double * 2)()
    rc = N.lib().map_batch(int(device), n, arr, C.byref(p), int(nworkers), int(bool(tune)), C.byref(variant),
                           C.cast(ms, C.c_void_p), C.byref(launches))
    if info is not None:
        info["variant"] = variant.value
        info["map_ms"] = (ms[0], ms[1])
    res = [dict(rho=outs[k][0], f=outs[k][1], npseudo=arr[k].npseudo, npairs=arr[k].npairs,
                nfp64=arr[k].nfp64, status=arr[k].status) for k in range(n)]
    if rc != N.EM_OK:
        err = N.NativeError("map_batch", rc, N.lib().em_last_error().decode(errors="replace"))
        err.results = res   # the snapshots that did finish keep their outputs
        raise err
    return res, launches.value


def voronoi_from_cells(ctx: Context, gen, cell_face_off, face_vert_off, verts, normals, nbr,
                       volume) -> Voronoi:
    """A Voronoi handle from cells built elsewhere (CSR layout as in
    Voronoi.get; nbr may be None), with the derived geometry map_exact uses."""
    nc = cell_face_off.numel() - 1
    nf = face_vert_off.numel() - 1
    nfv = verts.numel() // 3
    h = C.c_void_p()
    N.call("voronoi_from_cells", ctx.handle, nc, nf, nfv, _ptr(gen, f64, 3 * nc, "gen"),
           _ptr(cell_face_off, torch.int64, nc + 1), _ptr(face_vert_off, torch.int64, nf + 1),
           _ptr(verts, f64, 3 * nfv), _ptr(normals, f64, 3 * nf),
           _ptr(nbr, torch.int64, nf) if nbr is not None else None, _ptr(volume, f64, nc),
           C.byref(h))
    return Voronoi(ctx, h)


def find_pairs(ctx: Context, x, y, z, h_, vor: Voronoi) -> Pairs:
    """Every pair (i, j) whose kernel support reaches the cell:
    dist(x_i, V_j) < 2 h_i (Section 2.3), sorted by (j, i)."""
    n = x.numel()
    h = C.c_void_p()
    npairs = C.c_int64()
    N.call("find_pairs", ctx.handle, n, _ptr(x, f64, n, "x"), _ptr(y, f64, n, "y"),
           _ptr(z, f64, n, "z"), _ptr(h_, f64, n, "h"), vor.handle, C.byref(h), C.byref(npairs))
    return Pairs(ctx, h)


def find_pairs_plan(ctx: Context, x, y, z, h_, vor: Voronoi, chunk_capacity: int):
    """Cell ranges whose pairs number at most chunk_capacity each: returns
    (bounds as a list of ncell-range ends, starting with 0, total pairs)."""
    n = x.numel()
    nc = vor.info()[0]
    bounds = (C.c_int64 * (nc + 1))()
    nch = C.c_int64()
    tot = C.c_int64()
    N.call("find_pairs_plan", ctx.handle, n, _ptr(x, f64, n, "x"), _ptr(y, f64, n, "y"), _ptr(z, f64, n, "z"),
           _ptr(h_, f64, n, "h"), vor.handle, int(chunk_capacity), C.cast(bounds, C.c_void_p), C.byref(nch),
           C.byref(tot))
    return [bounds[c] for c in range(nch.value + 1)], tot.value


def find_pairs_cells(ctx: Context, x, y, z, h_, vor: Voronoi, cell_begin: int, cell_end: int,
                     npairs_hint: int = 0) -> Pairs:
    """The pairs of the cells [cell_begin, cell_end) only (the streamed form)."""
    n = x.numel()
    h = C.c_void_p()
    npairs = C.c_int64()
    N.call("find_pairs_cells", ctx.handle, n, _ptr(x, f64, n, "x"), _ptr(y, f64, n, "y"),
           _ptr(z, f64, n, "z"), _ptr(h_, f64, n, "h"), vor.handle, int(cell_begin), int(cell_end),
           int(npairs_hint), C.byref(h), C.byref(npairs))
    return Pairs(ctx, h)


def pairs_from_list(ctx: Context, pair_i, pair_j, np_: int, vor: Voronoi) -> Pairs:
    """A pair handle from a given list (int32 device tensors, sorted by
    (pair_j, pair_i)) over np_ particles and vor's cells; an unsorted list or
    an index out of range is rejected."""
    n = pair_i.numel()
    h = C.c_void_p()
    N.call("pairs_from_list", ctx.handle, n, _ptr(pair_i, torch.int32, n, "pair_i"),
           _ptr(pair_j, torch.int32, n, "pair_j"), int(np_), vor.handle, C.byref(h))
    return Pairs(ctx, h)


def map_exact(ctx: Context, pairs: Pairs, x, y, z, h_, m, vor: Voronoi, params: Params,
              want_wsum: bool = True, out=None, want_count: bool = True):
    """Returns (w per pair, rho per cell, sum_j w_ij per particle or None, #pairs in FP64).
    The count makes the call wait for the mixed pass; want_count=False leaves
    it asynchronous and returns None for the count."""
    npairs, np_, nc = pairs.info()
    if out is None:
        out = (ctx.empty(npairs), ctx.empty(nc), ctx.empty(np_) if want_wsum else None)
    w, rho, wsum = out
    nfp64 = C.c_int64()
    p = params.native()
    N.call("map_exact", ctx.handle, pairs.handle, _ptr(x, f64, np_, "x"), _ptr(y, f64, np_, "y"),
           _ptr(z, f64, np_, "z"), _ptr(h_, f64, np_, "h"), _ptr(m, f64, np_, "m"), vor.handle,
           C.byref(p), _ptr(w, f64, npairs), _ptr(rho, f64, nc), _ptr(wsum),
           C.byref(nfp64) if want_count else None)
    return w, rho, wsum, nfp64.value if want_count else None


FP32_VARIANTS = 4


def map_autotune(ctx: Context, pairs: Pairs, x, y, z, h_, vor: Voronoi, params: Params):
    """The fastest launch shape of map_exact's FP32 pass on these pairs:
    (variant for Params.fp32_variant, milliseconds of each variant)."""
    npairs, np_, _ = pairs.info()
    best = C.c_int32()
    ms = (C.c_double * FP32_VARIANTS)()
    p = params.native()
    N.call("map_autotune", ctx.handle, pairs.handle, _ptr(x, f64, np_, "x"), _ptr(y, f64, np_, "y"),
           _ptr(z, f64, np_, "z"), _ptr(h_, f64, np_, "h"), vor.handle, C.byref(p), C.byref(best),
           C.cast(ms, C.c_void_p))
    return best.value, list(ms)


def autotune_cached(ctx: Context, key: str, cache_path: str, tune):
    """A tuned variant from a JSON cache keyed by device name and workload
    key, or tune() (returning (variant, ms list)) and store its result."""
    import json
    import os
    dev = torch.cuda.get_device_name(ctx.device)
    cache = {}
    if cache_path and os.path.exists(cache_path):
        with open(cache_path) as f:
            cache = json.load(f)
    hit = cache.get(dev, {}).get(key)
    if hit is not None:
        return int(hit["variant"]), hit.get("ms"), True
    variant, ms = tune()
    if cache_path:
        cache.setdefault(dev, {})[key] = {"variant": int(variant), "ms": ms}
        os.makedirs(os.path.dirname(os.path.abspath(cache_path)), exist_ok=True)
        with open(cache_path, "w") as f:
            json.dump(cache, f, indent=1)
    return int(variant), ms, False


def map_exact_noalloc(ctx: Context, pairs: Pairs, x, y, z, h_, m, vor: Voronoi, params: Params,
                      out, want_count: bool = True):
    """map_exact into caller-supplied outputs out = (w, rho, wsum or None),
    without any device allocation by the library, for callers whose device
    memory is all owned by their own pool or that cannot take an allocation's
    synchronisation each step (at most NOALLOC_MAX_PAIRS pairs; calls that
    overlap on one device race on the library's fixed scratch array).
    Returns (w, rho, wsum, #pairs in FP64 or None)."""
    npairs, np_, nc = pairs.info()
    w, rho, wsum = out
    nfp64 = C.c_int64()
    p = params.native()
    N.call("map_exact_noalloc", ctx.handle, pairs.handle, _ptr(x, f64, np_, "x"), _ptr(y, f64, np_, "y"),
           _ptr(z, f64, np_, "z"), _ptr(h_, f64, np_, "h"), _ptr(m, f64, np_, "m"), vor.handle,
           C.byref(p), _ptr(w, f64, npairs), _ptr(rho, f64, nc), _ptr(wsum, f64, np_),
           C.byref(nfp64) if want_count else None)
    return w, rho, wsum, nfp64.value if want_count else None


NOALLOC_MAX_PAIRS = 1 << 20


def map_back_sums(ctx: Context, pairs: Pairs, w, f_cell, num, den):
    """Adds sum_j w_ij f_j to num and sum_j w_ij to den (device tensors, one
    entry per (pseudo-)particle) over the pairs given."""
    npairs, np_, nc = pairs.info()
    N.call("map_back_sums", ctx.handle, pairs.handle, _ptr(w, f64, npairs), _ptr(f_cell, f64, nc),
           _ptr(num, f64, np_, "num"), _ptr(den, f64, np_, "den"))
    return num, den


def inherit(ctx: Context, pseudo: Pseudo, tree: Tree, f_pseudo):
    """Each SPH particle takes its pseudo-particle's value (Section 2.5)."""
    n, _, _ = tree.info()
    fp = ctx.empty(n)
    N.call("inherit", ctx.handle, pseudo.handle, tree.handle, _ptr(f_pseudo, f64, pseudo.info()[0], "f_pseudo"),
           _ptr(fp))
    return fp


def map_back(ctx: Context, pairs: Pairs, w, f_cell, pseudo: Pseudo | None = None,
             tree: Tree | None = None):
    """Returns (f per (pseudo-)particle, f per SPH particle or None)."""
    npairs, np_, nc = pairs.info()
    f = ctx.empty(np_)
    fp = None
    if pseudo is not None:
        n, _, _ = tree.info()
        fp = ctx.empty(n)
    N.call("map_back", ctx.handle, pairs.handle, _ptr(w, f64, npairs), _ptr(f_cell, f64, nc),
           _ptr(f), pseudo.handle if pseudo is not None else None,
           tree.handle if tree is not None else None, _ptr(fp))
    return f, fp
