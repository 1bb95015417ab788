"""Pins of the oracle's octree, adaptive tree-walk, node h-solver and inverse
mapping: tree invariants, label arithmetic, an independent per-node statement
of the walk, the h-solver residual and its closed-form limits.  CPU only."""
import math

import numpy as np
import pytest

from paper_2410_15227_gb300 import inputs


def morton_numpy(x, y, z, box):
    """Morton keys written out independently: 21-bit quantisation, x bit highest."""
    def q(v, lo, hi):
        s = 2097152.0 / (hi - lo)
        return np.clip(np.floor((v - lo) * s), 0, 2097151).astype(np.uint64)
    ix, iy, iz = q(x, box[0], box[1]), q(y, box[2], box[3]), q(z, box[4], box[5])
    key = np.zeros(x.shape[0], np.uint64)
    for b in range(21):
        for v, sh in ((ix, 2), (iy, 1), (iz, 0)):
            key |= ((v >> np.uint64(b)) & np.uint64(1)) << np.uint64(3 * b + sh)
    return key


@pytest.fixture(scope="module")
def cloud():
    w = inputs.sphere_workload(6000, 600, 1.0, seed=21, field_seed=21)
    return w


@pytest.fixture(scope="module")
def tree(orc, cloud):
    w = cloud
    return orc.build_tree(w.x, w.y, w.z, w.m, w.box, 8)


def test_morton_keys(orc, cloud):
    w = cloud
    assert np.array_equal(orc.morton_keys(w.x, w.y, w.z, w.box), morton_numpy(w.x, w.y, w.z, w.box))


def test_tree_partitions_particles(tree, cloud):
    t = tree
    n = cloud.n
    leaves = t.nchild == 0
    cover = np.zeros(n, np.int64)
    for f, c in zip(t.first[leaves], t.count[leaves]):
        cover[f:f + c] += 1
    assert np.all(cover == 1)
    assert np.all((t.count[leaves] <= 8) | (t.level[leaves] == 21))
    assert np.array_equal(np.sort(t.perm), np.arange(n))
    for a in np.nonzero(~leaves)[0][:500]:
        cs = slice(t.first_child[a], t.first_child[a] + t.nchild[a])
        assert t.count[cs].sum() == t.count[a]
        assert t.first[cs][0] == t.first[a]
        assert np.all(t.first[cs][1:] == t.first[cs][:-1] + t.count[cs][:-1])
        assert np.all(t.parent[cs] == a)


def test_label_arithmetic(tree, cloud):
    # root 1; ancestor k levels up = label >> 3k; level = (bit length - 1) / 3
    t = tree
    assert t.label[0] == 1
    for a in range(1, t.nnode):
        assert t.label[a] >> np.uint64(3) == t.label[t.parent[a]]
        assert (int(t.label[a]).bit_length() - 1) // 3 == t.level[a]
    keys = morton_numpy(cloud.x, cloud.y, cloud.z, cloud.box)[t.perm]
    assert np.all(np.diff(keys.astype(np.float64)) >= 0)
    for a in range(0, t.nnode, 7):
        L = int(t.level[a])
        pre = int(t.label[a]) - (1 << (3 * L))
        ks = keys[t.first[a]:t.first[a] + t.count[a]] >> np.uint64(3 * (21 - L))
        assert np.all(ks == pre)
    # breadth-first numbering: levels non-decreasing, labels increasing within a level
    assert np.all(np.diff(t.level) >= 0)
    same = t.level[1:] == t.level[:-1]
    assert np.all(np.diff(t.label.astype(np.float64))[same] > 0)


def test_node_mass_com_size(tree, cloud):
    w, t = cloud, tree
    p = np.stack([w.x, w.y, w.z], 1)[t.perm]
    m = w.m[t.perm]
    for a in range(t.nnode):
        s = slice(t.first[a], t.first[a] + t.count[a])
        M = m[s].sum()
        assert abs(t.mass[a] - M) <= 1e-14 * M
        com = (m[s, None] * p[s]).sum(0) / M
        assert np.allclose(t.com[a], com, rtol=0, atol=1e-14)
        d = p[s] - t.com[a]
        assert t.size[a] == np.sqrt(d[:, 0] * d[:, 0] + d[:, 1] * d[:, 1] + d[:, 2] * d[:, 2]).max()


def _select_per_node(t, src, r_part, r_leaf, theta):
    """Independent statement of the walk: a node is reached iff every ancestor is
    opened; a reached internal node is selected iff not opened; a reached leaf is
    selected, or replaced by its particles inside r_part."""
    d2 = ((t.com[:, None, :] - np.asarray(src)[None, :, :]) ** 2).sum(2).min(1)
    dx = t.com[:, 0:1] - np.asarray(src)[None, :, 0]
    dy = t.com[:, 1:2] - np.asarray(src)[None, :, 1]
    dz = t.com[:, 2:3] - np.asarray(src)[None, :, 2]
    r2 = (dx * dx + dy * dy + dz * dz).min(1)
    assert np.allclose(r2, d2)
    leaf = t.nchild == 0
    opened = ~leaf & ((r2 < r_leaf * r_leaf) | (t.size * t.size > (theta * theta) * r2))
    reached = np.zeros(t.nnode, bool)
    reached[0] = True
    for a in range(1, t.nnode):
        reached[a] = reached[t.parent[a]] and opened[t.parent[a]]
    nodes = np.nonzero(reached & ((~leaf & ~opened) | (leaf & ~(r2 < r_part * r_part))))[0]
    expl = np.nonzero(reached & leaf & (r2 < r_part * r_part))[0]
    return set(nodes.tolist()), set(expl.tolist())


@pytest.mark.parametrize("theta", [0.3, 0.6, 1.0])
def test_selection(orc, tree, cloud, theta):
    t = tree
    src = np.array([[0.05, -0.02, 0.0]])
    sel = orc.select(t, src, 0.1, 0.2, theta)
    nodes, expl = _select_per_node(t, src, 0.1, 0.2, theta)
    assert set(sel.ref[sel.kind == 0].tolist()) == nodes
    parts = set(sel.ref[sel.kind == 1].tolist())
    assert parts == {k for a in expl for k in range(t.first[a], t.first[a] + t.count[a])}
    # re-tessellation: every particle covered exactly once, mass conserved (Section 2.2.2)
    cover = np.zeros(cloud.n, np.int64)
    for k, r in zip(sel.kind, sel.ref):
        if k == 0:
            cover[t.first[r]:t.first[r] + t.count[r]] += 1
        else:
            cover[r] += 1
    assert np.all(cover == 1)
    mass = t.mass[sel.ref[sel.kind == 0]].sum() + cloud.m[t.perm[sel.ref[sel.kind == 1]]].sum()
    assert abs(mass - cloud.m.sum()) < 1e-13
    # walk order is Morton order of the first constituent
    firsts = np.where(sel.kind == 0, t.first[np.where(sel.kind == 0, sel.ref, 0)], sel.ref)
    assert np.all(np.diff(firsts) > 0)
    # h-solver population: selected nodes plus the leaves of extracted particles
    assert set(sel.pop_node.tolist()) == nodes | expl


def w_np(q):
    return np.where(q < 1, 1 - 1.5 * q * q + 0.75 * q ** 3, np.where(q < 2, 0.25 * (2 - q) ** 3, 0.0))


def test_h_solver_residual(orc, tree, cloud):
    t = tree
    sel = orc.select(t, np.zeros((1, 3)), 0.05, 0.1, 0.5)
    nodes = sel.ref[sel.kind == 0]
    h0 = orc.h_initial(t, nodes, cloud.h, 1.2)
    pop = t.com[sel.pop_node]
    h, st, it = orc.h_solve(pop, t.com[nodes], h0, 1.2, 1e-13, 50)
    # Newton from h_0 (Eq. 11) mostly converges; a node with no neighbour inside 2 h_0
    # steps to h <= 0 and falls back to bisection (status 1)
    assert np.all(st <= 1) and (st == 0).mean() > 0.8
    assert it[st == 0].max() <= 12
    for a in range(0, nodes.shape[0], 5):
        r = np.linalg.norm(pop - t.com[nodes[a]], axis=1)
        n = (w_np(r / h[a]) / (math.pi * h[a] ** 3)).sum()
        assert abs(1.2 * n ** (-1 / 3) - h[a]) < 1e-12 * h[a]        # Eq. 8 at the root
    # paper tolerance (1e-2) converges in a few iterations (Section 2.4.2)
    h2, st2, it2 = orc.h_solve(pop, t.com[nodes], h0, 1.2, 1e-2, 50)
    assert np.median(it2[st2 == 0]) <= 4
    assert np.max(np.abs(h2 / h - 1)) < 0.05


def test_h_solver_lattice(orc):
    # equal nodes on a cubic lattice of spacing a: n ~ 1/a^3, so h -> h_fact a
    a = 0.1
    g = np.arange(-8, 9) * a
    X, Y, Z = np.meshgrid(g, g, g, indexing="ij")
    pop = np.stack([X.ravel(), Y.ravel(), Z.ravel()], 1)
    tgt = np.zeros((1, 3))
    h, st, _ = orc.h_solve(pop, tgt, np.array([2 * 1.2 * a]), 1.2, 1e-13, 50)
    assert st[0] == 0
    assert abs(h[0] / (1.2 * a) - 1) < 0.02
    r = np.linalg.norm(pop, axis=1)
    n = (w_np(r / h[0]) / (math.pi * h[0] ** 3)).sum()
    assert abs(1.2 * n ** (-1 / 3) - h[0]) < 1e-12 * h[0]


def test_h_solver_fallback_without_neighbours(orc):
    # a lone node: h_fact (1/(pi h^3))^(-1/3) - h > 0 for every h, no root, so
    # bisection fails and h_0 is kept (Section 2.4.2)
    pop = np.array([[0.0, 0, 0], [100.0, 0, 0]])
    h, st, _ = orc.h_solve(pop, pop[:1], np.array([0.3]), 1.2, 1e-13, 50)
    assert st[0] == 2 and h[0] == 0.3


def test_map_back_constant_and_linear(orc):
    w = inputs.uniform_cube(120, 100, seed=30, gen_seed=31)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs = orc.find_pairs(w.x, w.y, w.z, w.h, cells)
    wts = orc.map_exact(pairs, w.x, w.y, w.z, w.h, cells)
    f = orc.map_back(pairs, wts, np.full(cells.ncell, 0.37), w.n)
    assert np.max(np.abs(f - 0.37)) < 1e-15
    rng = np.random.default_rng(0)
    f1, f2 = rng.random(cells.ncell), rng.random(cells.ncell)
    a = orc.map_back(pairs, wts, 2 * f1 - 3 * f2, w.n)
    b = 2 * orc.map_back(pairs, wts, f1, w.n) - 3 * orc.map_back(pairs, wts, f2, w.n)
    assert np.max(np.abs(a - b)) < 1e-13


def _indicator_pin(map_back_fn, pairs, wts, n, ncell, cells_to_check):
    """Inverse mapping of the indicator field of cell j (1 on j, 0 elsewhere):
    f_i = w_ij / sum_j' w_ij' for exactly the particles paired with j, 0 for the
    other particles that have pairs.  The numerator is the single term w_ij and
    the denominator sums the same weights in the same order as u_i, so both
    sides are equal to the bit.  Returns the first failure, or None."""
    u = np.zeros(n)
    order = np.lexsort((pairs.pair_j, pairs.pair_i))
    for k in order:
        u[pairs.pair_i[k]] += wts[k]
    has = u > 0
    for j in cells_to_check:
        f_cell = np.zeros(ncell)
        f_cell[j] = 1.0
        f = map_back_fn(pairs, wts, f_cell, n)
        want = np.zeros(n)
        sel = np.flatnonzero(pairs.pair_j == j)
        want[pairs.pair_i[sel]] = wts[sel] / u[pairs.pair_i[sel]]
        if not np.array_equal(f[has], want[has]):
            return j
        if not np.all(np.isnan(f[~has])):
            return j
    return None


def test_map_back_indicator_field(orc):
    """An indicator field pins which cell value each pair reads: a constant or
    linear field cannot (Section 2.3, inverse mapping)."""
    w = inputs.uniform_cube(120, 100, seed=30, gen_seed=31)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs = orc.find_pairs(w.x, w.y, w.z, w.h, cells)
    wts = orc.map_exact(pairs, w.x, w.y, w.z, w.h, cells)
    js = [0, 17, 42, cells.ncell - 1]
    assert _indicator_pin(orc.map_back, pairs, wts, w.n, cells.ncell, js) is None

    # planted mistakes, each a copy of the oracle's sum with one index wrong
    def read_at_particle(pairs, wts, f_cell, n):   # f_cell[pair_i] instead of f_cell[pair_j]
        num, den = np.zeros(n), np.zeros(n)
        for k in np.lexsort((pairs.pair_j, pairs.pair_i)):
            i = pairs.pair_i[k]
            num[i] += wts[k] * f_cell[i % f_cell.shape[0]]
            den[i] += wts[k]
        with np.errstate(invalid="ignore", divide="ignore"):
            return num / den

    def weights_unsorted(pairs, wts, f_cell, n):   # weights read in the (i, j) order, cells in the (j, i) order
        num, den = np.zeros(n), np.zeros(n)
        order = np.lexsort((pairs.pair_j, pairs.pair_i))
        for t, k in enumerate(order):
            i = pairs.pair_i[k]
            num[i] += wts[order[t]] * f_cell[pairs.pair_j[t]]
            den[i] += wts[k]
        with np.errstate(invalid="ignore", divide="ignore"):
            return num / den

    for bad in (read_at_particle, weights_unsorted):
        assert _indicator_pin(bad, pairs, wts, w.n, cells.ncell, js) is not None, bad.__name__


def _inherit_pin(inherit_fn, ps, t, w):
    """Every particle takes the value of the pseudo-particle that stands for it
    (Section 2.5).  With f_pseudo = a (distinct per pseudo-particle), particle p
    must get the index of an extracted pseudo-particle whose origin is p
    itself, or of a node whose label is a prefix of p's Morton key (an
    independent restatement of membership: label = 1 followed by the node's
    3L key bits).  Returns the number of wrong particles."""
    f = inherit_fn(ps, t, np.arange(ps.n, dtype=np.float64))
    if f.shape[0] != w.n or not np.all(np.isfinite(f)):
        return w.n
    a = f.astype(np.int64)
    keys = morton_numpy(w.x, w.y, w.z, w.box)
    bad = 0
    org = ps.origin[a]
    part = org < 0
    bad += int(np.sum(-org[part] - 1 != np.flatnonzero(part)))
    lab = org[~part].astype(np.uint64)
    lev = np.array([(int(v).bit_length() - 1) // 3 for v in lab], np.uint64)
    pre = lab - (np.uint64(1) << (np.uint64(3) * lev))
    bad += int(np.sum((keys[~part] >> (np.uint64(3) * (np.uint64(21) - lev))) != pre))
    return bad


def test_inherit(orc, cloud):
    w = cloud
    ps, t, _ = orc.make_pseudo_particles(w.x, w.y, w.z, w.m, w.h, w.box, np.array([[0.05, -0.02, 0.0]]),
                                         0.1, 0.2, 0.5, solve=False)
    assert (ps.origin < 0).sum() > 20 and (ps.count[ps.origin > 0] > 1).sum() > 100
    assert _inherit_pin(orc.inherit, ps, t, w) == 0
    # a pseudo-particle of one particle hands back its own value
    f = orc.inherit(ps, t, np.arange(ps.n, dtype=np.float64))
    one = np.flatnonzero(ps.count == 1)
    assert np.array_equal(f[t.perm[ps.first[one]]], one.astype(np.float64))
    # a constant value is inherited unchanged by every particle
    assert np.all(orc.inherit(ps, t, np.full(ps.n, 0.3)) == 0.3)
    # planted mistake: the Morton positions taken as particle indices (perm dropped)
    import dataclasses
    no_perm = lambda ps_, t_, f_: orc.inherit(ps_, dataclasses.replace(t_, perm=np.arange(w.n)), f_)
    assert _inherit_pin(no_perm, ps, t, w) > 0
    # a double cover is rejected
    ps2 = dataclasses.replace(ps, first=ps.first.copy())
    ps2.first[1] = ps2.first[0]
    with pytest.raises(ValueError):
        orc.inherit(ps2, t, np.zeros(ps.n))


def test_h0_bypass(orc, cloud):
    """Above h0_above pseudo-particles no node is solved: each keeps h_0 of
    Eq. 11, 2 h_fact s_node (a one-particle node its particle's h), with
    status 2 (Section 2.4.2); at exactly h0_above the solver still runs."""
    w = cloud
    args = (w.x, w.y, w.z, w.m, w.h, w.box, np.zeros((1, 3)), 0.05, 0.1, 0.5)
    ps, t, sel = orc.make_pseudo_particles(*args)
    n = ps.n
    pb, _, selb = orc.make_pseudo_particles(*args, h0_above=n - 1)
    assert np.array_equal(selb.kind, sel.kind) and np.array_equal(selb.ref, sel.ref)
    isn = sel.kind == 0
    nodes = sel.ref[isn]
    multi = (t.count[nodes] > 1) & (t.size[nodes] > 0)
    assert multi.sum() > 10
    assert np.array_equal(pb.h[isn][multi], 2 * 1.2 * t.size[nodes][multi])
    one = t.count[nodes] == 1
    assert np.array_equal(pb.h[isn][one], w.h[t.perm[t.first[nodes[one]]]])
    assert np.all(pb.status[isn] == 2) and np.all(pb.status[~isn] == 3)
    assert np.array_equal(pb.h[~isn], ps.h[~isn])
    # the solved h differ from h_0: the bypass is not a no-op
    assert np.mean(np.abs(ps.h[isn][multi] / pb.h[isn][multi] - 1) > 1e-3) > 0.5
    pn, _, _ = orc.make_pseudo_particles(*args, h0_above=n)
    assert np.array_equal(pn.h, ps.h) and np.array_equal(pn.status, ps.status)
