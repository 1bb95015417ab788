"""Oracle pins for the adaptive refinement of Section 2.4.1 (Eq. 5): the
neutral-fraction threshold, the tree-walk with nodes forced open, and the
iteration that re-selects until no node pseudo-particle is under-resolved."""
import numpy as np
import pytest

from paper_2410_15227_gb300 import inputs

SRC = np.zeros((1, 3))


def test_refine_limit_closed_form(orc):
    # f_neu,limit = (1/K)(K - s_root/s): at s = s_root it is 1 - 1/K, at half the
    # root's size 1 - 2/K, and it falls without bound as the node shrinks
    assert orc.refine_limit(1.0, 1.0, 10.0) == pytest.approx(0.9, abs=1e-15)
    assert orc.refine_limit(0.5, 1.0, 10.0) == pytest.approx(0.8, abs=1e-15)
    assert orc.refine_limit(0.1, 1.0, 10.0) == pytest.approx(0.0, abs=1e-15)
    assert orc.refine_limit(2.0, 4.0, 4.0) == pytest.approx(0.5, abs=1e-15)
    assert orc.refine_limit(0.0, 1.0, 10.0) == -np.inf
    s = np.linspace(1e-3, 1.0, 200)
    lim = orc.refine_limit(s, 1.0, 50.0)
    assert np.all(np.diff(lim) > 0)                                   # larger nodes face a higher threshold
    assert np.all(orc.refine_limit(s, 1.0, 200.0) > lim)              # and a larger K raises it (Section 2.4.1)


@pytest.fixture(scope="module")
def small(orc):
    w = inputs.sphere_workload(3000, 600, 1.0, seed=5, field_seed=5)
    t = orc.build_tree(w.x, w.y, w.z, w.m, w.box, 8)
    return w, t


def _covers_all(t, sel, n):
    """Every particle belongs to exactly one selected node or is extracted."""
    hit = np.zeros(n, np.int64)
    for kind, ref in zip(sel.kind, sel.ref):
        if kind == 0:
            hit[t.first[ref]:t.first[ref] + t.count[ref]] += 1
        else:
            hit[ref] += 1
    return np.all(hit == 1)


def test_select_with_force(orc, small):
    w, t = small
    args = (t, SRC, 0.05, 0.1, 0.3)
    base = orc.select(*args)
    same = orc.select(*args, force=np.zeros(t.nnode, np.uint8))
    assert np.array_equal(base.kind, same.kind) and np.array_equal(base.ref, same.ref)
    assert _covers_all(t, base, w.n)
    nodes = base.ref[base.kind == 0]
    inner = nodes[t.nchild[nodes] > 0]
    leaves = nodes[t.nchild[nodes] == 0]
    assert inner.shape[0] > 0 and leaves.shape[0] > 0
    # a forced internal node is opened: it is no longer selected, its range is still covered
    f = np.zeros(t.nnode, np.uint8)
    f[inner[0]] = 1
    s1 = orc.select(*args, force=f)
    assert inner[0] not in set(s1.ref[s1.kind == 0].tolist())
    assert _covers_all(t, s1, w.n) and s1.n > base.n
    # a forced leaf has its particles extracted
    f = np.zeros(t.nnode, np.uint8)
    f[leaves[0]] = 1
    s2 = orc.select(*args, force=f)
    lo, cnt = t.first[leaves[0]], t.count[leaves[0]]
    ext = set(s2.ref[s2.kind == 1].tolist())
    assert set(range(lo, lo + cnt)) <= ext and leaves[0] not in set(s2.ref[s2.kind == 0].tolist())
    assert _covers_all(t, s2, w.n)


def test_refine_loop(orc, small):
    w, _ = small
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    # a Stromgren-like step: ionized (f_neu = 0) within 0.3 of the source
    f_cell = np.where(np.linalg.norm(cells.gen, axis=1) < 0.3, 0.0, 1.0)
    K = 20.0
    ps0, _, _ = orc.make_pseudo_particles(w.x, w.y, w.z, w.m, w.h, w.box, SRC, 0.05, 0.1, 0.3)
    ps, t, sel, force, it, fn, radii = orc.refine(w.x, w.y, w.z, w.m, w.h, w.box, SRC, 0.05, 0.1, 0.3, cells,
                                                  f_cell, K, max_iter=30)
    assert 2 <= it < 30                       # refinement happened, and ended
    isn = sel.kind == 0
    nodes = sel.ref[isn]
    assert not np.any(orc.refine_fail(t, nodes, fn[isn], K))   # every node passes Eq. 5
    assert ps.n > ps0.n and force.sum() > 0
    assert _covers_all(t, sel, w.n)
    # the flagged nodes are opened (internal) or extracted (leaves)
    assert not np.any(force[nodes])
    assert radii == (0.05, 0.1)             # the radii stay put when failing leaves are extracted


def test_refine_loop_radii_growth(orc, small):
    """The form of Section 2.4.1 and Section 3.3: a failing leaf raises r_part
    and r_leaf by a step for the next walk instead of being flagged."""
    w, _ = small
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    f_cell = np.where(np.linalg.norm(cells.gen, axis=1) < 0.3, 0.0, 1.0)
    K, step = 20.0, 0.05
    ps, t, sel, force, it, fn, (rp, rl) = orc.refine(w.x, w.y, w.z, w.m, w.h, w.box, SRC, 0.05, 0.1, 0.3,
                                                     cells, f_cell, K, max_iter=30, leaf_step=step)
    assert 2 <= it < 30
    isn = sel.kind == 0
    nodes = sel.ref[isn]
    assert not np.any(orc.refine_fail(t, nodes, fn[isn], K))
    assert not np.any(force[t.nchild == 0])  # no leaf is ever flagged in this form
    k = round((rp - 0.05) / step)
    assert k >= 1 and rp == pytest.approx(0.05 + k * step) and rl == pytest.approx(0.1 + k * step)
    # the last walk is the plain walk with the grown radii and the flags
    again = orc.select(t, SRC, rp, rl, 0.3, force=force)
    assert np.array_equal(again.kind, sel.kind) and np.array_equal(again.ref, sel.ref)
    assert _covers_all(t, sel, w.n)
