"""GPU parity of the adaptive refinement of Section 2.4.1 (Eq. 5) with the
oracle: the same sequence of tree-walks, maps and checks on a 3,000-particle
sphere with a Stromgren-like neutral-fraction step (0 within 0.3 of the
source, 1 outside), mapped in FP64 so that no Eq. 5 decision hangs on mixed
rounding."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api, inputs

pytestmark = pytest.mark.gpu

SRC = np.zeros((1, 3))
K = 20.0


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("leaf_step", [0.0, 0.05])
def test_refine_matches_oracle(orc, leaf_step):
    w = inputs.sphere_workload(3000, 600, 1.0, seed=5, field_seed=5)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    f_cell = np.where(np.linalg.norm(cells.gen, axis=1) < 0.3, 0.0, 1.0)
    ps_o, t_o, sel_o, force_o, it_o, fn_o, radii_o = orc.refine(w.x, w.y, w.z, w.m, w.h, w.box, SRC, 0.05, 0.1,
                                                                0.3, cells, f_cell, K, max_iter=30,
                                                                leaf_step=leaf_step)
    ctx = api.Context(0)
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, h_tol=1e-13, precision=0)
    tree = api.build_tree(ctx, dev(w.x), dev(w.y), dev(w.z), dev(w.m), w.box, 8)
    vor = api.build_voronoi(ctx, dev(w.gx), dev(w.gy), dev(w.gz), w.box, P)
    ps, pr, wts, force, it, fn, radii = api.refine(ctx, tree, dev(w.h), SRC, P, vor, dev(f_cell), K, max_iter=30,
                                                   leaf_step=leaf_step)
    torch.cuda.synchronize()
    assert it_o >= 2 and it == it_o
    assert radii == radii_o
    assert np.array_equal(force.cpu().numpy(), force_o)
    g = {k: v.cpu().numpy() for k, v in ps.get().items()}
    assert np.array_equal(g["origin"], ps_o.origin)
    for k in ("x", "y", "z", "m"):
        assert np.array_equal(g[k], getattr(ps_o, k)), k
    fn = fn.cpu().numpy()
    assert np.array_equal(np.isnan(fn), np.isnan(fn_o))
    ok = ~np.isnan(fn)
    assert np.max(np.abs(fn[ok] - fn_o[ok])) < 1e-10


def test_refine_check_flags_only_new(orc):
    """refine_check flags a failing node once: a second call on the same
    values flags nothing more."""
    w = inputs.sphere_workload(3000, 600, 1.0, seed=5, field_seed=5)
    ctx = api.Context(0)
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, h_tol=1e-13, precision=0)
    tree = api.build_tree(ctx, dev(w.x), dev(w.y), dev(w.z), dev(w.m), w.box, 8)
    ps = api.make_pseudo_particles(ctx, tree, dev(w.h), SRC, P)
    n, _ = ps.info()
    _, nnode, _ = tree.info()
    force = torch.zeros(nnode, dtype=torch.uint8, device="cuda")
    f_neu = torch.zeros(n, dtype=torch.float64, device="cuda")   # fully ionized: every sized node fails
    tg = {k: v.cpu().numpy() for k, v in tree.get().items()}
    leaf = np.zeros(nnode, bool)
    leaf[tg["nchild"] == 0] = True
    # without leaf flags only internal nodes are flagged, and the failing leaves counted
    first, nleaf = api.refine_check(ctx, ps, tree, f_neu, K, force, flag_leaves=False)
    fl = force.cpu().numpy().astype(bool)
    assert first > 0 and nleaf > 0 and fl.sum() == first and not np.any(fl & leaf)
    _, t_o, sel_o = orc.make_pseudo_particles(w.x, w.y, w.z, w.m, w.h, w.box, SRC, 0.05, 0.1, 0.3)
    nodes = sel_o.ref[sel_o.kind == 0]
    fail = orc.refine_fail(t_o, nodes, np.zeros(nodes.shape[0]), K)
    isleaf = t_o.nchild[nodes] == 0
    assert first == int((fail & ~isleaf).sum()) and nleaf == int((fail & isleaf).sum())
    assert np.array_equal(np.flatnonzero(fl), np.sort(nodes[fail & ~isleaf]))
    # with them the leaves are flagged too; the internal nodes are not counted again
    again, nleaf2 = api.refine_check(ctx, ps, tree, f_neu, K, force)
    fl = force.cpu().numpy().astype(bool)
    assert again == nleaf and nleaf2 == nleaf and (fl & leaf).sum() == nleaf
    assert api.refine_check(ctx, ps, tree, f_neu, K, force) == (0, nleaf)
    with pytest.raises(Exception):
        api.refine_check(ctx, ps, tree, f_neu, 1.0, force)   # K must exceed 1
