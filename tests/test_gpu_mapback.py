"""Inverse mapping (Section 2.3) and constituent inheritance (Section 2.5) on
the GPU against the oracle, with a random per-cell field, so that a wrong cell
index, pair order or particle-to-pseudo-particle assignment shows.

Two comparisons on an 8,000-particle sphere with 2,000 sites, mapped through
pseudo-particles:
  - given the oracle's pair list and weights, map_back and the inheritance are
    bit-identical with oracle.map_back and oracle.inherit (both sum each
    particle's pairs in ascending cell order, products and sums rounded one by
    one, and the GPU's tree and selection equal the oracle's bit for bit);
  - the whole GPU path (its own h, pairs and weights, FP64 and mixed) against
    the oracle's whole path, within the weights' tolerance carried into a
    weighted mean of values in [0, 1]."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api, inputs

pytestmark = pytest.mark.gpu

SRC = np.zeros((1, 3))
R_PART, R_LEAF, THETA = 0.05, 0.1, 0.4


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def case(orc):
    w = inputs.sphere_workload(8000, 2000, 1.0, seed=23, field_seed=23)
    ps_o, t_o, _ = orc.make_pseudo_particles(w.x, w.y, w.z, w.m, w.h, w.box, SRC, R_PART, R_LEAF, THETA,
                                             tol=1e-13)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs_o = orc.find_pairs(ps_o.x, ps_o.y, ps_o.z, ps_o.h, cells)
    w_o = orc.map_exact(pairs_o, ps_o.x, ps_o.y, ps_o.z, ps_o.h, cells)
    f_cell = np.random.default_rng([23, 1]).random(cells.ncell)
    f_o = orc.map_back(pairs_o, w_o, f_cell, ps_o.n)
    fp_o = orc.inherit(ps_o, t_o, f_o)
    ctx = api.Context(0)
    P = api.Params(r_part=R_PART, r_leaf=R_LEAF, theta=THETA, h_tol=1e-13)
    tree = api.build_tree(ctx, dev(w.x), dev(w.y), dev(w.z), dev(w.m), w.box, 8)
    ps = api.make_pseudo_particles(ctx, tree, dev(w.h), SRC, P)
    vor = api.build_voronoi(ctx, dev(w.gx), dev(w.gy), dev(w.gz), w.box, P)
    return dict(w=w, ps_o=ps_o, t_o=t_o, cells=cells, pairs_o=pairs_o, w_o=w_o, f_cell=f_cell, f_o=f_o,
                fp_o=fp_o, ctx=ctx, P=P, tree=tree, ps=ps, vor=vor)


def test_selection_matches(case):
    g = {k: v.cpu().numpy() for k, v in case["ps"].get().items()}
    ps_o = case["ps_o"]
    assert ps_o.n > 500 and (ps_o.count > 1).sum() > 300
    assert np.array_equal(g["origin"], ps_o.origin)
    assert np.array_equal(g["first"], ps_o.first) and np.array_equal(g["count"], ps_o.count)


def test_map_back_and_inherit_bit_exact_on_oracle_weights(case):
    ctx, po, ps_o = case["ctx"], case["pairs_o"], case["ps_o"]
    pr = api.pairs_from_list(ctx, dev(po.pair_i, torch.int32), dev(po.pair_j, torch.int32), ps_o.n, case["vor"])
    f, fp = api.map_back(ctx, pr, dev(case["w_o"]), dev(case["f_cell"]), case["ps"], case["tree"])
    f, fp = f.cpu().numpy(), fp.cpu().numpy()
    assert np.array_equal(f, case["f_o"], equal_nan=True)
    assert np.array_equal(fp, case["fp_o"], equal_nan=True)
    assert np.isfinite(fp).all() and np.std(fp) > 0.02   # a non-constant field reached every particle


@pytest.mark.parametrize("precision,tol", [(0, 1e-10), (1, 2e-5)])
def test_whole_path_against_oracle(orc, case, precision, tol):
    """Every step on the GPU.  The node h agree to 1e-12 with the oracle's, the
    weights to 1e-12 (FP64) or 1e-5 (mixed) relative; f_i is a weighted mean
    of values in [0, 1], so its error is at most the weights' relative error
    times 2 (numerator and denominator)."""
    ctx, ps, tree, vor = case["ctx"], case["ps"], case["tree"], case["vor"]
    g = ps.get()
    pr = api.find_pairs(ctx, g["x"], g["y"], g["z"], g["h"], vor)
    wts, _, _, _ = api.map_exact(ctx, pr, g["x"], g["y"], g["z"], g["h"], g["m"], vor,
                                 api.Params(precision=precision, fp64_threshold=1e-5))
    f, fp = api.map_back(ctx, pr, wts, dev(case["f_cell"]), ps, tree)
    f, fp = f.cpu().numpy(), fp.cpu().numpy()
    assert np.array_equal(np.isnan(f), np.isnan(case["f_o"]))
    ok = ~np.isnan(f)
    assert np.max(np.abs(f[ok] - case["f_o"][ok])) < tol
    assert np.max(np.abs(fp - case["fp_o"])) < tol
    # inheritance is a gather through the oracle's membership of every particle
    ps_o = case["ps_o"]
    owner = orc.inherit(ps_o, case["t_o"], np.arange(ps_o.n, dtype=np.float64)).astype(np.int64)
    assert np.array_equal(fp, f[owner], equal_nan=True)
