"""Streamed pair finding (find_pairs_plan, find_pairs_cells) and the inverse
mapping in parts (map_back_sums, inherit), against the whole-list calls on
an 8,000-particle sphere through pseudo-particles, with the oracle's pair
list as the anchor:
  - the chunks' pair lists, concatenated, are find_pairs' list (and the
    oracle's), each chunk within the capacity unless it is a single cell;
  - every weight of every chunk equals the whole list's, bit for bit, in both
    precisions (a pair's weight does not depend on the other pairs);
  - the chunks' cell densities add up to the whole list's, bit for bit (a
    cell's pairs are all in one chunk, and the others contribute exact zeros);
  - the weight sums and the inverse mapping's sums add over the chunks to the
    whole list's within rounding of the changed order of additions;
  - inherit equals map_back's inheritance bit for bit."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api, inputs

pytestmark = pytest.mark.gpu

SRC = np.zeros((1, 3))


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def case():
    w = inputs.sphere_workload(8000, 2000, 1.0, seed=29, field_seed=29)
    ctx = api.Context(0)
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.4, h_tol=1e-13)
    tree = api.build_tree(ctx, dev(w.x), dev(w.y), dev(w.z), dev(w.m), w.box, 8)
    ps = api.make_pseudo_particles(ctx, tree, dev(w.h), SRC, P)
    g = ps.get()
    vor = api.build_voronoi(ctx, dev(w.gx), dev(w.gy), dev(w.gz), w.box, P)
    full = api.find_pairs(ctx, g["x"], g["y"], g["z"], g["h"], vor)
    f_cell = dev(np.random.default_rng([29, 2]).random(w.ngen))
    return dict(w=w, ctx=ctx, P=P, tree=tree, ps=ps, g=g, vor=vor, full=full, f_cell=f_cell)


def pair_arrays(pr):
    d = pr.get()
    return d["pair_i"].cpu().numpy(), d["pair_j"].cpu().numpy()


def test_chunks_cover_the_pair_list(case, orc):
    ctx, g, vor = case["ctx"], case["g"], case["vor"]
    ntot = case["full"].info()[0]
    cap = ntot // 7
    bounds, total = api.find_pairs_plan(ctx, g["x"], g["y"], g["z"], g["h"], vor, cap)
    nc = vor.info()[0]
    assert total == ntot and bounds[0] == 0 and bounds[-1] == nc and len(bounds) >= 8
    assert all(a < b for a, b in zip(bounds[:-1], bounds[1:]))
    pi, pj = [], []
    for a, b in zip(bounds[:-1], bounds[1:]):
        pr = api.find_pairs_cells(ctx, g["x"], g["y"], g["z"], g["h"], vor, a, b)
        n = pr.info()[0]
        assert n <= cap or b == a + 1
        i, j = pair_arrays(pr)
        assert np.all((j >= a) & (j < b))
        pi.append(i)
        pj.append(j)
    fi, fj = pair_arrays(case["full"])
    assert np.array_equal(np.concatenate(pi), fi) and np.array_equal(np.concatenate(pj), fj)
    # the anchor: the oracle's all-pairs list on the same pseudo-particles and cells
    gp = {k: v.cpu().numpy() for k, v in g.items()}
    vc = {k: v.cpu().numpy() for k, v in vor.get().items()}
    w = case["w"]
    cells = orc.Cells(vc["cell_face_off"], vc["face_vert_off"], vc["verts"].reshape(-1, 3),
                      vc["normals"].reshape(-1, 3), vc["nbr"], vc["volume"], np.stack([w.gx, w.gy, w.gz], 1),
                      np.arange(nc))
    po = orc.find_pairs(gp["x"], gp["y"], gp["z"], gp["h"], cells)
    assert np.array_equal(po.pair_i, fi) and np.array_equal(po.pair_j, fj)
    # a capacity below every cell's count: one cell per chunk; an empty range
    b1, _ = api.find_pairs_plan(ctx, g["x"], g["y"], g["z"], g["h"], vor, 1)
    assert b1 == list(range(nc + 1))
    assert api.find_pairs_cells(ctx, g["x"], g["y"], g["z"], g["h"], vor, 5, 5).info()[0] == 0
    with pytest.raises(Exception):
        api.find_pairs_cells(ctx, g["x"], g["y"], g["z"], g["h"], vor, 5, nc + 1)


@pytest.mark.parametrize("precision", [0, 1])
def test_mapping_in_chunks(case, precision):
    ctx, g, vor, full = case["ctx"], case["g"], case["vor"], case["full"]
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.4, precision=precision)
    X = (g["x"], g["y"], g["z"], g["h"], g["m"])
    w_full, rho_full, u_full, _ = api.map_exact(ctx, full, *X, vor, P)
    f_full, fp_full = api.map_back(ctx, full, w_full, case["f_cell"], case["ps"], case["tree"])
    np_ = g["x"].numel()
    bounds, _ = api.find_pairs_plan(ctx, g["x"], g["y"], g["z"], g["h"], vor, full.info()[0] // 5)
    rho = torch.zeros_like(rho_full)
    u = torch.zeros_like(u_full)
    num = torch.zeros(np_, dtype=torch.float64, device="cuda")
    den = torch.zeros_like(num)
    ws = []
    for a, b in zip(bounds[:-1], bounds[1:]):
        pr = api.find_pairs_cells(ctx, g["x"], g["y"], g["z"], g["h"], vor, a, b)
        wc, rc, uc, _ = api.map_exact(ctx, pr, *X, vor, P)
        ws.append(wc)
        rho += rc
        u += uc
        api.map_back_sums(ctx, pr, wc, case["f_cell"], num, den)
    assert torch.equal(torch.cat(ws), w_full)
    assert torch.equal(rho, rho_full)
    assert torch.max(torch.abs(u - u_full)).item() < 1e-14
    f = num / den
    ok = den > 0
    assert torch.equal(ok, torch.isfinite(f_full))
    assert torch.max(torch.abs(f[ok] - f_full[ok]) / f_full[ok].abs()).item() < 1e-13
    # inheritance alone equals map_back's
    assert torch.equal(torch.nan_to_num(api.inherit(ctx, case["ps"], case["tree"], f_full), nan=-1.0),
                       torch.nan_to_num(fp_full, nan=-1.0))
