"""The GPU path of the spatial split, with its ranks run one after the other
on one GPU: generators in Morton order, each rank's contiguous range of cells
built (build_voronoi_cells), paired (find_pairs_cells) and mapped, the
inverse mapping's sums added (the all-reduce; its multi-process form is
tests/test_partition.py's).  Against the single-rank path on the same
inputs: each rank's cells are the full build's, bit for bit; the ranks' pair
lists together are the full list; weights and cell densities are bit-equal;
the mapped-back field is equal up to the order of its additions."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api, inputs, partition

pytestmark = pytest.mark.gpu

SRC = np.zeros((1, 3))


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.mark.parametrize("world,precision", [(2, 1), (3, 0)])
def test_ranks_equal_single_rank(world, precision):
    w = inputs.sphere_workload(8000, 2000, 1.0, seed=31, field_seed=31)
    order = partition.morton_order(w.gx, w.gy, w.gz, w.box)
    G = [dev(a[order]) for a in (w.gx, w.gy, w.gz)]
    f_cell = dev(np.random.default_rng([31, 1]).random(w.ngen)[order])
    ctx = api.Context(0)
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.4, precision=precision)
    tree = api.build_tree(ctx, dev(w.x), dev(w.y), dev(w.z), dev(w.m), w.box, 8)
    ps = api.make_pseudo_particles(ctx, tree, dev(w.h), SRC, P)
    g = ps.get()
    X = (g["x"], g["y"], g["z"], g["h"], g["m"])
    # single rank
    vor = api.build_voronoi(ctx, *G, w.box, P)
    full = api.find_pairs(ctx, g["x"], g["y"], g["z"], g["h"], vor)
    w1, rho1, u1, _ = api.map_exact(ctx, full, *X, vor, P)
    f1, fp1 = api.map_back(ctx, full, w1, f_cell, ps, tree)
    vc = vor.get()
    # the ranks
    npp = g["x"].numel()
    num = torch.zeros(npp, dtype=torch.float64, device="cuda")
    den = torch.zeros_like(num)
    rho = torch.zeros_like(rho1)
    ws, pis = [], []
    for a, b in partition.contiguous_ranges(w.ngen, world):
        vr = api.build_voronoi_cells(ctx, *G, w.box, a, b, P)
        r = vr.get()
        cfo, fvo = vc["cell_face_off"], vc["face_vert_off"]
        rcfo, rfvo = r["cell_face_off"], r["face_vert_off"]
        # the rank's cells are the full build's; the others have no faces
        assert torch.equal(rcfo[b] - rcfo[a], cfo[b] - cfo[a]) and torch.equal(rcfo[a:b + 1] - rcfo[a],
                                                                                 cfo[a:b + 1] - cfo[a])
        f0, f1_ = int(cfo[a]), int(cfo[b])
        g0, g1_ = int(rcfo[a]), int(rcfo[b])
        assert torch.equal(r["normals"][g0:g1_], vc["normals"][f0:f1_])
        assert torch.equal(r["verts"][int(rfvo[g0]):int(rfvo[g1_])], vc["verts"][int(fvo[f0]):int(fvo[f1_])])
        assert torch.equal(r["volume"][a:b], vc["volume"][a:b])
        assert float(r["volume"][:a].abs().sum()) == 0.0 and float(r["volume"][b:].abs().sum()) == 0.0
        pr = api.find_pairs_cells(ctx, g["x"], g["y"], g["z"], g["h"], vr, a, b)
        wr, rr, _, _ = api.map_exact(ctx, pr, *X, vr, P)
        ws.append(wr)
        pis.append(pr.get()["pair_i"])
        rho += rr
        api.map_back_sums(ctx, pr, wr, f_cell, num, den)
    assert torch.equal(torch.cat(pis), full.get()["pair_i"])
    assert torch.equal(torch.cat(ws), w1)
    assert torch.equal(rho, rho1)
    f = num / den
    ok = den > 0
    assert torch.equal(ok, torch.isfinite(f1))
    assert torch.max(torch.abs(f[ok] - f1[ok]) / f1[ok].abs()).item() < 1e-13
    fp = api.inherit(ctx, ps, tree, f)
    okp = torch.isfinite(fp1)
    assert torch.max(torch.abs(fp[okp] - fp1[okp]) / fp1[okp].abs()).item() < 1e-13
