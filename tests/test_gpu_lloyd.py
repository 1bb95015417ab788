"""GPU parity of the cell centroids and of Lloyd's iteration on the sites
(Section 2.3) with the oracle.

Tolerances: a centroid is a sum of O(100) tetrahedron moments of size up to
the cell's extent, so FP64 rounding leaves ~1e-15 of the box on either side
(1e-13 is asserted).  Five Lloyd moves compound those differences through
five Voronoi builds; the move is a contraction towards the centroid, so they
stay near the rounding level (1e-11 of the box is asserted)."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def ctx():
    return api.Context(0)


CASES = {"cube": lambda: inputs.uniform_cube(10, 1500, seed=40, gen_seed=41),
         "sphere": lambda: inputs.sphere_workload(6000, 1200, 1.0, seed=42, field_seed=42)}


def _scale(box):
    return max(box[1] - box[0], box[3] - box[2], box[5] - box[4])


@pytest.mark.parametrize("name", list(CASES))
def test_centroids_match_oracle(ctx, orc, name):
    w = CASES[name]()
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    cen_o, vol_o = orc.cell_centroids(cells)
    vor = api.build_voronoi(ctx, dev(w.gx), dev(w.gy), dev(w.gz), w.box, api.Params())
    cx, cy, cz = api.voronoi_centroids(ctx, vor)
    cen = torch.stack([cx, cy, cz], 1).cpu().numpy()
    assert np.max(np.abs(cen - cen_o)) < 1e-13 * _scale(w.box)


@pytest.mark.parametrize("name", list(CASES))
def test_lloyd_matches_oracle(ctx, orc, name):
    w = CASES[name]()
    ox, oy, oz = orc.lloyd(w.gx, w.gy, w.gz, w.box, iters=5)
    gx, gy, gz = dev(w.gx), dev(w.gy), dev(w.gz)
    api.lloyd(ctx, gx, gy, gz, w.box, iters=5)
    g = torch.stack([gx, gy, gz], 1).cpu().numpy()
    err = np.max(np.abs(g - np.stack([ox, oy, oz], 1)))
    assert err < 1e-11 * _scale(w.box), err
    moved = np.max(np.abs(g - np.stack([w.gx, w.gy, w.gz], 1)))
    assert moved > 1e-3 * _scale(w.box)


def test_lloyd_edge_cases(ctx):
    box = np.array([0.0, 1.0, 0.0, 1.0, 0.0, 1.0])
    # no iteration leaves the sites untouched
    w = inputs.uniform_cube(10, 100, seed=43, gen_seed=44)
    gx, gy, gz = dev(w.gx), dev(w.gy), dev(w.gz)
    api.lloyd(ctx, gx, gy, gz, w.box, iters=0)
    assert np.array_equal(gx.cpu().numpy(), w.gx)
    # one site moves to the centre of the box
    box2 = np.array([-1.0, 3.0, 0.0, 0.5, 2.0, 2.25])
    s = [dev([0.1]), dev([0.4]), dev([2.2])]
    api.lloyd(ctx, *s, box2, iters=1)
    assert np.max(np.abs(torch.cat(s).cpu().numpy() - [1.0, 0.25, 2.125])) < 1e-15
    # sites at the centres of a regular lattice of boxes stay put
    k = 5
    c = (np.arange(k) + 0.5) / k
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    L = [dev(X.ravel()), dev(Y.ravel()), dev(Z.ravel())]
    api.lloyd(ctx, *L, box, iters=3)
    assert np.max(np.abs(L[0].cpu().numpy() - X.ravel())) < 1e-14
    assert np.max(np.abs(L[2].cpu().numpy() - Z.ravel())) < 1e-14
    # a site outside the box is rejected, the sites keep their values
    bad = [dev([0.5, 1.5]), dev([0.5, 0.5]), dev([0.5, 0.5])]
    with pytest.raises(Exception):
        api.lloyd(ctx, *bad, box, iters=1)
    assert bad[0].cpu().numpy()[1] == 1.5


def test_lloyd_full_size(ctx, orc):
    """The benchmark's 262,144 sites: five moves on the GPU; then the cells of
    the moved sites tile the box (sum V_j c_j = V_box c_box), and the
    centroids of 24 sampled cells, each built by the oracle from all sites,
    match the GPU's."""
    w = inputs.workload_pseudo_1e6()
    gx, gy, gz = dev(w.gx), dev(w.gy), dev(w.gz)
    api.lloyd(ctx, gx, gy, gz, w.box, iters=5)
    vor = api.build_voronoi(ctx, gx, gy, gz, w.box, api.Params())
    cx, cy, cz = api.voronoi_centroids(ctx, vor)
    vol = vor.get()["volume"]
    b = w.box
    vbox = (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4])
    mid = [(b[0] + b[1]) / 2, (b[2] + b[3]) / 2, (b[4] + b[5]) / 2]
    for c, m in zip((cx, cy, cz), mid):
        assert abs(float((vol * c).sum()) - vbox * m) < 1e-11 * vbox * _scale(b)
    G = [t.cpu().numpy() for t in (gx, gy, gz)]
    ids = np.random.default_rng(45).choice(w.ngen, 24, replace=False)
    cells = orc.voronoi(*G, w.box, cells=ids)
    cen_o, _ = orc.cell_centroids(cells)
    cen = torch.stack([cx, cy, cz], 1).cpu().numpy()[ids]
    assert np.max(np.abs(cen - cen_o)) < 1e-13 * _scale(b)
