"""Oracle pins for the cell centroids and Lloyd's iteration on the sites
(Section 2.3): the cells tile the box, so their first moments add up to the
box's; a regular lattice of sites at the centres of equal boxes is a fixed
point; one site's cell is the box; Monte Carlo centroids; Lloyd's iteration
lowers the quantisation energy.  CPU only."""
import numpy as np

from paper_2410_15227_gb300 import inputs

BOX = np.array([0.0, 1.0, 0.0, 1.0, 0.0, 1.0])


def test_centroids_tile_the_box(orc):
    w = inputs.uniform_cube(10, 300, seed=3, gen_seed=4)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    cen, vol = orc.cell_centroids(cells)
    assert np.max(np.abs(vol - cells.volume)) < 1e-14          # against the oracle's own divergence-theorem volume
    b = w.box
    vbox = (b[1] - b[0]) * (b[3] - b[2]) * (b[5] - b[4])
    mid = np.array([(b[0] + b[1]) / 2, (b[2] + b[3]) / 2, (b[4] + b[5]) / 2])
    assert abs(vol.sum() - vbox) < 1e-13
    assert np.max(np.abs((vol[:, None] * cen).sum(0) - vbox * mid)) < 1e-13
    # a centroid lies inside its cell: on the inner side of every face plane
    for j in range(0, cells.ncell, 7):
        for verts, n, _ in cells.faces(j):
            assert np.dot(cen[j] - verts[0], n) < 0


def test_centroids_lattice_fixed_point(orc):
    k = 4
    c = (np.arange(k) + 0.5) / k
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    cells = orc.voronoi(X.ravel(), Y.ravel(), Z.ravel(), BOX)
    cen, vol = orc.cell_centroids(cells)
    assert np.max(np.abs(cen - cells.gen)) < 1e-15
    assert np.max(np.abs(vol - 1.0 / k ** 3)) < 1e-16
    gx, gy, gz = orc.lloyd(X.ravel(), Y.ravel(), Z.ravel(), BOX, iters=2)
    assert np.max(np.abs(gx - X.ravel())) < 1e-15 and np.max(np.abs(gz - Z.ravel())) < 1e-15


def test_centroid_single_site_and_off_centre(orc):
    box = np.array([-1.0, 3.0, 0.0, 0.5, 2.0, 2.25])
    cells = orc.voronoi([0.1], [0.4], [2.2], box)
    cen, vol = orc.cell_centroids(cells)
    assert np.max(np.abs(cen[0] - [1.0, 0.25, 2.125])) < 1e-15 and abs(vol[0] - 0.5) < 1e-15
    # two sites split the unit box by the plane x = 0.4 (sites at x = 0.3, 0.5)
    cells = orc.voronoi([0.3, 0.5], [0.5, 0.5], [0.5, 0.5], BOX)
    cen, vol = orc.cell_centroids(cells)
    assert np.max(np.abs(cen - [[0.2, 0.5, 0.5], [0.7, 0.5, 0.5]])) < 1e-15
    assert np.max(np.abs(vol - [0.4, 0.6])) < 1e-15


def test_centroids_monte_carlo(orc):
    w = inputs.uniform_cube(10, 40, seed=5, gen_seed=6)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    cen, _ = orc.cell_centroids(cells)
    rng = np.random.default_rng(7)
    b = w.box
    P = rng.uniform([b[0], b[2], b[4]], [b[1], b[3], b[5]], size=(400000, 3))
    G = cells.gen
    owner = np.argmin(((P[:, None, :] - G[None, :, :]) ** 2).sum(-1), axis=1)
    for j in range(cells.ncell):
        q = P[owner == j]
        se = q.std(0) / np.sqrt(q.shape[0])
        assert np.all(np.abs(q.mean(0) - cen[j]) < 5 * se + 1e-12), j


def test_lloyd_lowers_energy(orc):
    """Lloyd's iteration does not raise E = sum_j integral over V_j of
    |r - g_j|^2; checked on a fixed Monte Carlo sample, where every cell's
    term also does not rise when its site moves to the sample mean."""
    w = inputs.uniform_cube(10, 60, seed=8, gen_seed=9)
    rng = np.random.default_rng(10)
    P = rng.uniform(0, 1, size=(200000, 3))

    def energy(g):
        d = ((P[:, None, :] - g[None, :, :]) ** 2).sum(-1)
        return d.min(1).mean()

    g0 = np.stack([w.gx, w.gy, w.gz], 1)
    e = [energy(g0)]
    g = g0
    for _ in range(5):
        gx, gy, gz = orc.lloyd(g[:, 0], g[:, 1], g[:, 2], w.box, iters=1)
        g = np.stack([gx, gy, gz], 1)
        e.append(energy(g))
    assert e[-1] < 0.9 * e[0]
    assert all(e[k + 1] < e[k] + 2e-5 for k in range(5)), e
    gx, gy, gz = orc.lloyd(w.gx, w.gy, w.gz, w.box, iters=5)
    assert np.array_equal(np.stack([gx, gy, gz], 1), g)     # five single moves are five moves
