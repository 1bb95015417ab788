"""Pins of the oracle's brute-force Voronoi cells, all-pairs test, mapping and
cell densities: Voronoi invariants, partition of unity, mass conservation and
an independent distance computation.  CPU only."""
import math

import numpy as np
import pytest

from paper_2410_15227_gb300 import inputs


@pytest.fixture(scope="module")
def cube(orc):
    w = inputs.uniform_cube(300, 250, seed=10, gen_seed=11)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs = orc.find_pairs(w.x, w.y, w.z, w.h, cells)
    wts = orc.map_exact(pairs, w.x, w.y, w.z, w.h, cells)
    return w, cells, pairs, wts


def _area(v, n):
    s = np.zeros(3)
    for k in range(1, len(v) - 1):
        s += np.cross(v[k] - v[0], v[k + 1] - v[0])
    return 0.5 * float(s @ n)


def test_volumes_sum_to_box(cube):
    w, cells, _, _ = cube
    assert abs(cells.volume.sum() - 1.0) < 1e-12
    assert np.all(cells.volume > 0)


def test_face_reciprocity_and_vertices(cube):
    w, cells, _, _ = cube
    g = np.stack([w.gx, w.gy, w.gz], 1)
    faces = {}
    for j in range(cells.ncell):
        for v, n, k in cells.faces(j):
            faces[(j, k)] = (_area(v, n), n)
            if k >= 0:
                dj = np.linalg.norm(v - g[j], axis=1)
                dk = np.linalg.norm(v - g[k], axis=1)
                assert np.max(np.abs(dj - dk)) < 1e-12
                # no generator is closer to a vertex than its own two
                dall = np.linalg.norm(v[:, None, :] - g[None, :, :], axis=2).min(axis=1)
                assert np.all(dall >= dj - 1e-12)
    for (j, k), (a, n) in faces.items():
        if k >= 0:
            a2, n2 = faces[(k, j)]
            assert abs(a - a2) < 1e-12 * max(1.0, a)
            assert np.allclose(n, -n2, atol=1e-12)


def test_euler_characteristic(cube):
    _, cells, _, _ = cube
    for j in range(cells.ncell):
        fs = cells.faces(j)
        allv = np.concatenate([v for v, _, _ in fs])
        nv = len(np.unique(np.round(allv, 11), axis=0))
        ne = sum(len(v) for v, _, _ in fs) // 2
        assert nv - ne + len(fs) == 2


def test_cells_are_nearest_generator_regions(cube, orc):
    w, cells, _, _ = cube
    g = np.stack([w.gx, w.gy, w.gz], 1)
    rng = np.random.default_rng(3)
    pts = rng.random((2000, 3))
    nearest = np.argmin(np.linalg.norm(pts[:, None] - g[None], axis=2), axis=1)
    for p, j in zip(pts[:200], nearest[:200]):
        assert orc.cell_distance(p, cells, int(j)) == 0.0


def test_partition_of_unity(cube, orc):
    w, cells, pairs, wts = cube
    u = orc.particle_weight_sum(pairs, wts, w.n)
    inside = ((w.x - 2 * w.h > 0) & (w.x + 2 * w.h < 1) & (w.y - 2 * w.h > 0) & (w.y + 2 * w.h < 1)
              & (w.z - 2 * w.h > 0) & (w.z + 2 * w.h < 1))
    assert inside.sum() >= 5
    assert np.max(np.abs(u[inside] - 1)) < 1e-13
    # no particle gets more than its whole kernel
    assert np.all(u < 1 + 1e-13)


def test_mass_conservation(cube, orc):
    w, cells, pairs, wts = cube
    rho = orc.cell_density(pairs, wts, w.m, cells.volume)
    u = orc.particle_weight_sum(pairs, wts, w.n)
    assert abs((rho * cells.volume).sum() - (w.m * u).sum()) < 1e-14


def test_pairs_sorted_and_weights_positive(cube):
    _, cells, pairs, wts = cube
    assert np.all(np.diff(pairs.pair_j) >= 0)
    same = pairs.pair_j[1:] == pairs.pair_j[:-1]
    assert np.all(np.diff(pairs.pair_i)[same] > 0)
    assert np.all(wts > -1e-15)
    assert pairs.near.sum() == 0


def test_non_pairs_have_no_overlap(cube, orc):
    """Pairs absent from the list: the kernel sphere does not meet the cell.  The
    distance is re-computed by constrained minimisation (independent of the
    oracle's point-to-polygon routine) for candidates near the threshold."""
    from scipy.optimize import minimize
    w, cells, pairs, _ = cube
    have = set(zip(pairs.pair_i.tolist(), pairs.pair_j.tolist()))
    g = cells.gen
    rng = np.random.default_rng(5)
    checked = 0
    off = cells.offsets()
    for i in rng.choice(w.n, 40, replace=False):
        p = np.array([w.x[i], w.y[i], w.z[i]])
        d = np.linalg.norm(g - p, axis=1)
        for j in np.argsort(d)[:40]:
            f0, f1 = cells.cell_face_off[j], cells.cell_face_off[j + 1]
            A, b = cells.normals[f0:f1], off[f0:f1]
            res = minimize(lambda q: np.sum((q - p) ** 2), g[j], jac=lambda q: 2 * (q - p),
                           constraints=[{"type": "ineq", "fun": lambda q: b - A @ q,
                                         "jac": lambda q: -A}], method="SLSQP",
                           options={"ftol": 1e-15, "maxiter": 500})
            dist = math.sqrt(max(res.fun, 0.0))
            if abs(dist - 2 * w.h[i]) < 1e-6 * w.h[i]:
                continue
            assert ((int(i), int(j)) in have) == (dist < 2 * w.h[i])
            checked += 1
    assert checked > 500


def test_weights_against_quadrature_on_sample(cube, orc):
    w, cells, pairs, wts = cube
    rng = np.random.default_rng(6)
    for k in rng.choice(pairs.n, 6, replace=False):
        i, j = int(pairs.pair_i[k]), int(pairs.pair_j[k])
        q = orc.cell_weight_quadrature([w.x[i], w.y[i], w.z[i]], w.h[i], cells, j, 1e-9)
        assert abs(q - wts[k]) < 5e-8
