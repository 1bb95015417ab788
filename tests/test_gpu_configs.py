"""Parity on the two other workloads, at their own sizes.

* 1,000 equal-mass particles in the unit cube (seed 0), h from the
  57-neighbour rule, on 1,000 uniform generators (seed 1): everything is
  compared with the oracle's complete computation (brute-force cells,
  all-pairs test, closed-form weights).
* 100,000 particles of the r^-1.5 x lognormal sphere on 25,000 cells, mapped
  directly in FP64 and in mixed precision: sampled particles' complete pair
  lists and weights against the oracle (candidate cells from the bound
  |g_j - p| <= 4h + d_p), partition of unity and mass over every particle."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api, inputs

pytestmark = pytest.mark.gpu


def _area(v, n):
    t = np.zeros(3)
    for k in range(1, len(v) - 1):
        t += np.cross(v[k] - v[0], v[k + 1] - v[0])
    return 0.5 * float(t @ n)


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def ctx():
    return api.Context(0)


def _gpu_chain(ctx, w):
    X = [dev(a) for a in (w.x, w.y, w.z, w.h, w.m)]
    vor = api.build_voronoi(ctx, dev(w.gx), dev(w.gy), dev(w.gz), w.box, api.Params())
    pr = api.find_pairs(ctx, *X[:4], vor)
    w64, rho64, u64, _ = api.map_exact(ctx, pr, *X, vor, api.Params(precision=0))
    wm, rhom, um, nf = api.map_exact(ctx, pr, *X, vor, api.Params(precision=1, fp64_threshold=1e-5))
    torch.cuda.synchronize()
    c = lambda t: t.cpu().numpy()
    return dict(vor=vor, pr=pr, pg={k: c(v) for k, v in pr.get().items()}, vg={k: c(v) for k, v in vor.get().items()},
                w64=c(w64), rho64=c(rho64), u64=c(u64), wm=c(wm), rhom=c(rhom), um=c(um), nf=nf)


def test_cube_1k_against_full_oracle(ctx, orc):
    w = inputs.workload_cube_1k()
    g = _gpu_chain(ctx, w)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs = orc.find_pairs(w.x, w.y, w.z, w.h, cells)
    wo = orc.map_exact(pairs, w.x, w.y, w.z, w.h, cells)
    rho_o = orc.cell_density(pairs, wo, w.m, cells.volume)
    assert np.array_equal(g["pg"]["pair_i"], pairs.pair_i) and np.array_equal(g["pg"]["pair_j"], pairs.pair_j)
    vg = g["vg"]
    for j in range(cells.ncell):
        fo = {nb for v, n, nb in cells.faces(j) if abs(_area(v, n)) >= 1e-10}
        fg = {int(vg["nbr"][f]) for f in range(vg["cell_face_off"][j], vg["cell_face_off"][j + 1])
              if abs(_area(vg["verts"][vg["face_vert_off"][f]:vg["face_vert_off"][f + 1]], vg["normals"][f])) >= 1e-10}
        assert fo == fg, j
    assert np.all(np.abs(g["vg"]["volume"] - cells.volume) <= 1e-12 * cells.volume)
    assert np.all(np.abs(g["w64"] - wo) <= 1e-12 * np.abs(wo) + 1e-14)
    assert np.all(np.abs(g["wm"] - wo) <= 1e-5 * np.abs(wo) + 1e-14)
    assert np.all(np.abs(g["rho64"] - rho_o) <= 1e-12 * np.abs(rho_o) + 1e-13 * rho_o.max())
    assert np.all(np.abs(g["rhom"] - rho_o) <= 1e-5 * np.abs(rho_o) + 1e-13 * rho_o.max())
    # particles whose support lies inside the unit cube see all of their kernel
    inner = np.all((np.stack([w.x, w.y, w.z], 1) > 2 * w.h[:, None])
                   & (np.stack([w.x, w.y, w.z], 1) < 1 - 2 * w.h[:, None]), axis=1)
    assert inner.sum() > 50
    assert np.max(np.abs(g["u64"][inner] - 1)) < 1e-12 and np.max(np.abs(g["um"][inner] - 1)) < 1e-6


def test_sphere_1e5_sampled(ctx, orc):
    w = inputs.workload_sphere_100k()
    g = _gpu_chain(ctx, w)
    pg, vg = g["pg"], g["vg"]
    assert pg["pair_i"].shape[0] > 4_000_000
    gen = np.stack([w.gx, w.gy, w.gz], 1)
    rng = np.random.default_rng(23)
    checked = 0
    for a in rng.choice(w.n, 10, replace=False):
        p = np.array([w.x[a], w.y[a], w.z[a]])
        d = np.linalg.norm(gen - p, axis=1)
        cand = np.flatnonzero(d <= 4.0 * w.h[a] + d.min() + 1e-12)
        cells = orc.voronoi(w.gx, w.gy, w.gz, w.box, cells=cand)
        one = lambda v: np.array([v], dtype=np.float64)
        po = orc.find_pairs(one(p[0]), one(p[1]), one(p[2]), one(w.h[a]), cells)
        js_o = cells.cell_ids[po.pair_j]
        mine = np.flatnonzero(pg["pair_i"] == a)
        assert np.array_equal(np.sort(js_o), pg["pair_j"][mine]), a
        wo = orc.map_exact_list(po.pair_i, po.pair_j, one(p[0]), one(p[1]), one(p[2]), one(w.h[a]), cells)
        order = np.argsort(js_o)
        wo = wo[order]
        assert np.all(np.abs(g["w64"][mine] - wo) <= 1e-12 * np.abs(wo) + 1e-14)
        assert np.all(np.abs(g["wm"][mine] - wo) <= 1e-5 * np.abs(wo) + 1e-14)
        for jloc in range(cells.ncell):
            j = int(cells.cell_ids[jloc])
            assert abs(vg["volume"][j] - cells.volume[jloc]) <= 1e-12 * cells.volume[jloc]
        checked += mine.shape[0]
    assert checked > 300
    # every pair: mixed against FP64; every particle: partition of unity (the box
    # holds every kernel); mass
    assert np.all(np.abs(g["wm"] - g["w64"]) <= 1e-5 * np.abs(g["w64"]) + 1e-14)
    assert np.max(np.abs(g["u64"] - 1)) < 1e-12 and np.max(np.abs(g["um"] - 1)) < 1e-6
    mass = float(w.m.sum())
    assert abs(float((g["rho64"] * vg["volume"]).sum()) - mass) <= 1e-12 * mass
    assert abs(float((g["rhom"] * vg["volume"]).sum()) - mass) <= 1e-6 * mass
