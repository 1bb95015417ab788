"""GPU parity of map_exact and map_back against the oracle, on cells and pair
lists the oracle built (imported through the C ABI), so that only the mapping
is compared.

Tolerances (derived from the arithmetic): every term of the signed face sum
is bounded by 1/2 and a cell has O(100) edge terms, so FP64 rounding leaves
an absolute floor near 1e-15 on each side; hence
    FP64:  |w_gpu - w_oracle| <= 1e-12 |w_oracle| + 1e-14.
Mixed mode must meet the 1e-5 relative target; pairs whose estimated FP32
error is too large are recomputed in FP64 by the library itself."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api, inputs

pytestmark = pytest.mark.gpu

TOL_REL, TOL_ABS = 1e-12, 1e-14


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def ctx():
    return api.Context(0)


def import_cells(ctx, cells):
    return api.voronoi_from_cells(ctx, dev(cells.gen.reshape(-1)), dev(cells.cell_face_off, torch.int64),
                                  dev(cells.face_vert_off, torch.int64), dev(cells.verts.reshape(-1)),
                                  dev(cells.normals.reshape(-1)), dev(cells.nbr, torch.int64),
                                  dev(cells.volume))


def _case(orc, w):
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs = orc.find_pairs(w.x, w.y, w.z, w.h, cells)
    wts = orc.map_exact(pairs, w.x, w.y, w.z, w.h, cells)
    rho = orc.cell_density(pairs, wts, w.m, cells.volume)
    u = orc.particle_weight_sum(pairs, wts, w.n)
    return dict(w=w, cells=cells, pairs=pairs, wts=wts, rho=rho, u=u)


@pytest.fixture(scope="module", params=["cube", "sphere"])
def case(request, orc):
    if request.param == "cube":
        w = inputs.uniform_cube(500, 333, seed=12, gen_seed=13)
    else:
        w = inputs.sphere_workload(4000, 1000, 1.0, seed=14, field_seed=14)
    return _case(orc, w)


def run_gpu(ctx, c, precision=0, threshold=1e-6, block_pairs=0):
    w = c["w"]
    vor = import_cells(ctx, c["cells"])
    pr = api.pairs_from_list(ctx, dev(c["pairs"].pair_i, torch.int32), dev(c["pairs"].pair_j, torch.int32),
                             w.n, vor)
    res = api.map_exact(ctx, pr, dev(w.x), dev(w.y), dev(w.z), dev(w.h), dev(w.m), vor,
                        api.Params(precision=precision, fp64_threshold=threshold, block_pairs=block_pairs))
    torch.cuda.synchronize()
    return vor, pr, res


def test_map_exact_fp64_parity(ctx, case):
    _, _, (wg, rho, u, nf) = run_gpu(ctx, case, 0)
    wo = case["wts"]
    wg = wg.cpu().numpy()
    assert case["pairs"].n > 1000
    err = np.abs(wg - wo)
    assert np.all(err <= TOL_REL * np.abs(wo) + TOL_ABS), (err.max(), np.argmax(err / (np.abs(wo) + 1e-300)))
    r = rho.cpu().numpy()
    assert np.all(np.abs(r - case["rho"]) <= TOL_REL * np.abs(case["rho"]) + 1e-13 * case["rho"].max())
    assert np.max(np.abs(u.cpu().numpy() - case["u"])) < 1e-13
    assert nf == 0


@pytest.mark.parametrize("precision", [0, 1])
def test_map_exact_deterministic(ctx, case, precision):
    _, _, (a, ra, ua, na) = run_gpu(ctx, case, precision, 1e-5)
    _, _, (b, rb, ub, nb) = run_gpu(ctx, case, precision, 1e-5)
    assert torch.equal(a, b) and torch.equal(ra, rb) and torch.equal(ua, ub) and na == nb


@pytest.mark.parametrize("block_pairs", [32, 64, 96])
def test_map_exact_fp64_block_shape(ctx, case, block_pairs):
    """The FP64 kernels compute each pair with one warp whatever the block
    size, so every launch shape gives the same bits."""
    _, _, (a, ra, _, _) = run_gpu(ctx, case, 0)
    _, _, (b, rb, _, _) = run_gpu(ctx, case, 0, block_pairs=block_pairs)
    assert torch.equal(a, b) and torch.equal(ra, rb)
    _, _, (c, _, _, nc) = run_gpu(ctx, case, 1, 1e-5)
    _, _, (d, _, _, nd) = run_gpu(ctx, case, 1, 1e-5, block_pairs=block_pairs)
    assert torch.equal(c, d) and nc == nd


def test_map_exact_mixed(ctx, case):
    _, _, (wg, rho, u, nf) = run_gpu(ctx, case, 1, 1e-5)
    wo = case["wts"]
    wg = wg.cpu().numpy()
    # 1e-5 relative, down to the FP64 absolute floor that the oracle itself has
    err = np.abs(wg - wo)
    bad = err > 1e-5 * np.abs(wo) + TOL_ABS
    assert not bad.any(), (np.flatnonzero(bad)[:8], wg[bad][:8], wo[bad][:8], nf)
    w = case["w"]
    un = u.cpu().numpy()
    interior = case["u"] > 1 - 1e-12
    assert np.max(np.abs(un[interior] - 1)) < 1e-6
    r = rho.cpu().numpy()
    assert np.all(np.abs(r - case["rho"]) <= 1e-5 * np.abs(case["rho"]))
    mass_o = (case["rho"] * case["cells"].volume).sum()
    assert abs((r * case["cells"].volume).sum() - mass_o) <= 1e-6 * mass_o
    assert 0 <= nf <= case["pairs"].n
    del w


def test_map_back_parity(ctx, case, orc):
    vor, pr, (wg, _, _, _) = run_gpu(ctx, case, 0)
    rng = np.random.default_rng(5)
    f = rng.random(case["cells"].ncell)
    fo = orc.map_back(case["pairs"], case["wts"], f, case["w"].n)
    fg, _ = api.map_back(ctx, pr, wg, dev(f))
    fg = fg.cpu().numpy()
    have = np.isfinite(fo)
    assert np.array_equal(have, np.isfinite(fg))
    assert np.max(np.abs(fg[have] - fo[have])) < 1e-12
    fc, _ = api.map_back(ctx, pr, wg, dev(np.full(case["cells"].ncell, 0.25)))
    assert np.max(np.abs(fc.cpu().numpy()[have] - 0.25)) < 1e-15


def test_empty_and_single_pair(ctx, orc):
    w = inputs.uniform_cube(30, 20, seed=1, gen_seed=2)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    vor = import_cells(ctx, cells)
    pr = api.pairs_from_list(ctx, dev(np.zeros(0), torch.int32), dev(np.zeros(0), torch.int32), w.n, vor)
    wg, rho, u, _ = api.map_exact(ctx, pr, dev(w.x), dev(w.y), dev(w.z), dev(w.h), dev(w.m), vor,
                                  api.Params())
    torch.cuda.synchronize()
    assert wg.numel() == 0 and torch.all(rho == 0) and torch.all(u == 0)
    pairs = orc.find_pairs(w.x, w.y, w.z, w.h, cells)
    k = pairs.n // 2
    one_i, one_j = pairs.pair_i[k:k + 1], pairs.pair_j[k:k + 1]
    pr = api.pairs_from_list(ctx, dev(one_i, torch.int32), dev(one_j, torch.int32), w.n, vor)
    wg, _, _, _ = api.map_exact(ctx, pr, dev(w.x), dev(w.y), dev(w.z), dev(w.h), dev(w.m), vor, api.Params())
    wo = orc.map_exact_list(one_i, one_j, w.x, w.y, w.z, w.h, cells)
    assert abs(wg.item() - wo[0]) <= TOL_REL * abs(wo[0]) + TOL_ABS


def test_unsorted_pair_list_rejected(ctx, orc):
    w = inputs.uniform_cube(30, 20, seed=1, gen_seed=2)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    vor = import_cells(ctx, cells)
    from paper_2410_15227_gb300 import _native
    with pytest.raises(_native.NativeError):
        api.pairs_from_list(ctx, dev([0, 1], torch.int32), dev([3, 2], torch.int32), w.n, vor)


def _mixed_vs_oracle(ctx, orc, cells, x, y, z, h, m, n):
    pairs = orc.find_pairs(x, y, z, h, cells)
    wo = orc.map_exact(pairs, x, y, z, h, cells)
    vor = import_cells(ctx, cells)
    pr = api.pairs_from_list(ctx, dev(pairs.pair_i, torch.int32), dev(pairs.pair_j, torch.int32), n, vor)
    wg, _, _, nf = api.map_exact(ctx, pr, dev(x), dev(y), dev(z), dev(h), dev(m), vor,
                                 api.Params(precision=1, fp64_threshold=1e-5))
    return pairs, wo, wg.cpu().numpy(), nf


def test_mixed_particle_on_a_face(ctx, orc):
    """A particle on the face shared by two cells (the centre of mass of two
    equal-mass particles that are both generators lies there).  In the
    complement form that face subtends a half-space, so an exactly coplanar
    particle must reach the FP64 pass; a particle within rounding of the plane
    is handled by the FP32 form itself.  Both must match the oracle."""
    # exact: two half-box cells, P at the centre of the box; symmetry gives 1/2 each
    g = np.array([0.25, 0.75])
    cells = orc.voronoi(g, np.full(2, 0.5), np.full(2, 0.5), np.array([0., 1., 0., 1., 0., 1.]))
    one = lambda v: np.array([v], dtype=np.float64)
    pairs, wo, wg, nf = _mixed_vs_oracle(ctx, orc, cells, one(0.5), one(0.5), one(0.5), one(0.2), one(1.0), 1)
    assert pairs.n == 2 and nf >= 1
    assert np.all(np.abs(wo - 0.5) < 1e-14) and np.all(np.abs(wg - 0.5) <= 1e-5 * 0.5)
    # within rounding of the plane: the midpoint of two neighbours of a random tessellation
    w = inputs.uniform_cube(40, 60, seed=21, gen_seed=22)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    j, nb = 19, 34   # neighbours whose midpoint lies inside their shared face, 0.43 from the walls
    mid = 0.5 * (cells.gen[j] + cells.gen[nb])
    assert nb in [f[2] for f in cells.faces(j)]
    assert orc.cell_distance(mid, cells, j) == 0.0 and orc.cell_distance(mid, cells, nb) == 0.0
    x, y, z, h = w.x.copy(), w.y.copy(), w.z.copy(), w.h.copy()
    x[0], y[0], z[0] = mid
    h[0] = 0.2
    pairs, wo, wg, nf = _mixed_vs_oracle(ctx, orc, cells, x, y, z, h, w.m, w.n)
    assert np.all(np.abs(wg - wo) <= 1e-5 * np.abs(wo) + TOL_ABS)
    mine = pairs.pair_i == 0
    assert abs(wo[mine].sum() - 1.0) < 1e-12 and abs(wg[mine].sum() - 1.0) < 1e-6


def test_mixed_weight_independent_of_warp_neighbours(ctx, case):
    """A pair's mixed weight does not depend on which pairs share its warp:
    every third pair mapped on its own list (so in other warps, with other
    neighbours) gives the same bits as in the whole list."""
    w, c = case["w"], case
    vor, pr, (wg, _, _, _) = run_gpu(ctx, c, 1, 1e-5)
    sel = np.arange(0, c["pairs"].n, 3)
    sub = api.pairs_from_list(ctx, dev(c["pairs"].pair_i[sel], torch.int32), dev(c["pairs"].pair_j[sel], torch.int32),
                              w.n, vor)
    ws, _, _, _ = api.map_exact(ctx, sub, dev(w.x), dev(w.y), dev(w.z), dev(w.h), dev(w.m), vor,
                                api.Params(precision=1, fp64_threshold=1e-5))
    torch.cuda.synchronize()
    assert torch.equal(ws, wg[torch.as_tensor(sel, device="cuda")])
