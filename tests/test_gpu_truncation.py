"""Mixed-precision weights in the regime where the FP32 pass's quadrature
truncation, not its rounding, sets the error: tiny cells deep inside large
kernels (h / V^(1/3) of 12 to 24 for the cluster's cells), the particle in
the kernel's outer shell (r / h of 1.1 to 1.6), so that the faces of the small
cells lie beyond h, where the second kernel piece carries the integral and the
pyramid terms of a cell cancel by about h / V^(1/3).

On the oracle's cells and pair lists (imported through the C ABI, so only the
mapping is compared), every mixed weight must be within the mixed mode's
tolerance of the oracle's FP64 weight: 1e-5 |w| + 1e-14."""
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


@pytest.mark.parametrize("n_sites,seed", [(400, 41), (1000, 42), (2500, 43)])
def test_mixed_weights_in_the_outer_shell(orc, ctx, n_sites, seed):
    w = inputs.dense_cluster(n_sites=n_sites, n_outer=80, n_part=96, seed=seed)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs = orc.find_pairs(w.x, w.y, w.z, w.h, cells)
    wo = orc.map_exact(pairs, w.x, w.y, w.z, w.h, cells)
    vor = api.voronoi_from_cells(ctx, dev(cells.gen.reshape(-1)), dev(cells.cell_face_off, torch.int64),
                                 dev(cells.face_vert_off, torch.int64), dev(cells.verts.reshape(-1)),
                                 dev(cells.normals.reshape(-1)), dev(cells.nbr, torch.int64), dev(cells.volume))
    pr = api.pairs_from_list(ctx, dev(pairs.pair_i, torch.int32), dev(pairs.pair_j, torch.int32), w.n, vor)
    X = [dev(a) for a in (w.x, w.y, w.z, w.h, w.m)]
    wm, _, u, nf = api.map_exact(ctx, pr, *X, vor, api.Params(precision=1, fp64_threshold=1e-5))
    wm, u = wm.cpu().numpy(), u.cpu().numpy()
    assert pairs.n > 30000
    err = np.abs(wm - wo)
    tol = 1e-5 * np.abs(wo) + 1e-14
    worst = int(np.argmax(err / tol))
    assert np.all(err <= tol), (int(np.sum(err > tol)), float(err[worst] / np.abs(wo[worst])), float(wo[worst]))
    # every particle's kernel lies inside the box: the weights sum to 1
    assert np.max(np.abs(u - 1)) < 1e-6
    assert nf < 0.5 * pairs.n
