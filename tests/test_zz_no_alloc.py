"""map_exact_noalloc, the variant of map_exact for callers that cannot
allocate device memory during the call (a simulation code that owns all free
device memory through its own pool, or one that cannot take an allocation's
synchronisation every time step), against map_exact on the same inputs: identical weights, densities, sums and FP64
counts, on two calls in a row (the fixed counter must be reset by each call),
in both precision modes; and the capacity check.  Collected last so that it
also runs after every other GPU test in the same process."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import _native, api, inputs

pytestmark = pytest.mark.gpu


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def ctx():
    return api.Context(0)


@pytest.fixture(scope="module")
def setup(ctx, orc):
    w = inputs.sphere_workload(4000, 1000, 1.0, seed=14, field_seed=14)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    vor = api.voronoi_from_cells(ctx, dev(cells.gen.reshape(-1)), dev(cells.cell_face_off, torch.int64),
                                 dev(cells.face_vert_off, torch.int64), dev(cells.verts.reshape(-1)),
                                 dev(cells.normals.reshape(-1)), dev(cells.nbr, torch.int64), dev(cells.volume))
    X = [dev(a) for a in (w.x, w.y, w.z, w.h, w.m)]
    pr = api.find_pairs(ctx, *X[:4], vor)
    return w, vor, pr, X


@pytest.mark.parametrize("precision", [1, 0])
def test_noalloc_matches_map_exact_twice(ctx, setup, precision):
    w, vor, pr, X = setup
    P = api.Params(precision=precision, fp64_threshold=1e-5)
    ref = api.map_exact(ctx, pr, *X, vor, P)
    npairs, np_, nc = pr.info()
    assert 0 < npairs <= api.NOALLOC_MAX_PAIRS
    for _ in range(2):
        out = (ctx.empty(npairs), ctx.empty(nc), ctx.empty(np_))
        got = api.map_exact_noalloc(ctx, pr, *X, vor, P, out)
        torch.cuda.synchronize()
        for a, b in zip(ref[:3], got[:3]):
            assert torch.equal(a, b)
        assert got[3] == ref[3]
    if precision == 1:
        assert ref[3] > 0   # the fixed flagged list was exercised


def test_noalloc_rejects_too_many_pairs(ctx):
    # a valid pair list one entry over capacity: particle i with cell 0
    n = api.NOALLOC_MAX_PAIRS + 1
    w = inputs.uniform_cube(30, 20, seed=1, gen_seed=2)
    from test_gpu_mapping import import_cells
    import oracle
    vor = import_cells(ctx, oracle.voronoi(w.gx, w.gy, w.gz, w.box))
    pi = torch.arange(n, dtype=torch.int32, device="cuda")
    pj = torch.zeros(n, dtype=torch.int32, device="cuda")
    pr = api.pairs_from_list(ctx, pi, pj, n, vor)
    z = torch.zeros(n, dtype=torch.float64, device="cuda")
    out = (ctx.empty(n), ctx.empty(vor.info()[0]), None)
    with pytest.raises(_native.NativeError, match="capacity"):
        api.map_exact_noalloc(ctx, pr, z, z, z, z + 0.1, z, vor, api.Params(precision=1), out)
