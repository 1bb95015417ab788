"""build_voronoi on near-degenerate site sets, where the FP32 side tests of
the clipping cannot decide and the vertices' FP64 meets must: a cubic
lattice jittered by 1e-9 of its spacing (four planes nearly through every
vertex, faces of area ~1e-9 of the spacing squared between diagonal
neighbours) and the exact lattice with two sites nudged along a diagonal.

Against the oracle's brute-force cells: every face larger than 1e-10 L^2 on
either side is on both, with the same neighbour; volumes agree to 1e-12
relative and tile the box; faces are reciprocal (i lists j iff j lists i)
above the same size."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device="cuda")


@pytest.fixture(scope="module")
def ctx():
    return api.Context(0)


def _area(v, n):
    s = np.zeros(3)
    for k in range(1, len(v) - 1):
        s += np.cross(v[k] - v[0], v[k + 1] - v[0])
    return 0.5 * float(s @ n)


def lattice(k, jitter, seed):
    c = (np.arange(k) + 0.5) / k
    X, Y, Z = np.meshgrid(c, c, c, indexing="ij")
    p = np.stack([X.ravel(), Y.ravel(), Z.ravel()], axis=1)
    p += np.random.default_rng(seed).uniform(-1.0, 1.0, p.shape) * jitter / k
    return p


CASES = {
    "jittered_1e-9": lambda: lattice(7, 1e-9, 5),
    "nudged": lambda: lattice(6, 0.0, 0) + np.where(np.arange(216)[:, None] == 43, 1e-7, 0.0)
    + np.where(np.arange(216)[:, None] == 100, -2e-8, 0.0),
}


@pytest.mark.parametrize("name", list(CASES))
def test_near_degenerate_sites(ctx, orc, name):
    p = CASES[name]()
    box = np.array([0.0, 1.0, 0.0, 1.0, 0.0, 1.0])
    oc = orc.voronoi(p[:, 0], p[:, 1], p[:, 2], box)
    vor = api.build_voronoi(ctx, dev(p[:, 0]), dev(p[:, 1]), dev(p[:, 2]), box, api.Params())
    g = {k: v.cpu().numpy() for k, v in vor.get().items()}
    n = p.shape[0]
    tol_area = 1e-10
    big_g = []
    for j in range(n):
        fo = {nb: (v, nr) for v, nr, nb in oc.faces(j)}
        fg = {}
        for f in range(g["cell_face_off"][j], g["cell_face_off"][j + 1]):
            fg[int(g["nbr"][f])] = (g["verts"][g["face_vert_off"][f]:g["face_vert_off"][f + 1]], g["normals"][f])
        bo = {k for k, (v, nr) in fo.items() if abs(_area(v, nr)) >= tol_area}
        bg = {k for k, (v, nr) in fg.items() if abs(_area(v, nr)) >= tol_area}
        # every face above the size on one side is a face on the other
        assert bo <= set(fg) and bg <= set(fo), (j, sorted(bo ^ bg))
        for k in bo | bg:
            assert np.allclose(fo[k][1], fg[k][1], atol=1e-12)
        big_g.append(bg)
    vo, vg = oc.volume, g["volume"]
    assert np.max(np.abs(vg - vo) / vo) < 1e-12
    assert abs(vg.sum() - 1.0) < 1e-12
    for j in range(n):
        for k in big_g[j]:
            if k >= 0:
                assert j in big_g[k] or j in {int(x) for x in g["nbr"][g["cell_face_off"][k]:g["cell_face_off"][k + 1]]}
