"""Pins of the oracle's work counter (oracle/count.cpp): the counting build
computes the same weights to the bit, and its per-pair counts follow from the
closed form's structure on cells where the count is known by hand.  CPU only."""
import numpy as np
import pytest

from paper_2410_15227_gb300 import inputs


def one_pair(orc, cells, p, h, j=0):
    pairs = orc.Pairs(np.array([0]), np.array([j]), np.zeros(1, np.uint8), np.zeros(1, np.int64))
    w, c = orc.count_map_exact(pairs, [p[0]], [p[1]], [p[2]], [h], cells)
    return w[0], dict(zip(orc.WORK_FIELDS, (int(v) for v in c[0])))


def test_counted_weights_equal_the_oracles(orc):
    w = inputs.uniform_cube(300, 200, seed=5, gen_seed=6)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs = orc.find_pairs(w.x, w.y, w.z, w.h, cells)
    wo = orc.map_exact(pairs, w.x, w.y, w.z, w.h, cells)
    wc, c = orc.count_map_exact(pairs, w.x, w.y, w.z, w.h, cells)
    assert np.array_equal(wo, wc)
    # the counts of a pair do not depend on how the pairs are spread over threads
    _, c1 = orc.count_map_exact(pairs, w.x, w.y, w.z, w.h, cells, nthreads=1)
    assert np.array_equal(c, c1)
    # a Voronoi cell has ~15 faces of ~5 edges: two right sub-triangles per edge
    assert 100 < c[:, 0].mean() < 200
    assert np.all(c[:, 1:] > 0)


def test_box_cell_counts(orc):
    """A particle strictly inside an axis-aligned box, the foot of every edge
    line strictly inside its edge: 6 faces x 4 edges x 2 right sub-triangles.
    With the particle on the face x = 0 that face is skipped (its plane holds
    P), and on each of the four faces that meet it, the edge on x = 0 has P's
    foot on its line (A = 0: skipped) and the two edges across it have the foot
    of the perpendicular at a vertex (one leg of length 0: skipped), 4 each;
    the face x = 1 keeps its 8: 4 x 4 + 8 = 24."""
    cells = orc.cells_from_faces([orc.box_cell([0, 0, 0], [1, 1, 1])])
    w, c = one_pair(orc, cells, (0.3, 0.4, 0.45), 0.1)
    assert c["right_subtriangles"] == 48
    assert abs(w - 1.0) < 1e-13   # the kernel's support lies inside the box
    _, c = one_pair(orc, cells, (0.0, 0.4, 0.45), 0.1)
    assert c["right_subtriangles"] == 24


def test_transcendental_calls_of_one_region(orc):
    """A single right triangle wholly in the kernel's inner region (Q < 1 on it)
    as the only face: the closed form evaluates the region-1 primitive at the
    leg's end (asinh and two atan2), K(D) (two pow for D < 1) and the reference
    angle atan2, once for each of the triangle's two right sub-triangles."""
    # face in the plane z = 0.2 (outward normal +z) as seen from the origin:
    # a triangle with the foot (0, 0) as a vertex, legs 0.1 along x and y
    v = np.array([[0.0, 0.0, 0.2], [0.1, 0.0, 0.2], [0.0, 0.1, 0.2]])
    cells = orc.cells_from_faces([[(v, np.array([0.0, 0.0, 1.0]))]])
    _, c = one_pair(orc, cells, (0.0, 0.0, 0.0), 1.0)
    # edges: (0,0)-(0.1,0) lies on a line through the foot (A = 0, skipped);
    # (0.1,0)-(0,0.1) has A > 0 and two legs; (0,0.1)-(0,0) has A = 0
    assert c["right_subtriangles"] == 2
    assert c["transcendental"] == 2 * (3 + 2 + 1)
    assert c["sqrt"] >= 2 * 3   # B, t1, t2 and the primitive's S per sub-triangle, plus the face geometry
