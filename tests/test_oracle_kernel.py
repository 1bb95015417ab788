"""Pins of the oracle's kernel and of its analytic cell integral against what
the mathematics fixes: kernel normalisation, the half-space closed form, the
octant/edge/face fractions, symmetry, an independent ray quadrature, direct
face quadrature and Monte Carlo.  CPU only."""
import math

import numpy as np
import pytest
from scipy import integrate


def w_shape(q):
    """M4 shape written out again here, independently of the oracle."""
    if q < 1:
        return 1 - 1.5 * q * q + 0.75 * q ** 3
    if q < 2:
        return 0.25 * (2 - q) ** 3
    return 0.0


def test_kernel_normalisation(orc):
    # 4 pi int_0^2h W r^2 dr = 1 (Section 2.4.2: cubic spline truncated at 2h)
    for h in (0.3, 1.0, 2.7):
        val, _ = integrate.quad(lambda r: orc.W(r, h) * r * r, 0, 2 * h, points=[h], epsabs=1e-15)
        assert abs(4 * math.pi * val - 1) < 1e-13
    assert abs(orc.G(2.0, 1.0) - 1 / (4 * math.pi)) < 1e-16
    assert orc.W(2.0, 1.0) == 0.0 and orc.W(5.0, 1.0) == 0.0
    assert abs(orc.W(0.0, 1.0) - 1 / math.pi) < 1e-16


def test_kernel_shape_matches_textbook(orc):
    for q in np.linspace(0, 2.5, 51):
        assert abs(orc.W(q, 1.0) - w_shape(q) / math.pi) < 1e-15


def test_cumulative_G_is_integral_of_W(orc):
    for R in (0.0, 0.3, 0.99, 1.0, 1.4, 1.999, 2.0, 3.0):
        val, _ = integrate.quad(lambda r: w_shape(r) / math.pi * r * r, 0, min(R, 2.0),
                                points=[1.0] if R > 1 else None, epsabs=1e-15)
        assert abs(orc.G(R, 1.0) - val) < 1e-14


def test_K_is_antiderivative_of_g_over_Q2(orc):
    # K'(Q) = g(Q)/Q^2, K continuous at Q = 1 and Q = 2, K(0) = 0
    for Q in (0.2, 0.7, 1.3, 1.8, 2.5):
        eps = 1e-6
        num = (orc.K(Q + eps) - orc.K(Q - eps)) / (2 * eps)
        g = orc.G(Q, 1.0) * math.pi
        assert abs(num - g / Q ** 2) < 1e-8
    for Q in (1.0, 2.0):
        assert abs(orc.K(Q - 1e-12) - orc.K(Q + 1e-12)) < 1e-10
    assert orc.K(0.0) == 0.0


def test_dWdh_finite_difference(orc):
    for r in (0.0, 0.5, 1.2, 1.9):
        for h in (0.8, 1.1):
            e = 1e-6
            num = (orc.W(r, h + e) - orc.W(r, h - e)) / (2 * e)
            assert abs(orc.dWdh(r, h) - num) < 1e-7


def _rt_quad(D, A, T):
    """(1/pi) int_0^phi_X dphi int_0^{A/cos phi} g(sqrt(D^2+rho^2)) D rho/(D^2+rho^2)^1.5 drho
    by scipy quadrature with the kernel breakpoints (no closed form)."""
    def g(Q):
        return integrate.quad(lambda q: w_shape(q) * q * q, 0, min(Q, 2.0),
                              points=[1.0] if Q > 1 else None, epsabs=1e-15)[0]

    def inner(phi):
        re = A / math.cos(phi)
        pts = [math.sqrt(Q * Q - D * D) for Q in (1, 2) if Q > D and math.sqrt(Q * Q - D * D) < re]
        return integrate.quad(lambda r: g(math.hypot(D, r)) * D * r / (D * D + r * r) ** 1.5, 0, re,
                              points=pts or None, epsabs=1e-14, limit=200)[0]

    phx = math.atan(T / A)
    pts = [math.acos(A / math.sqrt(Q * Q - D * D)) for Q in (1, 2)
           if Q > D and math.sqrt(Q * Q - D * D) > A and math.acos(A / math.sqrt(Q * Q - D * D)) < phx]
    return integrate.quad(inner, 0, phx, points=pts or None, epsabs=1e-14, limit=200)[0] / math.pi


@pytest.mark.parametrize("D,A,T", [(0.3, 0.4, 0.5), (0.9, 0.2, 2.5), (1.4, 0.7, 0.3),
                                   (0.1, 1.5, 3.0), (1.9, 0.05, 0.8), (2.3, 0.6, 1.1)])
def test_right_triangle_vs_quadrature(orc, D, A, T):
    assert abs(orc.right_triangle(D, A, T) - _rt_quad(D, A, T)) < 1e-11
    assert orc.right_triangle(D, A, -T) == -orc.right_triangle(D, A, T)


def test_right_triangle_far_is_solid_angle(orc):
    # d >= 2h: the pyramid holds the kernel's whole mass per solid angle, 1/(4 pi)
    D, A, T = 2.5, 0.7, 1.3
    a, b = D, A
    # solid angle of the right triangle (P,F,X) seen from height D
    omega = math.atan(T / A) - math.atan(D * T / (A * math.sqrt(D * D + A * A + T * T)))
    assert abs(orc.right_triangle(D, A, T) - omega / (4 * math.pi)) < 1e-15
    del a, b


def _halfspace_exact(d, h=1.0):
    """w for the half-space {z > d}: 2 pi int_d^2h dz int_z^2h W(r) r dr, exact rational
    polynomial by sympy (independent of the cone decomposition)."""
    import sympy as sp
    r, z, dd = sp.symbols("r z d", nonnegative=True)
    W1 = (1 - sp.Rational(3, 2) * r ** 2 + sp.Rational(3, 4) * r ** 3) / sp.pi
    W2 = sp.Rational(1, 4) * (2 - r) ** 3 / sp.pi
    inner_lo = sp.integrate(W1 * r, (r, z, 1)) + sp.integrate(W2 * r, (r, 1, 2))   # z < 1
    inner_hi = sp.integrate(W2 * r, (r, z, 2))                                     # 1 <= z < 2
    if d < 1:
        val = 2 * sp.pi * (sp.integrate(inner_lo, (z, dd, 1)) + sp.integrate(inner_hi, (z, 1, 2)))
    else:
        val = 2 * sp.pi * sp.integrate(inner_hi, (z, dd, 2))
    return float(sp.nsimplify(val).subs(dd, sp.Rational(d).limit_denominator(10 ** 12)))


@pytest.mark.parametrize("d", [0.05, 0.4, 0.95, 1.0, 1.3, 1.75, 1.99])
def test_halfspace_closed_form(orc, d):
    # a box much larger than 2h with one face at distance d from p
    c = orc.cells_from_faces([orc.box_cell([-9, -9, d], [9, 9, 9])])
    w = orc.cell_weight([0, 0, 0], 1.0, c)
    assert abs(w - _halfspace_exact(d)) < 2e-15


def test_halfspace_complement(orc):
    # the two half-spaces split the kernel: w(z>d) + w(z<d) = 1
    for d in (0.2, 1.1, 1.7):
        a = orc.cells_from_faces([orc.box_cell([-9, -9, d], [9, 9, 9])])
        b = orc.cells_from_faces([orc.box_cell([-9, -9, -9], [9, 9, d])])
        s = orc.cell_weight([0, 0, 0], 1.0, a) + orc.cell_weight([0, 0, 0], 1.0, b)
        assert abs(s - 1) < 1e-14


def test_box_around_particle_is_one(orc):
    c = orc.cells_from_faces([orc.box_cell([-2.2, -2.5, -3], [2.1, 2.6, 2.05])])
    assert abs(orc.cell_weight([0.01, -0.02, 0.03], 1.0, c) - 1) < 1e-14


@pytest.mark.parametrize("h", [0.3, 0.9])
def test_octant_edge_face_fractions(orc, h):
    side = 4 * h + 0.1
    c = orc.cells_from_faces([orc.box_cell([0, 0, 0], [side, side, side])])
    assert abs(orc.cell_weight([0, 0, 0], h, c) - 1 / 8) < 1e-14             # shared vertex
    assert abs(orc.cell_weight([side / 2, 0, 0], h, c) - 1 / 4) < 1e-14      # shared edge
    assert abs(orc.cell_weight([side / 2, side / 2, 0], h, c) - 1 / 2) < 1e-14  # shared face


def test_cube_symmetry(orc):
    # mirror and 90-degree rotations of p about a cubic cell's centre give the same w
    c = orc.cells_from_faces([orc.box_cell([-0.5, -0.5, -0.5], [0.5, 0.5, 0.5])])
    rng = np.random.default_rng(4)
    for _ in range(4):
        p = rng.uniform(-1.2, 1.2, 3)
        h = rng.uniform(0.2, 0.9)
        ref = orc.cell_weight(p, h, c)
        for q in ([-p[0], p[1], p[2]], [p[1], p[0], p[2]], [p[0], -p[2], p[1]],
                  [p[2], p[0], p[1]], [-p[0], -p[1], -p[2]]):
            assert abs(orc.cell_weight(q, h, c) - ref) < 1e-14


def _random_convex_cell(orc, rng, n_planes=12):
    """A Voronoi-like convex cell: the unit box around the origin clipped by random
    planes, built with the oracle's brute-force clipper on generators."""
    g = np.concatenate([np.zeros((1, 3)), rng.normal(size=(n_planes, 3)) * 0.7])
    cells = orc.voronoi(g[:, 0], g[:, 1], g[:, 2], [-1, 1, -1, 1, -1, 1], cells=[0])
    return cells


def test_ray_quadrature_agrees(orc):
    rng = np.random.default_rng(7)
    for _ in range(3):
        cells = _random_convex_cell(orc, rng)
        for _ in range(2):
            p = rng.uniform(-1.0, 1.0, 3)
            h = rng.uniform(0.15, 0.7)
            a = orc.cell_weight(p, h, cells)
            b = orc.cell_weight_quadrature(p, h, cells, 0, 1e-10)
            assert abs(a - b) < 5e-8, (a, b)


def test_monte_carlo(orc):
    rng = np.random.default_rng(8)
    cells = _random_convex_cell(orc, rng)
    nrm = cells.normals
    off = cells.offsets()
    for _ in range(2):
        p = rng.uniform(-0.5, 0.5, 3)
        h = rng.uniform(0.2, 0.5)
        n = 2_000_000
        u = rng.normal(size=(n, 3))
        u /= np.linalg.norm(u, axis=1)[:, None]
        r = 2 * h * rng.random(n) ** (1 / 3)
        pts = p + u * r[:, None]
        inside = np.all(pts @ nrm.T <= off, axis=1)
        Wv = np.array([w_shape(q) for q in (r[:20000] / h)])  # shape check on a slice
        q = r / h
        wv = np.where(q < 1, 1 - 1.5 * q ** 2 + 0.75 * q ** 3, 0.25 * (2 - q) ** 3) / (math.pi * h ** 3)
        assert np.allclose(wv[:20000], Wv / (math.pi * h ** 3))
        vol = 4 / 3 * math.pi * (2 * h) ** 3
        samples = vol * wv * inside
        est, err = samples.mean(), samples.std() / math.sqrt(n)
        w = orc.cell_weight(p, h, cells)
        assert abs(w - est) < 5 * err + 1e-12, (w, est, err)


def test_planted_mistakes_are_caught(orc):
    # A reversed vertex loop (wrong face orientation) changes the closed form; a
    # flipped normal changes the planes the ray quadrature sees.  Either way the
    # closed form and the quadrature then disagree.
    rng = np.random.default_rng(9)
    cells = _random_convex_cell(orc, rng)
    p, h = np.array([0.1, -0.05, 0.02]), 0.4
    good = orc.cell_weight(p, h, cells)
    assert abs(good - orc.cell_weight_quadrature(p, h, cells, 0, 1e-10)) < 5e-8
    bad = cells.sub(0)
    v0, v1 = bad.face_vert_off[0], bad.face_vert_off[1]
    bad.verts = bad.verts.copy()
    bad.verts[v0:v1] = bad.verts[v0:v1][::-1]
    assert abs(orc.cell_weight(p, h, bad) - orc.cell_weight_quadrature(p, h, bad, 0, 1e-10)) > 1e-4
    bad = cells.sub(0)
    bad.normals = bad.normals.copy()
    bad.normals[0] *= -1
    assert abs(orc.cell_weight(p, h, bad) - orc.cell_weight_quadrature(p, h, bad, 0, 1e-10)) > 1e-4
