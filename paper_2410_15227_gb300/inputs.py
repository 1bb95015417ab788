"""Seeded synthetic workloads shaped like the paper's particle clouds.

This module only draws inputs: particle positions, masses and smoothing
lengths, Voronoi generators, sources and per-cell fields.  It holds none of
the mapping method's arithmetic, so both the CPU oracle and the CUDA path can
consume its arrays.

The paper's own workloads (StarBench glass and evolved turbulent boxes,
Sections 3.1-3.3) are not public; the clouds below stand in for them:

* a uniform cube (the plain Exact-mapping case),
* a unit sphere with density ~ r^-1.5 times a lognormal field drawn from a
  32^3 Gaussian random field with a Kolmogorov-like spectrum P(k) ~ k^-11/3
  (the fractal structure that the turbulent boxes of Section 3.2 develop).

Particle smoothing lengths follow the "57 neighbours" rule: with d_k the
distance to the k-th nearest *other* particle, h = (d_57 + d_58) / 4, so that
exactly 57 other particles lie inside the 2h support sphere.
"""
from __future__ import annotations

import os
from dataclasses import dataclass, field

import numpy as np

N_NEIGH = 57          # neighbours inside 2h for particle smoothing lengths
GRF_N = 32            # Gaussian random field grid per axis, spanning [-1, 1]^3


@dataclass
class Workload:
    """Arrays of one synthetic problem (all float64 unless noted)."""
    name: str
    x: np.ndarray
    y: np.ndarray
    z: np.ndarray
    m: np.ndarray
    h: np.ndarray
    gx: np.ndarray
    gy: np.ndarray
    gz: np.ndarray
    box: np.ndarray                    # [xlo, xhi, ylo, yhi, zlo, zhi]
    sources: np.ndarray = field(default_factory=lambda: np.zeros((0, 3)))
    params: dict = field(default_factory=dict)
    f_cell: np.ndarray | None = None   # per-cell field for the inverse mapping

    @property
    def n(self) -> int:
        return int(self.x.shape[0])

    @property
    def ngen(self) -> int:
        return int(self.gx.shape[0])


def grf(seed: int, n: int = GRF_N) -> np.ndarray:
    """Periodic Gaussian random field on an n^3 grid, P(k) ~ k^-11/3, k=0 removed,
    normalised to zero mean and unit variance."""
    rng = np.random.default_rng([seed, 7])
    noise = rng.standard_normal((n, n, n))
    k1 = np.fft.fftfreq(n) * n
    kx, ky, kz = np.meshgrid(k1, k1, k1, indexing="ij")
    k = np.sqrt(kx * kx + ky * ky + kz * kz)
    amp = np.zeros_like(k)
    nz = k > 0
    amp[nz] = k[nz] ** (-11.0 / 6.0)          # sqrt(P(k))
    g = np.real(np.fft.ifftn(np.fft.fftn(noise) * amp))
    g -= g.mean()
    g /= g.std()
    return g


def _grid_lookup(g: np.ndarray, p: np.ndarray) -> np.ndarray:
    n = g.shape[0]
    idx = np.floor((p + 1.0) * 0.5 * n).astype(np.int64)
    np.clip(idx, 0, n - 1, out=idx)
    return g[idx[:, 0], idx[:, 1], idx[:, 2]]


def sphere_cloud(n: int, sigma: float, seed: int, field_seed: int) -> np.ndarray:
    """n points in the unit sphere with density ~ r^-1.5 * exp(sigma g - sigma^2/2).

    Radius by the inverse CDF of r^-1.5 (mass inside r ~ r^1.5, so r = u^(2/3)),
    isotropic direction, then rejection on the lognormal factor."""
    rng = np.random.default_rng([seed, 11])
    g = grf(field_seed)
    gmax = g.max()
    out = []
    have = 0
    while have < n:
        batch = max(4 * (n - have), 1024)
        u = rng.random(batch)
        r = u ** (2.0 / 3.0)
        v = rng.standard_normal((batch, 3))
        v /= np.linalg.norm(v, axis=1)[:, None]
        p = v * r[:, None]
        acc = rng.random(batch) < np.exp(sigma * (_grid_lookup(g, p) - gmax))
        p = p[acc]
        out.append(p)
        have += p.shape[0]
    return np.concatenate(out)[:n]


def smoothing_lengths(p: np.ndarray, nneigh: int = N_NEIGH) -> np.ndarray:
    """h = (d_nneigh + d_(nneigh+1)) / 4 with d_k the k-th nearest other point."""
    from scipy.spatial import cKDTree
    tree = cKDTree(p)
    d, _ = tree.query(p, k=nneigh + 2, workers=-1)
    return 0.25 * (d[:, nneigh] + d[:, nneigh + 1])


def _sphere_box(p: np.ndarray, h: np.ndarray) -> np.ndarray:
    L = float(np.max(np.max(np.abs(p), axis=1) + 2.0 * h))
    return np.array([-L, L, -L, L, -L, L])


def uniform_cube(n: int, ngen: int, seed: int = 0, gen_seed: int = 1,
                 mass: float | None = None) -> Workload:
    """Uniform particles and generators in the unit cube; domain = unit cube."""
    rng = np.random.default_rng(seed)
    p = rng.random((n, 3))
    g = np.random.default_rng(gen_seed).random((ngen, 3))
    h = smoothing_lengths(p, min(N_NEIGH, n - 2))
    m = np.full(n, 1.0 / n if mass is None else mass)
    return Workload(f"cube_n{n}_g{ngen}", p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(),
                    m, h, g[:, 0].copy(), g[:, 1].copy(), g[:, 2].copy(),
                    np.array([0.0, 1.0, 0.0, 1.0, 0.0, 1.0]))


def sphere_workload(n: int, ngen: int, sigma: float = 1.0, seed: int = 2,
                    field_seed: int = 2, gen_seed: int | None = None,
                    name: str | None = None) -> Workload:
    """Sphere cloud; generators are a random subset of the particles."""
    p = sphere_cloud(n, sigma, seed, field_seed)
    h = smoothing_lengths(p, min(N_NEIGH, n - 2))
    rng = np.random.default_rng([seed if gen_seed is None else gen_seed, 1])
    sel = np.sort(rng.choice(n, size=ngen, replace=False))
    g = p[sel]
    return Workload(name or f"sphere_n{n}_g{ngen}_s{sigma}", p[:, 0].copy(), p[:, 1].copy(),
                    p[:, 2].copy(), np.full(n, 1.0 / n), h, g[:, 0].copy(), g[:, 1].copy(),
                    g[:, 2].copy(), _sphere_box(p, h), sources=np.zeros((1, 3)))


def dense_cluster(n_sites: int = 400, n_outer: int = 80, n_part: int = 96, radius: float = 0.05,
                  seed: int = 41) -> Workload:
    """Tiny cells deep inside large kernels: n_sites sites uniform in a ball of
    the given radius at the origin, n_outer sites uniform in [-1, 1]^3 beyond
    three radii, and n_part particles at distance q h from the origin with q
    uniform in [1.1, 1.6] and h / V^(1/3) uniform in [12, 24], V the mean
    volume of the ball's cells.  Domain [-1, 1]^3, equal masses summing to 1.
    The configuration that stresses the mixed pass: the faces of the small
    cells lie in the kernel's outer shell, where their pyramid terms cancel
    by about h / V^(1/3)."""
    rng = np.random.default_rng(seed)

    def ball(n, r):
        v = rng.normal(size=(n, 3))
        v /= np.linalg.norm(v, axis=1, keepdims=True)
        return v * (r * rng.random(n) ** (1.0 / 3.0))[:, None]

    inner = ball(n_sites, radius)
    outer = []
    while len(outer) < n_outer:
        q = rng.uniform(-1.0, 1.0, 3)
        if np.linalg.norm(q) > 3.0 * radius:
            outer.append(q)
    g = np.concatenate([inner, np.array(outer)])
    ell = (4.0 / 3.0 * np.pi * radius ** 3 / n_sites) ** (1.0 / 3.0)
    h = ell * rng.uniform(12.0, 24.0, n_part)
    d = rng.normal(size=(n_part, 3))
    d /= np.linalg.norm(d, axis=1, keepdims=True)
    p = d * (h * rng.uniform(1.1, 1.6, n_part))[:, None]
    return Workload(f"dense_cluster_{n_sites}_{n_part}", p[:, 0].copy(), p[:, 1].copy(), p[:, 2].copy(),
                    np.full(n_part, 1.0 / n_part), h, g[:, 0].copy(), g[:, 1].copy(), g[:, 2].copy(),
                    np.array([-1.0, 1.0, -1.0, 1.0, -1.0, 1.0]))


# ---------------------------------------------------------------------------
# The five named workloads.  Pseudo-particle parameters (r_part, r_leaf) are the
# paper's Table 1 values read as dimensionless radii; theta for the 1e6-particle
# cloud is the value that yields about 1e5 pseudo-particles.
# ---------------------------------------------------------------------------

PSEUDO_PARAMS = dict(r_part=0.05, r_leaf=0.1, h_fact=1.2)
# on the 1e6-particle cloud below, theta = 0.065 selects 102,908 pseudo-particles
# (88,654 nodes, 5,566 leaves and 8,688 particles inside r_part)
THETA_1E6 = 0.065


def workload_cube_1k() -> Workload:
    """1,000 equal-mass (1e-3) particles uniform in the unit cube (seed 0), h from
    the 57-neighbour rule, 1,000 uniform generators (seed 1), domain = unit cube."""
    w = uniform_cube(1000, 1000, seed=0, gen_seed=1, mass=1e-3)
    w.name = "cube_1k_particles_1k_cells"
    return w


def workload_sphere_100k() -> Workload:
    """1e5 particles, r^-1.5 x lognormal(sigma=1) sphere (seed 2), 25,000 generators."""
    return sphere_workload(100_000, 25_000, 1.0, seed=2, field_seed=2, gen_seed=2,
                           name="sphere_100k_particles_25k_cells")


def workload_pseudo_1e6(theta: float | None = None) -> Workload:
    """1e6 particles of the sphere profile (seed 3, m=1e-6), source at the origin,
    262,144 generators drawn from the particles (seed 3)."""
    w = sphere_workload(1_000_000, 262_144, 1.0, seed=3, field_seed=2, gen_seed=3,
                        name="pseudo_1M_particles_262k_cells")
    w.params = dict(PSEUDO_PARAMS, theta=THETA_1E6 if theta is None else theta)
    return w


def workload_pseudo_2e5() -> Workload:
    """A fifth of the benchmark cloud: 2e5 particles of the sphere profile (seed
    6, m = 5e-6), 52,428 generators drawn from them; theta = 0.12 selects
    19,241 pseudo-particles.  The profiling case of the pseudo-particle path."""
    w = sphere_workload(200_000, 52_428, 1.0, seed=6, field_seed=2, gen_seed=6,
                        name="pseudo_200k_particles_52k_cells")
    w.params = dict(PSEUDO_PARAMS, theta=0.12)
    return w


def workload_batched(nsnap: int = 64):
    """64 independent sphere snapshots, N_s log-uniform in [1e3, 1e5] (seed 100+s),
    generators 0.25 N_s."""
    out = []
    for s in range(nsnap):
        rng = np.random.default_rng(100 + s)
        ns = int(round(10 ** rng.uniform(3.0, 5.0)))
        out.append(sphere_workload(ns, max(ns // 4, 8), 1.0, seed=100 + s,
                                   field_seed=100 + s, name=f"snapshot_{s}"))
    return out


def workload_full_8m() -> Workload:
    """8e6 particles, sigma=1.5 lognormal (field seed 5), 2e6 generators (seed 4),
    uniform [0,1] per-cell field (seed 5)."""
    w = sphere_workload(8_000_000, 2_000_000, 1.5, seed=5, field_seed=5, gen_seed=4,
                        name="full_8M_particles_2M_cells")
    w.params = dict(PSEUDO_PARAMS, theta=THETA_1E6)
    w.f_cell = np.random.default_rng([5, 3]).random(w.ngen)
    return w


def cached(fn, *args, cache_dir: str | None = None, **kw) -> Workload:
    """Memoise a workload on disk (npz) under cache_dir, if given."""
    if not cache_dir:
        return fn(*args, **kw)
    os.makedirs(cache_dir, exist_ok=True)
    key = fn.__name__ + "_" + "_".join(str(a) for a in args) + "_".join(
        f"{k}{v}" for k, v in sorted(kw.items()))
    path = os.path.join(cache_dir, key + ".npz")
    if os.path.exists(path):
        d = np.load(path, allow_pickle=True)
        w = Workload(str(d["name"]), *(d[k] for k in
                     ("x", "y", "z", "m", "h", "gx", "gy", "gz", "box")),
                     sources=d["sources"], params=d["params"].item(),
                     f_cell=None if d["f_cell"].shape == () else d["f_cell"])
        return w
    w = fn(*args, **kw)
    np.savez(path, name=w.name, x=w.x, y=w.y, z=w.z, m=w.m, h=w.h, gx=w.gx, gy=w.gy,
             gz=w.gz, box=w.box, sources=w.sources, params=np.array(w.params, dtype=object),
             f_cell=np.array(None) if w.f_cell is None else w.f_cell)
    return w
