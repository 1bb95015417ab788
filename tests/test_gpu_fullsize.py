"""Parity at the benchmark's full size, in bench.py's launch configuration:
1,000,000 particles, 102,908 pseudo-particles, 262,144 cells, 24 million
pairs, mapped in mixed precision with the default launch shapes.

What the oracle can compute at this size is compared directly: the whole
octree and pseudo-particle selection (bit for bit), the node smoothing
lengths of sampled pseudo-particles (solved by the oracle against the whole
population), and for sampled pseudo-particles their complete pair lists,
cells and weights.  The candidate cells of a particle p come from a rigorous
bound: a cell j reaches within 2h of p only if |g_j - p| <= 4h + d_p, with
d_p the distance from p to its nearest generator (a point x of the cell with
|x - p| < 2h is no farther from g_j than from the generator nearest p).
The sampled weights are mapped on the GPU with the oracle's own h and pair
list, so that FP64 mode is held to 1e-12.  Properties that hold at any size
are checked over all particles: partition of unity, mass conservation, the
inverse mapping of a constant field, and, for a random cell field, every
particle's value equal to its pseudo-particle's through the oracle's own
membership (Section 2.5)."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api, inputs

pytestmark = pytest.mark.gpu

RNG_SEED = 17


def _area(v, n):
    t = np.zeros(3)
    for k in range(1, len(v) - 1):
        t += np.cross(v[k] - v[0], v[k + 1] - v[0])
    return 0.5 * float(t @ n)


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


@pytest.fixture(scope="module")
def full():
    w = inputs.workload_pseudo_1e6()
    pr_ = w.params
    ctx = api.Context(0)
    X = [dev(a) for a in (w.x, w.y, w.z, w.m, w.h)]
    G = [dev(a) for a in (w.gx, w.gy, w.gz)]
    P = api.Params(r_part=pr_["r_part"], r_leaf=pr_["r_leaf"], theta=pr_["theta"], h_fact=pr_["h_fact"],
                   h_tol=1e-13, precision=1, fp64_threshold=1e-5)
    tree = api.build_tree(ctx, X[0], X[1], X[2], X[3], w.box, 8)
    ps = api.make_pseudo_particles(ctx, tree, X[4], np.zeros((1, 3)), P)
    g = ps.get()
    vor = api.build_voronoi(ctx, *G, w.box, P)
    pairs = api.find_pairs(ctx, g["x"], g["y"], g["z"], g["h"], vor)
    wm, rho_m, u_m, nf = api.map_exact(ctx, pairs, g["x"], g["y"], g["z"], g["h"], g["m"], vor, P)
    w64, rho64, u64, _ = api.map_exact(ctx, pairs, g["x"], g["y"], g["z"], g["h"], g["m"], vor,
                                       api.Params(precision=0))
    torch.cuda.synchronize()
    host = lambda d: {k: v.cpu().numpy() for k, v in d.items()}
    return dict(w=w, ctx=ctx, tree=tree, ps=ps, vor=vor, pairs=pairs, g=host(g), tg=host(tree.get()),
                pg=host(pairs.get()), wm=wm.cpu().numpy(), w64=w64.cpu().numpy(), u_m=u_m.cpu().numpy(),
                u64=u64.cpu().numpy(), rho_m=rho_m.cpu().numpy(), rho64=rho64.cpu().numpy(), nf=nf,
                vg=host(vor.get()))


@pytest.fixture(scope="module")
def oracle_pseudo(full, orc):
    w = full["w"]
    pr_ = w.params
    return orc.make_pseudo_particles(w.x, w.y, w.z, w.m, w.h, w.box, np.zeros((1, 3)), pr_["r_part"],
                                     pr_["r_leaf"], pr_["theta"], h_fact=pr_["h_fact"], solve=False)


def test_tree_and_selection_bit_exact(full, oracle_pseudo):
    ps_o, t_o, _ = oracle_pseudo
    tg, g = full["tg"], full["g"]
    assert np.array_equal(tg["perm"], t_o.perm)
    assert np.array_equal(tg["label"].astype(np.uint64), t_o.label)
    for k in ("level", "parent", "first", "count", "nchild", "mass", "com", "size"):
        assert np.array_equal(tg[k], getattr(t_o, k)), k
    assert g["x"].shape[0] == ps_o.n == 102908
    assert np.array_equal(g["origin"], ps_o.origin)
    for k in ("x", "y", "z", "m"):
        assert np.array_equal(g[k], getattr(ps_o, k)), k


def _sample_nodes(full, oracle_pseudo, n):
    ps_o, _, _ = oracle_pseudo
    rng = np.random.default_rng(RNG_SEED)
    nodes = np.flatnonzero(ps_o.origin > 0)
    parts = np.flatnonzero(ps_o.origin < 0)
    return np.sort(rng.choice(nodes, n, replace=False)), np.sort(rng.choice(parts, 2, replace=False))


@pytest.fixture(scope="module")
def sampled_h(full, oracle_pseudo, orc):
    """Oracle smoothing lengths of sampled node pseudo-particles, solved against
    the whole population (Section 2.4.2)."""
    ps_o, t_o, sel = oracle_pseudo
    tg_nodes, tg_parts = _sample_nodes(full, oracle_pseudo, 40)
    ids = sel.ref[tg_nodes]
    h0 = orc.h_initial(t_o, ids, full["w"].h, full["w"].params["h_fact"])
    h, st, _ = orc.h_solve(t_o.com[sel.pop_node], t_o.com[ids], h0, full["w"].params["h_fact"], 1e-13, 50)
    return tg_nodes, h, st, tg_parts


def test_sampled_node_h(full, sampled_h):
    tg_nodes, h, st, _ = sampled_h
    hg, sg = full["g"]["h"][tg_nodes], full["g"]["status"][tg_nodes]
    ok = (st <= 1) & (sg <= 1)
    assert ok.sum() >= 35
    assert np.all(np.abs(hg[ok] / h[ok] - 1) < 1e-12), np.max(np.abs(hg[ok] / h[ok] - 1))
    assert np.array_equal(st == 2, sg == 2)


@pytest.fixture(scope="module")
def sampled(full, oracle_pseudo, sampled_h, orc):
    """The oracle's cells, pairs and weights of sampled pseudo-particles, each
    with its own h (the oracle's h-solver for nodes, the input h for extracted
    particles), from the candidate cells of the bound in the module docstring.
    Positions are the oracle's own pseudo-particles'."""
    w = full["w"]
    ps_o = oracle_pseudo[0]
    g = dict(x=ps_o.x, y=ps_o.y, z=ps_o.z, origin=ps_o.origin)
    tg_nodes, h_orc, st, tg_parts = sampled_h
    gen = np.stack([w.gx, w.gy, w.gz], 1)
    targets = [(int(a), float(hh)) for a, hh, s in zip(tg_nodes[:6], h_orc[:6], st[:6]) if s <= 1]
    targets += [(int(a), float(w.h[a_part])) for a, a_part in zip(tg_parts, -g["origin"][tg_parts] - 1)]
    out = []
    for a, ha in targets:
        p = np.array([g["x"][a], g["y"][a], g["z"][a]])
        d = np.linalg.norm(gen - p, axis=1)
        cand = np.flatnonzero(d <= 4.0 * ha + d.min() + 1e-12)
        cells = orc.voronoi(w.gx, w.gy, w.gz, w.box, cells=cand)
        one = lambda v: np.array([v], dtype=np.float64)
        po = orc.find_pairs(one(p[0]), one(p[1]), one(p[2]), one(ha), cells)
        wo = orc.map_exact_list(po.pair_i, po.pair_j, one(p[0]), one(p[1]), one(p[2]), one(ha), cells)
        out.append(dict(a=a, h=ha, cells=cells, po=po, js=cells.cell_ids[po.pair_j], wo=wo))
    return out


def test_sampled_pairs_and_cells(full, sampled):
    """Complete pair lists and cells of sampled pseudo-particles: the GPU's own
    pairs (its own h) against the oracle's, up to pairs flagged near the
    support's edge."""
    w, pg, vg = full["w"], full["pg"], full["vg"]
    L = float(np.max(w.box[1::2] - w.box[0::2]))
    cfo, fvo = vg["cell_face_off"], vg["face_vert_off"]
    checked = 0
    for s in sampled:
        a, cells, po, js_o = s["a"], s["cells"], s["po"], s["js"]
        mine = pg["pair_i"] == a
        js_g = pg["pair_j"][mine]
        near = set(js_g[pg["near"][mine] == 1].tolist())
        assert set(js_o.tolist()) - near == set(js_g.tolist()) - near, a
        for jloc, j in zip(po.pair_j, js_o):
            # the cell itself: neighbours (faces above 1e-10 L^2) and volume
            fo = {int(n) for v, nrm, n in cells.faces(int(jloc)) if abs(_area(v, nrm)) >= 1e-10 * L * L}
            fg = set()
            for f in range(cfo[j], cfo[j + 1]):
                v = vg["verts"][fvo[f]:fvo[f + 1]]
                if abs(_area(v, vg["normals"][f])) >= 1e-10 * L * L:
                    fg.add(int(vg["nbr"][f]))
            assert fo == fg, j
            assert abs(vg["volume"][j] - cells.volume[jloc]) <= 1e-12 * cells.volume[jloc]
            checked += 1
    assert checked > 300


@pytest.mark.parametrize("precision,tol", [(0, 1e-12), (1, 1e-5)])
def test_sampled_weights(full, oracle_pseudo, sampled, precision, tol):
    """Weights of the sampled pseudo-particles on the GPU's cells, mapped with
    the oracle's h and the oracle's pair list (pairs_from_list), against the
    oracle's weights: 1e-12 relative in FP64 mode, 1e-5 in mixed mode, above
    the absolute floor 1e-14."""
    ctx, vor = full["ctx"], full["vor"]
    ps_o = oracle_pseudo[0]
    h = ps_o.h.copy()
    pi, pj, wref = [], [], []
    for s in sampled:
        h[s["a"]] = s["h"]
        pi.append(np.full(s["js"].shape[0], s["a"]))
        pj.append(s["js"])
        wref.append(s["wo"])
    pi, pj, wref = np.concatenate(pi), np.concatenate(pj), np.concatenate(wref)
    order = np.lexsort((pi, pj))
    pi, pj, wref = pi[order], pj[order], wref[order]
    pr = api.pairs_from_list(ctx, dev(pi, torch.int32), dev(pj, torch.int32), ps_o.n, vor)
    X = [dev(a) for a in (ps_o.x, ps_o.y, ps_o.z, h, ps_o.m)]
    wg, _, _, _ = api.map_exact(ctx, pr, *X, vor, api.Params(precision=precision, fp64_threshold=1e-5),
                                want_wsum=False)
    wg = wg.cpu().numpy()
    assert wg.shape[0] > 300
    err = np.abs(wg - wref)
    assert np.all(err <= tol * np.abs(wref) + 1e-14), float(np.max(err / (np.abs(wref) + 1e-300)))


def test_partition_of_unity_and_mass(full):
    w, g = full["w"], full["g"]
    L = w.box[1]
    inner = np.max(np.abs(np.stack([g["x"], g["y"], g["z"]], 1)), axis=1) + 2.0 * g["h"] < L
    assert inner.sum() > 90000
    assert np.max(np.abs(full["u64"][inner] - 1)) < 1e-12
    assert np.max(np.abs(full["u_m"][inner] - 1)) < 1e-6
    vol = full["vg"]["volume"]
    mass_cells = float((full["rho64"] * vol).sum())
    mass_parts = float((g["m"] * full["u64"]).sum())
    assert abs(mass_cells - mass_parts) <= 1e-12 * mass_parts
    assert abs(float((full["rho_m"] * vol).sum()) - mass_parts) <= 1e-6 * mass_parts
    # the mixed weights against the FP64 weights over every pair
    big = np.abs(full["w64"]) >= 1e-9
    err = np.abs(full["wm"] - full["w64"])
    assert np.all(err <= 1e-5 * np.abs(full["w64"]) + 1e-14)
    assert np.max(err[big] / np.abs(full["w64"][big])) < 1e-5
    assert 0 < full["nf"] < 0.05 * full["wm"].shape[0]


def test_map_back_random_field(full, oracle_pseudo, sampled, orc):
    """Inverse mapping of a random cell field (uniform [0, 1], seed 5) at full
    size.  Every particle's value is its pseudo-particle's, through the
    oracle's own membership of the 1e6 particles (tree and selection, Section
    2.5); the sampled pseudo-particles' values equal the weighted means of the
    oracle's own pairs and weights, within the weights' tolerance carried into
    a mean of values in [0, 1] (twice the relative error)."""
    ctx, pairs, ps, tree = full["ctx"], full["pairs"], full["ps"], full["tree"]
    nc = full["vg"]["volume"].shape[0]
    f_cell = np.random.default_rng([5, 5]).random(nc)
    ps_o, t_o, _ = oracle_pseudo
    owner = orc.inherit(ps_o, t_o, np.arange(ps_o.n, dtype=np.float64)).astype(np.int64)
    for wk, tol in (("w64", 1e-8), ("wm", 2e-5)):
        f, fp = api.map_back(ctx, pairs, torch.as_tensor(full[wk], device="cuda"), dev(f_cell), ps, tree)
        f, fp = f.cpu().numpy(), fp.cpu().numpy()
        assert np.all(np.isfinite(f)) and np.std(fp) > 0.02
        assert np.array_equal(fp, f[owner])
        for s in sampled:
            fo = float(np.sum(s["wo"] * f_cell[s["js"]]) / np.sum(s["wo"]))
            assert abs(f[s["a"]] - fo) < tol, (wk, s["a"], f[s["a"]], fo)


def test_map_back_constant_field(full):
    ctx, pairs, ps, tree = full["ctx"], full["pairs"], full["ps"], full["tree"]
    nc = full["vg"]["volume"].shape[0]
    fc = torch.full((nc,), 0.25, dtype=torch.float64, device="cuda")
    f, fp = api.map_back(ctx, pairs, torch.as_tensor(full["wm"], device="cuda"), fc, ps, tree)
    f, fp = f.cpu().numpy(), fp.cpu().numpy()
    assert np.all(np.isfinite(f)) and np.max(np.abs(f - 0.25)) < 1e-14
    assert fp.shape[0] == full["w"].n and np.max(np.abs(fp - 0.25)) < 1e-14
