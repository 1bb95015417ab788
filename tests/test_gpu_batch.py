"""GPU tests of map_batch, the executor for many independent snapshots: the
same results, bit for bit, as the entry points called one snapshot at a
time (the kernels sum in fixed orders, so the stream a snapshot runs on
cannot change them); the smallest snapshot against the oracle; a failing
snapshot reported on its own while the others finish."""
import numpy as np
import pytest
import torch

from paper_2410_15227_gb300 import api, inputs

pytestmark = pytest.mark.gpu

SRC = np.zeros((1, 3))


def dev(a, dt=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device="cuda")


def snapshots(count=12, lo=3.0, hi=4.3):
    out = []
    for s in range(count):
        rng = np.random.default_rng(200 + s)
        ns = int(round(10 ** rng.uniform(lo, hi)))
        w = inputs.sphere_workload(ns, max(ns // 4, 8), 1.0, seed=200 + s, field_seed=200 + s)
        fc = np.random.default_rng(300 + s).random(w.ngen)
        out.append((w, fc))
    return out


SNAPS = snapshots()


def as_dicts(snaps, with_f=True):
    return [dict(x=dev(w.x), y=dev(w.y), z=dev(w.z), m=dev(w.m), h=dev(w.h), gx=dev(w.gx), gy=dev(w.gy),
                 gz=dev(w.gz), box=w.box, sources=SRC, f_cell=dev(fc) if with_f else None) for w, fc in snaps]


def serial(ctx, w, fc, P):
    t = api.build_tree(ctx, dev(w.x), dev(w.y), dev(w.z), dev(w.m), w.box, P.leaf_max)
    ps = api.make_pseudo_particles(ctx, t, dev(w.h), SRC, P)
    g = ps.get()
    vor = api.build_voronoi(ctx, dev(w.gx), dev(w.gy), dev(w.gz), w.box, P)
    pr = api.find_pairs(ctx, g["x"], g["y"], g["z"], g["h"], vor)
    wts, rho, _, nf = api.map_exact(ctx, pr, g["x"], g["y"], g["z"], g["h"], g["m"], vor, P)
    _, f = api.map_back(ctx, pr, wts, dev(fc), ps, t)
    return rho, f, ps.info()[0], pr.info()[0], nf


@pytest.mark.parametrize("precision", [0, 1])
def test_batch_equals_serial(precision):
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, precision=precision)
    res, launches = api.map_batch(0, as_dicts(SNAPS), P, nworkers=4)
    ctx = api.Context(0)
    assert launches > 10 * len(SNAPS)
    for (w, fc), r in zip(SNAPS, res):
        rho, f, npseudo, npairs, nf = serial(ctx, w, fc, P)
        assert r["status"] == 0
        assert (r["npseudo"], r["npairs"], r["nfp64"]) == (npseudo, npairs, nf)
        assert torch.equal(r["rho"], rho)
        assert torch.equal(torch.nan_to_num(r["f"], nan=-1.0), torch.nan_to_num(f, nan=-1.0))
    # one worker gives the same
    res1, _ = api.map_batch(0, as_dicts(SNAPS[:4], with_f=False), P, nworkers=1)
    for a, b in zip(res1, res[:4]):
        assert torch.equal(a["rho"], b["rho"]) and a["f"] is None


def test_batch_smallest_against_oracle(orc):
    w, fc = min(SNAPS, key=lambda s: s[0].n)
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, precision=0, h_tol=1e-13)
    (r,), _ = api.map_batch(0, as_dicts([(w, fc)]), P, nworkers=2)
    ps, _, _ = orc.make_pseudo_particles(w.x, w.y, w.z, w.m, w.h, w.box, SRC, 0.05, 0.1, 0.3)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs = orc.find_pairs(ps.x, ps.y, ps.z, ps.h, cells)
    wo = orc.map_exact(pairs, ps.x, ps.y, ps.z, ps.h, cells)
    rho_o = orc.cell_density(pairs, wo, ps.m, cells.volume)
    rho = r["rho"].cpu().numpy()
    assert r["npairs"] == pairs.n
    assert np.all(np.abs(rho - rho_o) <= 1e-10 * np.abs(rho_o) + 1e-12 * np.abs(rho_o).max())


def test_batch_failing_snapshot():
    snaps = as_dicts(SNAPS[:5])
    bad = dict(snaps[2])
    gx = bad["gx"].clone()
    gx[0] = float(SNAPS[2][0].box[1]) + 1.0      # a site outside the box
    bad["gx"] = gx
    snaps[2] = bad
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3)
    with pytest.raises(Exception) as ei:
        api.map_batch(0, snaps, P, nworkers=3)
    res = ei.value.results
    assert res[2]["status"] == 1                     # EM_EINVAL, from build_voronoi
    assert "snapshot 2" in str(ei.value)
    good, _ = api.map_batch(0, as_dicts(SNAPS[:5]), P, nworkers=3)
    for k in (0, 1, 3, 4):
        assert res[k]["status"] == 0 and torch.equal(res[k]["rho"], good[k]["rho"])


def test_batch_tuned_equals_serial_with_its_variant():
    """The batch with its launch shape picked by map_autotune on the batch's
    pairs equals the snapshots mapped one at a time with that shape, bit for
    bit; the mapping's device time is reported."""
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, precision=1)
    info = {}
    res_t, _ = api.map_batch(0, as_dicts(SNAPS[:6]), P, nworkers=3, tune=True, info=info)
    assert 0 <= info["variant"] < api.FP32_VARIANTS and info["map_ms"][0] > 0
    Pv = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, precision=1, fp32_variant=info["variant"])
    ctx = api.Context(0)
    for (w, fc), r in zip(SNAPS[:6], res_t):
        rho, f, npseudo, npairs, nf = serial(ctx, w, fc, Pv)
        assert r["status"] == 0 and (r["npairs"], r["nfp64"]) == (npairs, nf)
        assert torch.equal(r["rho"], rho)
        assert torch.equal(torch.nan_to_num(r["f"], nan=-1.0), torch.nan_to_num(f, nan=-1.0))


@pytest.mark.parametrize("variant", range(api.FP32_VARIANTS))
def test_every_launch_shape_independent_of_warp_neighbours(variant):
    """In every launch shape of the FP32 pass, a pair's weight does not depend
    on which pairs share its warp: the batch, where each snapshot's pairs sit
    at other offsets of the concatenated list, equals the snapshots mapped
    one at a time with that shape, bit for bit."""
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, precision=1, fp32_variant=variant)
    res, _ = api.map_batch(0, as_dicts(SNAPS[:6], with_f=False), P, nworkers=2)
    ctx = api.Context(0)
    for (w, fc), r in zip(SNAPS[:6], res):
        rho, _, _, npairs, nf = serial(ctx, w, fc, P)
        assert r["status"] == 0 and (r["npairs"], r["nfp64"]) == (npairs, nf)
        assert torch.equal(r["rho"], rho)


def test_autotune_variants():
    """Every launch shape of the FP32 pass is deterministic (the same bits on
    a second call) and within the mixed mode's tolerance of the default shape
    (the shapes are compiled separately, and the compiler may fuse a multiply
    and an add differently in each); map_autotune times them all and returns
    one of them."""
    w, _ = max(SNAPS, key=lambda s: s[0].n)
    ctx = api.Context(0)
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, precision=1)
    t = api.build_tree(ctx, dev(w.x), dev(w.y), dev(w.z), dev(w.m), w.box, 8)
    g = api.make_pseudo_particles(ctx, t, dev(w.h), SRC, P).get()
    vor = api.build_voronoi(ctx, dev(w.gx), dev(w.gy), dev(w.gz), w.box, P)
    pr = api.find_pairs(ctx, g["x"], g["y"], g["z"], g["h"], vor)
    best, ms = api.map_autotune(ctx, pr, g["x"], g["y"], g["z"], g["h"], vor, P)
    assert 0 <= best < api.FP32_VARIANTS and len(ms) == api.FP32_VARIANTS and min(ms) > 0
    w64, _, _, _ = api.map_exact(ctx, pr, g["x"], g["y"], g["z"], g["h"], g["m"], vor, api.Params(precision=0))
    for v in range(api.FP32_VARIANTS):
        Pv = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, precision=1, fp32_variant=v)
        a, _, _, _ = api.map_exact(ctx, pr, g["x"], g["y"], g["z"], g["h"], g["m"], vor, Pv)
        b, _, _, _ = api.map_exact(ctx, pr, g["x"], g["y"], g["z"], g["h"], g["m"], vor, Pv)
        assert torch.equal(a, b), v
        assert bool(((a - w64).abs() <= 1e-5 * w64.abs() + 1e-14).all()), v
    with pytest.raises(Exception):
        api.map_exact(ctx, pr, g["x"], g["y"], g["z"], g["h"], g["m"], vor,
                      api.Params(precision=1, fp32_variant=api.FP32_VARIANTS))


def test_batch_handle_equals_map_batch():
    """The handle form (create, add, run, get) maps what map_batch maps, bit
    for bit; a second run after more adds maps the enlarged batch; a bad
    index is rejected."""
    P = api.Params(r_part=0.05, r_leaf=0.1, theta=0.3, precision=1)
    snaps = as_dicts(SNAPS[:6])
    ref, _ = api.map_batch(0, snaps, P, nworkers=3)
    b = api.Batch(0, P, nworkers=3)
    assert [b.add(s) for s in snaps[:4]] == [0, 1, 2, 3]
    assert b.get(2)["status"] == -1   # not run yet
    res, launches = b.run()
    assert len(res) == 4 and launches > 0
    for r, q in zip(res, ref[:4]):
        assert r["status"] == 0
        assert (r["npseudo"], r["npairs"], r["nfp64"]) == (q["npseudo"], q["npairs"], q["nfp64"])
        assert torch.equal(r["rho"], q["rho"])
        assert torch.equal(torch.nan_to_num(r["f"], nan=-1.0), torch.nan_to_num(q["f"], nan=-1.0))
    assert b.add(snaps[4]) == 4 and b.add(snaps[5]) == 5
    res, _ = b.run()
    for r, q in zip(res, ref):
        assert torch.equal(r["rho"], q["rho"])
    with pytest.raises(Exception):
        b.get(6)
