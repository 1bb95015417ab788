"""The spatial split of the mapping over ranks (paper_2410_15227_gb300.partition)
on the CPU: two gloo processes stand in for two GPUs.  Each rank takes the
cells of its Morton range and the particles that reach the bounding boxes of
their groups,
finds and maps its pairs through the oracle, and the inverse mapping's sums
are added with the all-reduce.  Against the single-rank result: the ranks'
pair lists together are the single-rank list with each pair once, every
weight is the same, and the reduced f equals the single-rank f up to the
order of the additions."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2410_15227_gb300 import inputs, partition

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _workload(kind="sphere"):
    # a sphere profile (uneven cell sizes and kernel radii, hull cells out to
    # the box walls), or a uniform cube (compact cells)
    if kind == "cube":
        return inputs.uniform_cube(8000, 2000, seed=12, gen_seed=13)
    return inputs.sphere_workload(1500, 300, seed=12)


def _field(ngen):
    return np.random.default_rng(77).random(ngen)


def _worker(rank, world, port, kind, out):
    sys.path.insert(0, ROOT)
    import oracle as orc
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        w = _workload(kind)
        mine = partition.cell_ranges(w.gx, w.gy, w.gz, w.box, world)[rank]
        cells = orc.voronoi(w.gx, w.gy, w.gz, w.box, cells=mine, nthreads=2)
        lo, hi = partition.cell_boxes(cells.cell_face_off, cells.face_vert_off, cells.verts)
        order = np.argsort(partition.morton_keys(w.gx[mine], w.gy[mine], w.gz[mine], w.box), kind="stable")
        sel = partition.reaching(w.x, w.y, w.z, w.h, *partition.group_boxes(lo, hi, order, 64))
        pairs = orc.find_pairs(w.x[sel], w.y[sel], w.z[sel], w.h[sel], cells, nthreads=2)
        wts = orc.map_exact(pairs, w.x[sel], w.y[sel], w.z[sel], w.h[sel], cells, nthreads=2)
        gi, gj = sel[pairs.pair_i], mine[pairs.pair_j]
        glob = orc.Pairs(gi, gj, pairs.near, np.zeros(1, np.int64))
        num, den = orc.map_back_sums(glob, wts, _field(w.ngen), w.n)
        num, den = torch.from_numpy(num), torch.from_numpy(den)
        partition.reduce_sums(num, den)
        out[rank] = (gi, gj, wts, num.numpy(), den.numpy(), len(sel))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("kind", ["sphere", "cube"])
def test_two_ranks_equal_the_single_rank_result(orc, kind):
    world = 2
    w = _workload(kind)
    with mp.get_context("spawn").Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(world, _free_port(), kind, out), nprocs=world, join=True)
        res = dict(out)
    cells = orc.voronoi(w.gx, w.gy, w.gz, w.box)
    pairs = orc.find_pairs(w.x, w.y, w.z, w.h, cells)
    wts = orc.map_exact(pairs, w.x, w.y, w.z, w.h, cells)
    f = orc.map_back(pairs, wts, _field(w.ngen), w.n)
    # each pair on exactly one rank, the union the single-rank list
    gi = np.concatenate([res[r][0] for r in range(world)])
    gj = np.concatenate([res[r][1] for r in range(world)])
    wr = np.concatenate([res[r][2] for r in range(world)])
    order = np.lexsort((gi, gj))
    assert np.array_equal(gj[order], pairs.pair_j) and np.array_equal(gi[order], pairs.pair_i)
    # a cell's geometry does not depend on which rank built it
    assert np.array_equal(wr[order], wts)
    # compact cells split the particles too: each rank took a proper subset,
    # the halo (2h of 0.12 beside cells of 0.08 in the unit cube) aside
    if kind == "cube":
        assert all(0 < res[r][5] < w.n for r in range(world))
        assert sum(res[r][5] for r in range(world)) < 1.6 * w.n
    # the reduced sums, identical on both ranks, give the single-rank f
    num, den = res[0][3], res[0][4]
    assert np.array_equal(num, res[1][3]) and np.array_equal(den, res[1][4])
    with np.errstate(invalid="ignore", divide="ignore"):
        fr = num / den
    ok = den > 0
    assert np.array_equal(ok, np.isfinite(f))
    assert np.max(np.abs(fr[ok] - f[ok]) / np.abs(f[ok])) < 1e-13


def test_morton_keys_interleave_bits():
    rng = np.random.default_rng(3)
    box = np.array([-1.0, 2.0, 0.0, 1.0, 5.0, 9.0])
    p = rng.random((50, 3)) * [3.0, 1.0, 4.0] + [-1.0, 0.0, 5.0]
    k = partition.morton_keys(p[:, 0], p[:, 1], p[:, 2], box)
    for i in range(p.shape[0]):
        q = [min(int(np.floor((p[i, a] - box[2 * a]) * (2 ** 21 / (box[2 * a + 1] - box[2 * a])))), 2 ** 21 - 1)
             for a in range(3)]
        ref = 0
        for b in range(21):
            for a in range(3):
                ref |= ((q[a] >> b) & 1) << (3 * b + 2 - a)
        assert int(k[i]) == ref


def test_cell_ranges_cover_the_generators_once():
    w = _workload()
    for world in (1, 2, 3, 7):
        parts = partition.cell_ranges(w.gx, w.gy, w.gz, w.box, world)
        assert len(parts) == world
        allp = np.concatenate(parts)
        assert np.array_equal(np.sort(allp), np.arange(w.ngen))
        sizes = [len(p) for p in parts]
        assert max(sizes) - min(sizes) <= 1
        # contiguous in Morton order: every key of range r is at most every key of range r + 1
        keys = partition.morton_keys(w.gx, w.gy, w.gz, w.box)
        for a, b in zip(parts[:-1], parts[1:]):
            assert keys[a].max() <= keys[b].min()
    with pytest.raises(ValueError):
        partition.cell_ranges(w.gx, w.gy, w.gz, w.box, 0)


def test_cell_and_group_boxes(orc):
    cells = orc.cells_from_faces([orc.box_cell([0, 0, 0], [1, 2, 3]), orc.box_cell([-1, 0.5, 0], [0, 1, 1]),
                                  orc.box_cell([4, 4, 4], [5, 6, 7])])
    lo, hi = partition.cell_boxes(cells.cell_face_off, cells.face_vert_off, cells.verts)
    assert np.array_equal(lo, [[0, 0, 0], [-1, 0.5, 0], [4, 4, 4]])
    assert np.array_equal(hi, [[1, 2, 3], [0, 1, 1], [5, 6, 7]])
    glo, ghi = partition.group_boxes(lo, hi, np.array([1, 0, 2]), 2)
    assert np.array_equal(glo, [[-1, 0, 0], [4, 4, 4]]) and np.array_equal(ghi, [[1, 2, 3], [5, 6, 7]])


def test_reaching_is_the_ball_box_test():
    lo, hi = np.array([0.0, 0.0, 0.0]), np.array([1.0, 1.0, 1.0])
    x = np.array([0.5, 1.5, 1.5, -0.2, 3.0])
    y = np.array([0.5, 0.5, 1.5, 0.5, 0.5])
    z = np.array([0.5, 0.5, 1.5, 0.5, 0.5])
    h = np.array([0.01, 0.25, 0.4, 0.05, 0.9])
    # inside; 0.5 from the face with 2h = 0.5; sqrt(0.75) = 0.866 from the corner with 2h = 0.8;
    # 0.2 from the face with 2h = 0.1; 2 from the face with 2h = 1.8
    assert list(partition.reaching(x, y, z, h, lo, hi)) == [0, 1]
    # several boxes: the union
    lo2, hi2 = np.array([lo, [2.9, 0.0, 0.0]]), np.array([hi, [3.1, 1.0, 1.0]])
    assert list(partition.reaching(x, y, z, h, lo2, hi2)) == [0, 1, 4]


def test_morton_order_and_contiguous_ranges():
    w = _workload()
    order = partition.morton_order(w.gx, w.gy, w.gz, w.box)
    keys = partition.morton_keys(w.gx, w.gy, w.gz, w.box)
    assert np.all(np.diff(keys[order].astype(np.float64)) >= 0)
    for world in (1, 2, 5):
        rng = partition.contiguous_ranges(w.ngen, world)
        parts = partition.cell_ranges(w.gx, w.gy, w.gz, w.box, world)
        assert rng[0][0] == 0 and rng[-1][1] == w.ngen
        # rank r's Morton range, in the sorted order, is the generators cell_ranges gives it
        for (a, b), p in zip(rng, parts):
            assert np.array_equal(np.sort(order[a:b]), p)
