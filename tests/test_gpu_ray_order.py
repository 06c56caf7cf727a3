"""The trace's schedule (a whole equiangular lattice taken in compact tiles of each face's
triangular grid instead of lattice id order) changes no result: with either order every
ray's face sequence, every reception record and the counters are the same.  Every ray is
traced exactly once (a dump row per ray, the segment count unchanged), at the division
levels where the tiling has no full tile, one block of rows, or blocks in both directions,
with several transmitters and on ray-id ranges (which keep lattice id order)."""
import numpy as np
import pytest
import torch

from paper_2208_10009_gb300 import scenes

pytestmark = pytest.mark.gpu
SQ3 = float(np.sqrt(3.0))


def _sorted_records(recs):
    # tx, rx, ray, order, faces, err, dray as raw 32-bit words (the slot a record was
    # written to depends on the order the warps reached it)
    rows = np.ascontiguousarray(recs).view(np.uint32).reshape(len(recs), 16)[:, :14]
    return rows[np.lexsort(rows.T[::-1])]


def _run(ctx, scene, tx, rxs, paths, n, order, id_order, ray_range=None):
    N = 10 * n * n + 2
    dump = torch.full((len(tx), N, order + 1), -3, dtype=torch.int32, device="cuda")
    ctx.launch(scene, tx, rxs, paths, n, order, rx_angle_scale=SQ3, sync=True, dump_stride=1, dump=dump,
               records_only=True, id_order=id_order, ray_range=ray_range)
    return dump.cpu().numpy(), _sorted_records(ctx.records(paths)), ctx.launch_stats(paths)


def _same(ctx, sc, tx, rx, n, order, ray_range=None):
    scene = ctx.scene_from(sc)
    rxs = ctx.rx_upload(rx)
    paths = ctx.paths_create(1 << 21, 1 << 10)
    d1, r1, s1 = _run(ctx, scene, tx, rxs, paths, n, order, False, ray_range)
    d0, r0, s0 = _run(ctx, scene, tx, rxs, paths, n, order, True, ray_range)
    for h in (paths, rxs, scene):
        h.close()
    for k in ("rays", "segments", "node_visits", "tri_tests", "rx_tests", "records"):
        assert s1[k] == s0[k], k
    bad = np.nonzero(np.any(d1 != d0, axis=-1))
    assert len(bad[0]) == 0, (len(bad[0]), d1[bad][:3], d0[bad][:3])
    assert np.array_equal(r1, r0)
    return s1, d1


def test_schedule_urban_canyon(gpu_ctx):
    sc, tx, rx = scenes.urban_canyon()
    st, dump = _same(gpu_ctx, sc, tx, rx, 300, 6)
    # every ray was traced exactly once: each dump row starts with a face or a miss
    assert st["rays"] == 10 * 300 * 300 + 2 and np.all(dump[..., 0] >= -1)


def test_schedule_ray_range_and_several_tx(gpu_ctx):
    sc, tx, rx = scenes.office(ntx=3, nrx=64)
    N = 10 * 96 * 96 + 2
    st, dump = _same(gpu_ctx, sc, tx, rx, 96, 4, ray_range=(12345, N - 777))
    assert st["rays"] == 3 * (N - 777 - 12345)
    assert np.all(dump[:, 12345:N - 777, 0] >= -1)
    assert np.all(dump[:, :12345] == -3) and np.all(dump[:, N - 777:] == -3)


def test_schedule_several_tx(gpu_ctx):
    sc, tx, rx = scenes.office(ntx=3, nrx=64)
    st, dump = _same(gpu_ctx, sc, tx, rx, 96, 4)
    assert st["rays"] == 3 * (10 * 96 * 96 + 2) and np.all(dump[..., 0] >= -1)


@pytest.mark.parametrize("n", [1, 2, 3, 5, 9, 12, 13, 17, 64])
def test_schedule_small_lattices(gpu_ctx, n):
    sc, tx, rx = scenes.shoebox_config()
    st, dump = _same(gpu_ctx, sc, tx, rx, n, 3)
    assert st["rays"] == 10 * n * n + 2 and np.all(dump[..., 0] >= -1)
