"""Edge case at the largest supported division level, n = 14000: N = 10 n^2 + 2 =
1,960,000,002 ray ids, the most that the 32-bit per-ray index arithmetic allows below 2^31.
The ray generator against the oracle's lattice on sampled ids up to the last one, and a
launch over the last two million ray ids against the oracle's brute-force trace of the same
ids: per-ray face sequences, the segment count and the rough paths after double-count
removal.  Runs in a context of its own, closed at the end (the directions take 31 GB)."""
import numpy as np
import pytest
import torch

from paper_2208_10009_gb300 import api, scenes

from parity_util import EDGE_MARGIN, ang

pytestmark = pytest.mark.gpu
SQ3 = float(np.sqrt(3.0))
N_DIV = 14000
TOL = 5e-7   # FP32 slerp + normalisation against the FP64 lattice (the raygen tests' bound)


def _angles(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.sum(a * b, axis=1))


def test_largest_lattice_and_top_ray_range(oracle_mod):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n = N_DIV
    N = 10 * n * n + 2
    assert N < 2 ** 31
    ctx = api.Context(0)
    try:
        # a1 at the largest size: sampled ids including the first and the last ones and the
        # ends of the vertex, edge and face-interior blocks
        d = ctx.raygen(n)
        rng = np.random.default_rng(14000)
        edges_end = 12 + 30 * (n - 1)
        ids = np.unique(np.concatenate([rng.integers(0, N, 20000), np.arange(0, 64), np.arange(N - 2000, N),
                                        np.arange(edges_end - 32, edges_end + 32)]))
        got = d[torch.as_tensor(ids, device=d.device)].cpu().numpy()[:, :3].astype(np.float64)
        assert _angles(got, oracle_mod.lattice_ids(n, ids)).max() < TOL
        del d
        torch.cuda.empty_cache()

        # a2-a5 over the last two million ray ids of the shoebox
        sc, tx, rx = scenes.shoebox_config()
        order, stride = 3, 997
        lo, hi = N - 2_000_000, N
        # the shoebox's receiver and six more half a metre from Tx along ray ids of the range
        # (the range's directions form one patch of the sphere that misses the first one)
        along = oracle_mod.lattice_ids(n, np.linspace(lo, hi - 1, 6).astype(np.int64))
        rx = scenes.f32_exact(np.concatenate([rx, tx[0] + 0.5 * along]))
        scene = ctx.scene_from(sc)
        rxs = ctx.rx_upload(rx)
        paths = ctx.paths_create(1 << 20, 1 << 14)
        per = (N + stride - 1) // stride
        dump = torch.full((1, per, order + 1), -3, dtype=torch.int32, device="cuda")
        ctx.launch(scene, tx, rxs, paths, n, order, rx_angle_scale=SQ3, sync=True, dump_stride=stride, dump=dump,
                   ray_range=(lo, hi))
        st = ctx.launch_stats(paths)
        rough = ctx.query(paths)
        dump = dump.cpu().numpy()[0]

        S = oracle_mod.Scene.from_generated(sc)
        cone = SQ3 * oracle_mod.theta_launch(n)
        ray_ids = np.arange(lo, hi, dtype=np.int64)
        tr = oracle_mod.trace(S, tx[0], oracle_mod.lattice_ids(n, ray_ids), rx, order, cone, ray_ids=ray_ids,
                              want_margin=True)
        assert st["rays"] == hi - lo and st["segments"] == tr.nsegments == 4 * (hi - lo)

        # every dumped ray id of the range (ids that are multiples of the stride); ids
        # outside the range were not traced
        dumped = np.arange((lo + stride - 1) // stride * stride, hi, stride)
        keep = tr.ray_margin[dumped - lo] >= EDGE_MARGIN
        assert keep.sum() > 1900
        mism = np.nonzero(np.any(dump[dumped // stride][keep] != tr.ray_faces[dumped - lo][keep], axis=1))[0]
        assert len(mism) == 0, (len(mism), dumped[keep][mism[:3]])
        assert np.all(dump[: lo // stride - 1] == -3)

        # rough paths: every key the oracle surely receives (error angle clear of the cone's
        # edge by 1e-6) is found, and nothing beyond the keys it may receive; the winners'
        # error angles agree
        ora = oracle_mod.dedup(tr)
        sure = {(p["tx"], p["rx"], p["order"], p["faces"]) for p in ora if p["err"] < cone - 1e-6}
        ora_by_key = {(p["tx"], p["rx"], p["order"], p["faces"]): p for p in ora}
        gpu = {(int(r["tx"]), int(r["rx"]), int(r["order"]), tuple(int(f) for f in r["faces"][: r["order"]])): r
               for r in rough}
        assert len(sure) > 0
        assert sure <= set(gpu) <= set(ora_by_key), (sorted(sure - set(gpu))[:3], sorted(set(gpu) - set(ora_by_key))[:3])
        for k, r in gpu.items():
            assert lo <= int(r["ray"]) < hi
            assert abs(float(r["rough_err"]) - ora_by_key[k]["err"]) < 1e-6
            d_gpu = np.asarray(r["dir"], np.float64)
            assert ang(d_gpu, oracle_mod.lattice_ids(n, [int(r["ray"])])[0]) < TOL
        for h in (paths, rxs, scene):
            h.close()
    finally:
        ctx.close()
        torch.cuda.empty_cache()


def test_largest_lattice_tiled_schedule():
    """A whole n = 14000 launch (1.96e9 rays) in the tiled schedule against lattice id order:
    the same segment count and the same face sequence for every 997th ray id, so the
    schedule's closed form visits every ray once at the largest size too."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    n, order, stride = N_DIV, 2, 997
    N = 10 * n * n + 2
    sc, tx, rx = scenes.shoebox_config()
    ctx = api.Context(0)
    try:
        scene = ctx.scene_from(sc)
        rxs = ctx.rx_upload(rx)
        paths = ctx.paths_create(1 << 20, 1 << 14)
        per = (N + stride - 1) // stride
        out = []
        for id_order in (False, True):
            dump = torch.full((1, per, order + 1), -3, dtype=torch.int32, device="cuda")
            ctx.launch(scene, tx, rxs, paths, n, order, rx_angle_scale=SQ3, sync=True, dump_stride=stride,
                       dump=dump, records_only=True, id_order=id_order)
            out.append((dump.cpu().numpy()[0], ctx.launch_stats(paths)))
        (d1, s1), (d0, s0) = out
        assert s1["rays"] == s0["rays"] == N
        assert s1["segments"] == s0["segments"] and s1["records"] == s0["records"]
        assert np.all(d1[:, 0] >= -1) and np.array_equal(d1, d0)
        for h in (paths, rxs, scene):
            h.close()
    finally:
        ctx.close()
        torch.cuda.empty_cache()
