"""a2-a8 parity on seeded random scenes whose faces lie on no coordinate plane: a room with
twenty arbitrarily rotated, interpenetrating boxes.  Every ray's face sequence and every
reception record against the oracle's brute-force trace, every refinement decision against
the oracle's replay, and every refined path's validity and outputs against the oracle and
the image method."""
import numpy as np
import pytest
import torch

from paper_2208_10009_gb300 import scenes

from parity_util import EDGE_MARGIN, ang, dir_of, in_key_order, replay_refinement

pytestmark = pytest.mark.gpu
SQ3 = float(np.sqrt(3.0))
ACC = np.radians(0.01)


def _records_by_key(rx, ray, order, faces, err, dray):
    out = {}
    for i in range(len(err)):
        k = int(order[i])
        out[(int(ray[i]), int(rx[i]), k, tuple(int(f) for f in faces[i, :k]))] = (float(err[i]), float(dray[i]))
    return out


@pytest.mark.parametrize("seed", [1, 2, 3])
def test_random_clutter_every_ray_and_path(gpu_ctx, oracle_mod, seed):
    sc, tx, rx = scenes.random_clutter(scenes.SEED_BASE + 9 + seed)
    n, order, K, cap = 32, 3, 9, 8
    N = 10 * n * n + 2
    cone = SQ3 * oracle_mod.theta_launch(n)
    scene = gpu_ctx.scene_from(sc)
    rxs = gpu_ctx.rx_upload(rx)
    paths = gpu_ctx.paths_create(1 << 18, 1 << 14)
    dump = torch.full((1, N, order + 1), -3, dtype=torch.int32, device="cuda")
    gpu_ctx.launch(scene, tx, rxs, paths, n, order, rx_angle_scale=SQ3, sync=True, dump_stride=1, dump=dump)
    S = oracle_mod.Scene.from_generated(sc)
    tr = oracle_mod.trace(S, tx[0], oracle_mod.lattice(n), rx, order, cone, want_margin=True)

    # every ray's face sequence (rays within 1e-6 rad of an edge or grazing excluded)
    keep = tr.ray_margin >= EDGE_MARGIN
    d = dump.cpu().numpy()[0]
    mism = np.nonzero(np.any(d[keep] != tr.ray_faces[keep], axis=1))[0]
    assert keep.sum() > 0.97 * N
    assert len(mism) == 0, (len(mism), d[keep][mism[:3]], tr.ray_faces[keep][mism[:3]])
    assert gpu_ctx.launch_stats(paths)["segments"] == tr.nsegments

    # every reception record of the kept rays (records within rounding of the cone's edge
    # may fall on either side of it)
    ok = set(np.nonzero(keep)[0].tolist())
    ora = _records_by_key(tr.rec_rx, tr.rec_ray, tr.rec_order, tr.rec_faces, tr.rec_err, tr.rec_dray)
    g = gpu_ctx.records(paths)
    gpu = _records_by_key(g["rx"], g["ray"], g["order"], g["faces"], g["err"], g["dray"])
    edge = lambda e: abs(e - cone) <= 1e-6
    o_keys = {k for k, v in ora.items() if k[0] in ok and not edge(v[0])}
    g_keys = {k for k, v in gpu.items() if k[0] in ok and not edge(v[0])}
    assert len(o_keys) > 100
    assert o_keys == g_keys, (sorted(o_keys - g_keys)[:4], sorted(g_keys - o_keys)[:4])
    for k in o_keys:
        assert abs(gpu[k][0] - ora[k][0]) <= 1e-6 and abs(gpu[k][1] / ora[k][1] - 1.0) <= 1e-6, k

    # refined paths: validity on the GPU's own direction equals the oracle's; valid paths
    # with an exact image-method counterpart agree with it (AOD within 0.01 deg, delay within
    # 1e-6; AOA within 0.01 deg where the early stop ended the refinement)
    choice = torch.full((paths.path_cap, cap), -1, dtype=torch.int8, device="cuda")
    gpu_ctx.batch_refine(scene, paths, cap, K, target=ACC, choice_log=choice)
    got, ch = in_key_order(gpu_ctx.query(paths), choice.cpu().numpy())
    assert len(got) > 20
    n_valid = n_im = 0
    tl = np.float32(oracle_mod.theta_launch(n))
    for i, r in enumerate(got):
        faces = tuple(int(f) for f in r["faces"][: r["order"]])
        # every decision of the refinement (argmin, frame axis, stop) against the oracle's
        # FP64 replay of the same decisions
        c0 = oracle_mod.lattice_ids(n, [int(r["ray"])])[0]
        replay_refinement(oracle_mod, S, tx[0], rx[r["rx"]], faces, c0, max(float(tl), float(r["rough_err"])), K, r,
                          ch[i], cap, ACC)
        R0 = max(oracle_mod.theta_launch(n), float(r["rough_err"]))
        bound = oracle_mod.refined_err_bound(R0, K, int(r["iters"])) if r["iters"] > 0 else 0.0
        ev = oracle_mod.path_eval(S, tx[0], rx[r["rx"]], faces, r["dir"], err_bound=bound)
        im = oracle_mod.image_path(S, tx[0], rx[r["rx"]], faces)
        assert bool(r["valid"]) == ev["valid"], (faces, r["valid"], ev)
        if not r["valid"]:
            continue
        n_valid += 1
        if not im["valid"]:
            continue
        n_im += 1
        assert ang(r["dir"], im["aod_dir"]) <= ACC * (1 + 1e-6), faces
        assert abs(r["delay"] / im["delay"] - 1) < 1e-6, faces
        if int(r["iters"]) < cap:
            assert ang(dir_of(*r["aoa"]), dir_of(*im["aoa"])) <= ACC * (1 + 1e-3) + 1e-6, faces
    assert n_valid > 10 and n_im >= 0.9 * n_valid
    for h in (paths, rxs, scene):
        h.close()
