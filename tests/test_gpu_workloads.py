"""Parity at the workloads' full sizes, in the launch configuration bench.py uses, on
outputs the oracle can compute one by one: sampled rays' face sequences, every refined
path against the image method, sampled refinements against the oracle, the batched
office workload, the unfolding gradients at 1M paths, and the large city."""
import numpy as np
import pytest
import torch

from paper_2208_10009_gb300 import api, scenes

from parity_util import (EDGE_MARGIN, PATH_STALLED, PATH_TRACE_FAIL, TOL_ANGLE_RAD, TOL_DELAY_REL, ang, dir_of,
                         in_key_order, replay_refinement)


def _bound(oracle_mod, n, K, r):
    R0 = max(oracle_mod.theta_launch(n), float(r["rough_err"]))
    return oracle_mod.refined_err_bound(R0, K, int(r["iters"])) if r["iters"] > 0 else 0.0

pytestmark = pytest.mark.gpu
SQ3 = float(np.sqrt(3.0))
ACC = np.radians(0.01)


@pytest.fixture(scope="module")
def canyon(gpu_ctx):
    sc, tx, rx = scenes.urban_canyon()
    scene = gpu_ctx.scene_from(sc)
    rxs = gpu_ctx.rx_upload(rx)
    paths = gpu_ctx.paths_create(1 << 18, 1 << 15)
    yield sc, tx, rx, scene, rxs, paths
    for h in (paths, rxs, scene):
        h.close()


def test_canyon_sampled_rays(gpu_ctx, oracle_mod, canyon):
    """Every 997th ray of the 4.9M-ray launch (n = 700, order 6): face sequence per segment
    equals the oracle's brute-force trace, rays within 1e-6 rad of an edge or grazing
    excluded and counted."""
    sc, tx, rx, scene, rxs, paths = canyon
    n, order, stride = 700, 6, 997
    N = 10 * n * n + 2
    per = (N + stride - 1) // stride
    dump = torch.full((1, per, order + 1), -3, dtype=torch.int32, device="cuda")
    gpu_ctx.launch(scene, tx, rxs, paths, n, order, rx_angle_scale=SQ3, sync=True, dump_stride=stride, dump=dump)
    d = dump.cpu().numpy()[0]
    ids = np.arange(0, N, stride)
    S = oracle_mod.Scene.from_generated(sc)
    tr = oracle_mod.trace(S, tx[0], oracle_mod.lattice_ids(n, ids), rx, order, SQ3 * oracle_mod.theta_launch(n),
                          ray_ids=ids, want_margin=True)
    keep = tr.ray_margin >= EDGE_MARGIN
    mism = np.nonzero(np.any(d[keep] != tr.ray_faces[keep], axis=1))[0]
    assert keep.sum() > 0.98 * len(ids)
    assert len(mism) == 0, (len(mism), d[keep][mism[:3]], tr.ray_faces[keep][mism[:3]])
    # segments traced for the sampled rays agree
    assert int((d[keep] != -2).sum()) == int(tr.ray_nseg[keep].sum())


def test_canyon_paths_vs_image_method_and_oracle(gpu_ctx, oracle_mod, canyon):
    """All refined paths of the bench workload (6 iterations, K = 9, batched kernel): every
    valid one is a valid image-method path with AOD within 0.01 deg and delay within 1e-6;
    a sample of paths refined by the oracle from the same rough ray agrees to 1e-4 deg."""
    sc, tx, rx, scene, rxs, paths = canyon
    n, order, iters, K = 700, 6, 6, 9
    gpu_ctx.launch(scene, tx, rxs, paths, n, order, rx_angle_scale=SQ3, sync=True)
    choice = torch.full((paths.path_cap, iters), -1, dtype=torch.int8, device="cuda")
    gpu_ctx.batch_refine(scene, paths, iters, K, choice_log=choice)
    got, ch = in_key_order(gpu_ctx.query(paths), choice.cpu().numpy())
    assert len(got) > 300
    S = oracle_mod.Scene.from_generated(sc)
    valid = got[got["valid"] == 1]
    assert len(valid) > 0.7 * len(got)
    marginal = 0
    for r in got:
        faces = tuple(int(f) for f in r["faces"][: r["order"]])
        # the validity test itself: same refined direction, oracle in FP64
        ev = oracle_mod.path_eval(S, tx[r["tx"]], rx[r["rx"]], faces, r["dir"], err_bound=_bound(oracle_mod, n, K, r))
        assert bool(r["valid"]) == ev["valid"], faces
        if not r["valid"]:
            continue
        im = oracle_mod.image_path(S, tx[r["tx"]], rx[r["rx"]], faces)
        # the refined bounce points lie within (AOD error x path length) of the exact ones,
        # so a path whose exact point sits on a face edge may be judged differently
        if not im["valid"]:
            marginal += 1
            continue
        assert ang(r["dir"], im["aod_dir"]) < ACC
        assert abs(r["delay"] / im["delay"] - 1) < TOL_DELAY_REL
    assert marginal <= 0.02 * len(valid)
    # every path: the oracle replays the GPU's logged decisions, each is the oracle's own on
    # the same cone or a tie within the GPU's rounding, and the GPU's result is the
    # replay's; where the decisions equal the oracle's own run, so do the directions
    tl = np.float32(oracle_mod.theta_launch(n))
    ties = 0
    for i, r in enumerate(got):
        faces = tuple(int(f) for f in r["faces"][: r["order"]])
        c0 = oracle_mod.lattice_ids(n, [int(r["ray"])])[0]
        R0 = max(float(tl), float(r["rough_err"]))
        rep = replay_refinement(oracle_mod, S, tx[r["tx"]], rx[r["rx"]], faces, c0, R0, K, r, ch[i], iters)
        ties += rep["ties"] + rep["axis_ties"] > 0
        ref = oracle_mod.refine(S, tx[r["tx"]], rx[r["rx"]], faces, c0, R0, K, iters)
        if np.array_equal(ch[i, : ref["iters"]] & 15, ref["choice"]):
            assert ang(r["dir"], ref["dir"]) < TOL_ANGLE_RAD
    assert ties <= 0.05 * len(got)
    # outputs of the GPU's own refined direction on a sample
    rng = np.random.default_rng(0)
    for i in rng.choice(len(got), size=min(120, len(got)), replace=False):
        r = got[i]
        faces = tuple(int(f) for f in r["faces"][: r["order"]])
        # outputs of the same refined direction (AOA amplifies any launch difference by
        # path length / last-leg length, so it is compared on the GPU's own direction)
        ev = oracle_mod.path_eval(S, tx[r["tx"]], rx[r["rx"]], faces, r["dir"], err_bound=_bound(oracle_mod, n, K, r))
        assert bool(r["valid"]) == ev["valid"]
        assert abs(r["delay"] / ev["delay"] - 1) < TOL_DELAY_REL
        assert ang(dir_of(*r["aod"]), dir_of(*ev["aod"])) < TOL_ANGLE_RAD
        assert ang(dir_of(*r["aoa"]), dir_of(*ev["aoa"])) < TOL_ANGLE_RAD
        assert abs(r["power_dbm"] - ev["power"]) < 1e-3


def test_office_batched(gpu_ctx, oracle_mod):
    """Office workload (~55k triangles, 16 Tx x 1024 Rx, n = 128, orders 0-6): batched
    refinement with K = 16, early stop at 0.01 deg, cap 8; sampled paths agree with the
    oracle's refinement and with the image method."""
    sc, tx, rx = scenes.office()
    scene = gpu_ctx.scene_from(sc)
    rxs = gpu_ctx.rx_upload(rx)
    paths = gpu_ctx.paths_create(1 << 24, 1 << 23)
    n, order, K, cap = 128, 6, 16, 8
    gpu_ctx.launch(scene, tx, rxs, paths, n, order, rx_angle_scale=SQ3, sync=True)
    choice = torch.full((paths.path_cap, cap), -1, dtype=torch.int8, device="cuda")
    gpu_ctx.batch_refine(scene, paths, cap, K, target=ACC, choice_log=choice)
    got, ch = in_key_order(gpu_ctx.query(paths), choice.cpu().numpy())
    assert len(got) > 10000
    assert np.all(got["iters"] <= cap)
    its = np.bincount(got["iters"], minlength=cap + 1)
    assert its[1:].sum() > 0 and np.count_nonzero(its) >= 3     # uneven iteration counts
    tl = np.float32(oracle_mod.theta_launch(n))
    # every path: a path flagged as stalled has its error above the stall bound of its last
    # cone (R0 s^iters (1 / (1 - s) + 2 s) + 1e-6, the test that stopped it), and a path that
    # stopped before the cap without stalling met the target (AOD error within 0.01 deg)
    s = api.subray_pattern(K)[2]
    R = np.maximum(tl, got["rough_err"]).astype(np.float64) * s ** got["iters"].astype(np.float64)
    bound = R * (1.0 / (1.0 - s) + 2.0 * s) + 1e-6
    ok = (got["flags"] & PATH_TRACE_FAIL) == 0
    st = ok & ((got["flags"] & PATH_STALLED) != 0)
    assert np.all(got["err"][st] > bound[st] * (1 - 1e-5)), np.nonzero(got["err"][st] <= bound[st] * (1 - 1e-5))
    early = ok & ~st & (got["iters"] < cap) & (got["iters"] > 0)
    assert np.all(got["err"][early] <= ACC * (1 + 1e-4))
    S = oracle_mod.Scene.from_generated(sc)
    rng = np.random.default_rng(1)
    marginal = ties = early = 0
    for i in rng.choice(len(got), size=400, replace=False):
        r = got[i]
        faces = tuple(int(f) for f in r["faces"][: r["order"]])
        c0 = oracle_mod.lattice_ids(n, [int(r["ray"])])[0]
        R0 = max(float(tl), float(r["rough_err"]))
        # every decision (argmin, frame axis, early stop at 0.01 deg) against the oracle's
        # replay; where the decisions equal the oracle's own run, so do the directions
        rep = replay_refinement(oracle_mod, S, tx[r["tx"]], rx[r["rx"]], faces, c0, R0, K, r, ch[i], cap, ACC)
        ties += rep["ties"] + rep["axis_ties"] > 0
        ref = oracle_mod.refine(S, tx[r["tx"]], rx[r["rx"]], faces, c0, R0, K, cap, ACC)
        if ref["iters"] == r["iters"] and np.array_equal(ch[i, : ref["iters"]] & 15, ref["choice"]):
            assert ang(r["dir"], ref["dir"]) < TOL_ANGLE_RAD
        ev = oracle_mod.path_eval(S, tx[r["tx"]], rx[r["rx"]], faces, r["dir"], err_bound=_bound(oracle_mod, n, K, r))
        assert bool(r["valid"]) == ev["valid"]
        if r["valid"]:
            im = oracle_mod.image_path(S, tx[r["tx"]], rx[r["rx"]], faces)
            if im["valid"]:
                assert ang(r["dir"], im["aod_dir"]) <= ACC * (1 + 1e-6)
                if int(r["iters"]) < cap:
                    assert ang(dir_of(*r["aoa"]), dir_of(*im["aoa"])) <= ACC * (1 + 1e-3) + 1e-6
                    early += 1
            else:
                # stopped at 0.01 deg: bounce points up to ~1e-4 x path length from the
                # exact ones, enough to cross the edge of a small furniture face
                marginal += 1
    assert marginal <= 4 and ties <= 20 and early >= 60
    for h in (paths, rxs, scene):
        h.close()


def test_unfold_gradients_1m(gpu_ctx, oracle_mod, canyon):
    """1M fixed face-sequence paths (orders 1-6 from the canyon's refined paths, Tx/Rx
    jittered by +-1 m): forward values and vector-Jacobian products of the adjoint kernel
    vs the oracle's closed form and FP64 central differences, relative error < 1e-3."""
    from paper_2208_10009_gb300.autograd import unfold
    sc, tx, rx, scene, rxs, paths = canyon
    gpu_ctx.launch(scene, tx, rxs, paths, 700, 6, rx_angle_scale=SQ3, sync=True)
    gpu_ctx.batch_refine(scene, paths, 6, 9)
    got = gpu_ctx.query(paths)
    base = got[(got["valid"] == 1) & (got["order"] >= 1)]
    assert len(base) > 100
    P = 1 << 20
    rng = np.random.default_rng(4)
    pick = rng.integers(0, len(base), P)
    b = base[pick]
    T = scenes.jitter(rng, tx[b["tx"]], 1.0)
    R = scenes.jitter(rng, rx[b["rx"]], 1.0)
    d = b["dir"]
    AE = np.stack([np.arctan2(d[:, 1], d[:, 0]), np.arctan2(d[:, 2], np.hypot(d[:, 0], d[:, 1]))], -1)
    dev = "cuda"
    t_tx = torch.tensor(T, dtype=torch.float32, device=dev, requires_grad=True)
    t_rx = torch.tensor(R, dtype=torch.float32, device=dev, requires_grad=True)
    t_ae = torch.tensor(AE, dtype=torch.float32, device=dev, requires_grad=True)
    F = torch.tensor(b["faces"], dtype=torch.int32, device=dev)
    O = torch.tensor(b["order"], dtype=torch.int32, device=dev)
    out = unfold(gpu_ctx, scene, t_tx, t_rx, t_ae, F, O)
    G = rng.normal(size=(P, 8))
    G[:, 3] *= 299792458.0        # delay in metres
    (out * torch.tensor(G, dtype=torch.float32, device=dev)).sum().backward()
    o = out.detach().cpu().numpy().astype(np.float64)
    g_tx, g_rx, g_ae = (x.grad.cpu().numpy().astype(np.float64) for x in (t_tx, t_rx, t_ae))
    S = oracle_mod.Scene.from_generated(sc)
    Tq, Rq, AEq = T.astype(np.float32).astype(np.float64), R.astype(np.float32).astype(np.float64), \
        AE.astype(np.float32).astype(np.float64)

    def rel(a, bref, floor):
        return np.linalg.norm(a - bref) / max(np.linalg.norm(bref), floor)

    for i in rng.choice(P, size=400, replace=False):
        faces = tuple(int(f) for f in b["faces"][i, : b["order"][i]])
        val, J = oracle_mod.unfold(S, faces, Tq[i], Rq[i], AEq[i, 0], AEq[i, 1])
        w = val[3] * 299792458.0
        # FP32 forward: the miss vector carries an absolute error of a few ulps of |Rx' - Tx|
        assert np.linalg.norm(o[i, :3] - val[:3]) <= 1e-3 * np.linalg.norm(val[:3]) + 4e-6 * w
        assert abs(o[i, 3] / val[3] - 1) < 1e-6
        assert ang(dir_of(*o[i, 4:6]), dir_of(*val[4:6])) < 1e-6
        assert ang(dir_of(*o[i, 6:8]), dir_of(*val[6:8])) < 1e-6
        vjp = G[i] @ J                      # (az, el, tx xyz, rx xyz)
        assert rel(g_ae[i], vjp[:2], 1e-6 * w) < 1e-3
        assert rel(g_tx[i], vjp[2:5], 1e-6) < 1e-3
        assert rel(g_rx[i], vjp[5:8], 1e-6) < 1e-3
    # FP64 central differences of the oracle's forward values on a few paths
    for i in rng.choice(P, size=40, replace=False):
        faces = tuple(int(f) for f in b["faces"][i, : b["order"][i]])
        x0 = np.concatenate([AEq[i], Tq[i], Rq[i]])
        fd = np.zeros(8)
        for c in range(8):
            h = 1e-6 if c < 2 else 1e-4
            e = np.zeros(8)
            e[c] = h
            vp = oracle_mod.unfold(S, faces, (x0 + e)[2:5], (x0 + e)[5:8], (x0 + e)[0], (x0 + e)[1])[0]
            vm = oracle_mod.unfold(S, faces, (x0 - e)[2:5], (x0 - e)[5:8], (x0 - e)[0], (x0 - e)[1])[0]
            dv = vp - vm
            dv[4] = np.angle(np.exp(1j * dv[4]))
            dv[6] = np.angle(np.exp(1j * dv[6]))
            fd[c] = G[i] @ (dv / (2 * h))
        gpu = np.concatenate([g_ae[i], g_tx[i], g_rx[i]])
        w = oracle_mod.unfold(S, faces, Tq[i], Rq[i], AEq[i, 0], AEq[i, 1])[0][3] * 299792458.0
        assert rel(gpu[:2], fd[:2], 1e-6 * w) < 1e-3
        assert rel(gpu[2:], fd[2:], 1e-6) < 1e-3


@pytest.mark.slow
def test_large_city_sampled(gpu_ctx, oracle_mod):
    """Large city (~1.07M triangles, 4 Tx x 4096 Rx, n = 2200, order 8): sampled rays of Tx 0
    match the oracle's brute-force trace; sampled refined paths match the image method."""
    sc, tx, rx = scenes.large_city()
    scene = gpu_ctx.scene_from(sc)
    rxs = gpu_ctx.rx_upload(rx)
    n, order, stride = 2200, 8, 199999
    N = 10 * n * n + 2
    per = (N + stride - 1) // stride
    paths = gpu_ctx.paths_create(1 << 24, 1 << 22)
    dump = torch.full((len(tx), per, order + 1), -3, dtype=torch.int32, device="cuda")
    gpu_ctx.launch(scene, tx, rxs, paths, n, order, rx_angle_scale=SQ3, sync=True, dump_stride=stride, dump=dump)
    d = dump.cpu().numpy()[0]
    ids = np.arange(0, N, stride)
    S = oracle_mod.Scene.from_generated(sc)
    tr = oracle_mod.trace(S, tx[0], oracle_mod.lattice_ids(n, ids), rx[:64], order,
                          SQ3 * oracle_mod.theta_launch(n), ray_ids=ids, want_margin=True)
    keep = tr.ray_margin >= EDGE_MARGIN
    assert keep.sum() > 0.9 * len(ids)
    mism = np.nonzero(np.any(d[keep] != tr.ray_faces[keep], axis=1))[0]
    assert len(mism) == 0, (len(mism), d[keep][mism[:3]], tr.ray_faces[keep][mism[:3]])
    # refined far below 0.01 deg (n = 2200 rough rays already meet it) so that the
    # validity test sees bounce points within millimetres of the exact ones
    gpu_ctx.batch_refine(scene, paths, 16, 9)
    (got,) = in_key_order(gpu_ctx.query(paths))
    assert len(got) > 1000
    rng = np.random.default_rng(5)
    valid = got[got["valid"] == 1]
    marginal = 0
    for r in valid[rng.choice(len(valid), size=min(40, len(valid)), replace=False)]:
        faces = tuple(int(f) for f in r["faces"][: r["order"]])
        ev = oracle_mod.path_eval(S, tx[r["tx"]], rx[r["rx"]], faces, r["dir"], err_bound=_bound(oracle_mod, n, 9, r))
        assert ev["valid"]
        im = oracle_mod.image_path(S, tx[r["tx"]], rx[r["rx"]], faces)
        if im["valid"]:
            assert ang(r["dir"], im["aod_dir"]) <= 1e-6
        else:
            marginal += 1
    assert marginal <= 2
    for h in (paths, rxs, scene):
        h.close()


def test_batched_equal_plain_many_paths(gpu_ctx):
    """With enough paths for the batched form's large-launch kernels (planes unfolded one
    path per thread, validity one path per thread) and iterations reaching the FP64 phase,
    the batched form still gives the plain form's results, in the 8-lane and the one-lane
    forms (FP64 iterations in the thread-per-path tail kernel)."""
    sc, tx, rx = scenes.office(ntx=2, nrx=256)
    scene = gpu_ctx.scene_from(sc)
    rxs = gpu_ctx.rx_upload(rx)
    paths = gpu_ctx.paths_create(1 << 22, 1 << 20)
    out = []
    for mode in ("plain", "batch8", "batch1"):
        gpu_ctx.launch(scene, tx, rxs, paths, 128, 6, rx_angle_scale=SQ3, sync=True)
        if mode == "plain":
            gpu_ctx.refine(scene, paths, 12, 16)
        else:
            gpu_ctx.batch_refine(scene, paths, 12, 16, lanes_per_path=int(mode[5:]))
        got = gpu_ctx.query(paths)
        order = np.lexsort((got["order"], got["ray"], got["rx"], got["tx"]))   # (tx, rx, ray, order) is unique
        out.append(got[order])
    a = out[0]
    assert len(a) >= 16 * 32 * gpu_ctx.num_sms
    assert np.any(a["flags"] & 2)                 # some paths iterated in FP64
    for b in out[1:]:
        assert np.array_equal(a["tx"], b["tx"]) and np.array_equal(a["faces"], b["faces"])
        assert np.array_equal(a["iters"], b["iters"]) and np.array_equal(a["valid"], b["valid"])
        assert np.array_equal(a["flags"], b["flags"])
        assert np.max(np.abs(a["dir"] - b["dir"])) < 1e-12
        assert np.all(np.abs(a["delay"] - b["delay"]) <= 1e-12 * np.abs(a["delay"]))
    for h in (paths, rxs, scene):
        h.close()
