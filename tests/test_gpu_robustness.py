"""Failure handling and resume through the C ABI, without faulting the GPU: a failing
allocator callback (host-side injection), export / import of rough paths, and the
precise algorithm's long FP64 run (§IV, Fig. 8a)."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2208_10009_gb300 import _binding as B
from paper_2208_10009_gb300 import api, scenes

from parity_util import ang, replay_refinement

pytestmark = pytest.mark.gpu
SQ3 = float(np.sqrt(3.0))


def test_allocator_failure_is_reported_and_recoverable():
    """The allocator callback starts refusing after a few allocations: the failing call
    returns SBR_ENOMEM with a message, nothing is leaked into a half-built handle, and once
    the allocator works again the same context runs the whole path."""
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    lib = B.load()
    state = {"left": 3, "live": {}}

    def alloc(nbytes, stream, user):
        if state["left"] <= 0:
            return None
        state["left"] -= 1
        p = torch.cuda.caching_allocator_alloc(int(nbytes), 0, int(stream or 0))
        state["live"][p] = nbytes
        return p

    def free(ptr, nbytes, stream, user):
        state["live"].pop(int(ptr), None)
        torch.cuda.caching_allocator_delete(int(ptr))

    a, f = B.ALLOC_FN(alloc), B.FREE_FN(free)
    h = ctypes.c_void_p()
    assert lib.sbr_ctx_create(0, None, a, f, None, ctypes.byref(h)) == 0
    ctx = h.value
    sc, tx, rx = scenes.shoebox_config()
    v = np.ascontiguousarray(sc.verts, np.float32)
    t = np.ascontiguousarray(sc.tris, np.int32)
    tf = np.ascontiguousarray(sc.tri_face, np.int32)
    scene = ctypes.c_void_p()
    assert lib.sbr_scene_upload(ctx, v.ctypes.data_as(B._pf), len(v), t.ctypes.data_as(B._pi32),
                                tf.ctypes.data_as(B._pi32), len(t), None, sc.nf, ctypes.byref(scene)) == 0
    r = np.ascontiguousarray(rx, np.float32)
    rxs = ctypes.c_void_p()
    assert lib.sbr_rx_upload(ctx, r.ctypes.data, 1, ctypes.byref(rxs)) == 0
    paths = ctypes.c_void_p()
    assert lib.sbr_paths_create(ctx, 1 << 16, 1 << 12, ctypes.byref(paths)) == 0
    # the launch needs the direction workspace and lattice tables: refused
    prm = B.LaunchParams(64, 3, SQ3, B.LAUNCH_SYNC, 0, None, 0, 0, 0, 0)
    txh = np.ascontiguousarray(tx, np.float32)
    st = lib.sbr_launch(ctx, scene, txh.ctypes.data, 1, rxs, ctypes.byref(prm), paths)
    assert st == 2 and b"allocation failed" in lib.sbr_last_error(ctx)
    # a new container is refused too
    p2 = ctypes.c_void_p()
    assert lib.sbr_paths_create(ctx, 16, 16, ctypes.byref(p2)) == 2 and not p2.value
    # the allocator recovers: the same context completes launch + refine
    state["left"] = 1 << 30
    assert lib.sbr_launch(ctx, scene, txh.ctypes.data, 1, rxs, ctypes.byref(prm), paths) == 0
    rp = B.RefineParams(5, 9, 0.0, 0.0, 0.0, 0.0, None)
    assert lib.sbr_refine(ctx, scene, paths, ctypes.byref(rp)) == 0
    n = ctypes.c_int64()
    assert lib.sbr_paths_count(ctx, paths, ctypes.byref(n)) == 0 and n.value == 63
    for fn, hh in ((lib.sbr_paths_destroy, paths), (lib.sbr_rx_destroy, rxs), (lib.sbr_scene_destroy, scene)):
        assert fn(ctx, hh) == 0
    assert lib.sbr_ctx_destroy(ctx) == 0
    torch.cuda.synchronize()
    assert not state["live"]          # every block the library took was given back


def test_export_import_resume(gpu_ctx):
    """Checkpoint / resume: rough paths exported with sbr_query and imported into a fresh
    container refine to exactly what the original container gives."""
    sc, tx, rx = scenes.urban_canyon()
    scene = gpu_ctx.scene_from(sc)
    rxs = gpu_ctx.rx_upload(rx)
    a = gpu_ctx.paths_create(1 << 18, 1 << 14)
    b = gpu_ctx.paths_create(1 << 10, 1 << 14)
    gpu_ctx.launch(scene, tx, rxs, a, 300, 4, rx_angle_scale=SQ3, sync=True)
    rough = gpu_ctx.query(a).copy()
    assert len(rough) > 50
    gpu_ctx.paths_import(b, rough, tx, rxs, 300)
    gpu_ctx.refine(scene, a, 6, 9)
    gpu_ctx.refine(scene, b, 6, 9)
    ra = {(int(r["rx"]), tuple(r["faces"])): r for r in gpu_ctx.query(a)}
    rb = {(int(r["rx"]), tuple(r["faces"])): r for r in gpu_ctx.query(b)}
    assert set(ra) == set(rb)
    for k in ra:
        assert ra[k].tobytes() == rb[k].tobytes()
    # records with ids out of range are refused by the kernels, not read out of bounds
    bad = rough[:4].copy()
    bad["rx"] = 10 ** 6
    bad["faces"][:, 0] = -7
    gpu_ctx.paths_import(b, bad, tx, rxs, 300)
    gpu_ctx.batch_refine(scene, b, 3, 9)
    out = gpu_ctx.query(b)
    assert np.all(out["valid"] == 0) and np.all(out["flags"] & B.PATH_TRACE_FAIL)
    for h in (b, a, rxs, scene):
        h.close()


def test_sixty_iterations_plateau(gpu_ctx, oracle_mod):
    """§IV / Fig. 8a: the paper's six sub-rays for 60 iterations.  After the cone falls
    below 1e-5 rad the iterations run in FP64 and the error reaches the double-precision
    floor, and every iteration's decision is checked against the oracle's replay."""
    sc, tx, rx = scenes.shoebox_config()
    scene = gpu_ctx.scene_from(sc)
    rxs = gpu_ctx.rx_upload(rx)
    paths = gpu_ctx.paths_create(1 << 16, 1 << 12)
    gpu_ctx.launch(scene, tx, rxs, paths, 64, 3, rx_angle_scale=SQ3, sync=True)
    choice = torch.full((paths.path_cap, 60), -1, dtype=torch.int8, device="cuda")
    gpu_ctx.batch_refine(scene, paths, 60, 6, choice_log=choice)
    got = gpu_ctx.query(paths)
    ch = choice.cpu().numpy()
    S = oracle_mod.Scene.from_generated(sc)
    tl = oracle_mod.theta_launch(64)
    for i, r in enumerate(got):
        faces = tuple(int(f) for f in r["faces"][: r["order"]])
        im = oracle_mod.image_path(S, tx[0], rx[0], faces)
        assert r["flags"] & B.PATH_FP64
        assert r["err"] < 1e-12 and ang(r["dir"], im["aod_dir"]) < 1e-12
        c0 = oracle_mod.lattice_ids(64, [int(r["ray"])])[0]
        ref = oracle_mod.refine(S, tx[0], rx[0], faces, c0, max(tl, float(r["rough_err"])), 6, 60)
        assert ref["err"] < 1e-12
        # every one of the 60 logged decisions is the oracle's on the same cone, or a tie
        # within the GPU's rounding (once the cone is below the FP32 phase's rounding offset
        # of the centre, all six sub-rays are such ties)
        replay_refinement(oracle_mod, S, tx[0], rx[0], faces, c0, max(float(np.float32(tl)), float(r["rough_err"])),
                          6, r, ch[i], 60)
    for h in (paths, rxs, scene):
        h.close()


def test_checked_build_reports_failed_checks(gpu_ctx, monkeypatch):
    """The SBR_CHECKED build: with its default limits it gives the normal build's results;
    with the traversal stack limited to two entries (SBR_CHECKED_STACK_LIMIT, read at scene
    upload) every walk's bounds check fails before its first push, the kernels record it in
    the launch's status word and return, and the synchronous launch and the query report
    SBR_ECHECK naming the failed checks.  The context stays usable."""
    sc, tx, rx = scenes.shoebox_config()
    ctx = api.Context(0, checked=True)
    scene = ctx.scene_from(sc)
    rxs = ctx.rx_upload(rx)
    paths = ctx.paths_create(1 << 16, 1 << 12)
    ctx.launch(scene, tx, rxs, paths, 32, 3, rx_angle_scale=SQ3, sync=True)
    ctx.refine(scene, paths, 5, 9)
    got = ctx.query(paths)
    assert ctx.launch_stats(paths)["check_flags"] == 0
    ref_scene = gpu_ctx.scene_from(sc)
    ref_rx = gpu_ctx.rx_upload(rx)
    ref_paths = gpu_ctx.paths_create(1 << 16, 1 << 12)
    gpu_ctx.launch(ref_scene, tx, ref_rx, ref_paths, 32, 3, rx_angle_scale=SQ3, sync=True)
    gpu_ctx.refine(ref_scene, ref_paths, 5, 9)
    want = gpu_ctx.query(ref_paths)
    key = lambda a: a[np.lexsort((a["order"], a["ray"]))]
    assert key(got).tobytes() == key(want).tobytes()
    monkeypatch.setenv("SBR_CHECKED_STACK_LIMIT", "2")
    small = ctx.scene_from(sc)
    monkeypatch.delenv("SBR_CHECKED_STACK_LIMIT")
    with pytest.raises(api.SbrError) as e:
        ctx.launch(small, tx, rxs, paths, 32, 3, rx_angle_scale=SQ3, sync=True)
    assert e.value.status == 8 and "trace stack" in str(e.value)
    st = ctx.launch_stats(paths)
    assert st["check_flags"] & 1 and st["segments"] == st["rays"]   # every walk stopped at the root
    with pytest.raises(api.SbrError) as e:
        ctx.query(paths)
    assert e.value.status == 8
    # the same context and container run cleanly on the unrestricted scene again
    ctx.launch(scene, tx, rxs, paths, 32, 3, rx_angle_scale=SQ3, sync=True)
    ctx.refine(scene, paths, 5, 9)
    assert len(ctx.query(paths)) == len(want)
    for h in (small, paths, rxs, scene, ref_paths, ref_rx, ref_scene):
        h.close()
    ctx.close()


def test_nonfinite_output_scan(gpu_ctx):
    """The output scan counts valid paths with a NaN or Inf output: none after a normal
    run; an imported record set with one valid path's delay set to NaN and another's power
    to +Inf counts two (an invalid path's outputs are not scanned)."""
    sc, tx, rx = scenes.shoebox_config()
    scene = gpu_ctx.scene_from(sc)
    rxs = gpu_ctx.rx_upload(rx)
    paths = gpu_ctx.paths_create(1 << 16, 1 << 12)
    gpu_ctx.launch(scene, tx, rxs, paths, 32, 3, rx_angle_scale=SQ3, sync=True)
    gpu_ctx.refine(scene, paths, 5, 9)
    assert gpu_ctx.paths_nonfinite(paths) == 0
    got = gpu_ctx.query(paths)
    v = np.nonzero(got["valid"] == 1)[0]
    assert len(v) > 10
    bad = got.copy()
    bad["delay"][v[0]] = np.nan
    bad["power_dbm"][v[1]] = np.inf
    bad["valid"][v[2]] = 0
    bad["err"][v[2]] = np.nan
    gpu_ctx.paths_import(paths, bad, tx, rxs, 32)
    assert gpu_ctx.paths_nonfinite(paths) == 2
    for h in (paths, rxs, scene):
        h.close()
