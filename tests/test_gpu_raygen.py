"""a1 parity: the CUDA ray generator against the oracle's equiangular lattice."""
import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

# FP32 slerp + normalisation: every direction within 5e-7 rad of the FP64 lattice point
TOL = 5e-7


def _angles(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=1), np.sum(a * b, axis=1))


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 21, 64, 129])
def test_raygen_matches_oracle(gpu_ctx, oracle_mod, n):
    d = gpu_ctx.raygen(n).cpu().numpy()
    assert d.shape == (10 * n * n + 2, 4)
    want = oracle_mod.lattice(n)
    got = d[:, :3].astype(np.float64)
    assert np.abs(np.linalg.norm(got, axis=1) - 1).max() < 3e-7
    assert _angles(got, want).max() < TOL
    assert np.all(d[:, 3] == 0)


@pytest.mark.parametrize("n", [700, 2200])
def test_raygen_full_size_sampled(gpu_ctx, oracle_mod, n):
    d = gpu_ctx.raygen(n)
    N = 10 * n * n + 2
    rng = np.random.default_rng(n)
    ids = np.unique(np.concatenate([rng.integers(0, N, 20000), np.arange(0, 200), np.arange(N - 200, N)]))
    got = d[torch.as_tensor(ids, device=d.device)].cpu().numpy()[:, :3].astype(np.float64)
    want = oracle_mod.lattice_ids(n, ids)
    assert _angles(got, want).max() < TOL
    del d
    torch.cuda.empty_cache()


def test_raygen_rejects_bad_sizes(gpu_ctx):
    from paper_2208_10009_gb300 import api
    small = torch.empty((10, 4), dtype=torch.float32, device="cuda")
    with pytest.raises(api.SbrError):
        gpu_ctx.raygen(2, small)
    with pytest.raises(api.SbrError):
        gpu_ctx.raygen(0, small)


@pytest.mark.parametrize("poly", [20, 8])
@pytest.mark.parametrize("n", [1, 2, 3, 7, 21, 64, 250])
def test_equidistant_matches_oracle(gpu_ctx, oracle_mod, poly, n):
    d = gpu_ctx.raygen_equidistant(n, poly).cpu().numpy()
    want = oracle_mod.equidistant(n, poly)
    assert d.shape == (len(want), 4)
    assert _angles(d[:, :3].astype(np.float64), want).max() < TOL


def test_equidistant_launch_matches_oracle(gpu_ctx, oracle_mod):
    """The whole path on the equidistant icosahedron (launcher 20): rough paths after
    double-count removal equal the oracle's, refined paths reach the image method."""
    from paper_2208_10009_gb300 import scenes
    sc, tx, rx = scenes.shoebox_config()
    scene = gpu_ctx.scene_from(sc)
    rxs = gpu_ctx.rx_upload(rx)
    paths = gpu_ctx.paths_create(1 << 16, 1 << 12)
    sq3 = float(np.sqrt(3.0))
    gpu_ctx.launch(scene, tx, rxs, paths, 48, 3, rx_angle_scale=sq3, sync=True, launcher=20)
    rough = gpu_ctx.query(paths)
    S = oracle_mod.Scene.from_generated(sc)
    ora = oracle_mod.sbr_pipeline(S, tx, rx, 48, 3, sq3, 9, 0, refine_paths=False, launcher=20)
    g = {tuple(int(f) for f in r["faces"][: r["order"]]) for r in rough}
    o = {p["faces"] for p in ora.paths}
    assert g == o
    gpu_ctx.refine(scene, paths, 10, 9)
    got = gpu_ctx.query(paths)
    im = {p["faces"]: p for p in oracle_mod.image_enumerate(S, tx[0], rx[0], 3)}
    for r in got:
        key = tuple(int(f) for f in r["faces"][: r["order"]])
        if r["valid"]:
            a = np.asarray(r["dir"], np.float64)
            assert np.arctan2(np.linalg.norm(np.cross(a, im[key]["aod_dir"])), a @ im[key]["aod_dir"]) < np.radians(0.01)
    for h in (paths, rxs, scene):
        h.close()
