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
