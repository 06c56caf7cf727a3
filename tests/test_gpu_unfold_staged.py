"""GPU tests of the adjoint's two forms: the staged kernel (bulk copies of whole 256-path
tiles into shared memory, the ragged last tile from global memory) must give, path for path,
the bits of the direct kernel (each thread loads its own path), which runs when an input
array is not 16-byte aligned.  The staged form's values against the oracle are checked by
the 1M-path gradient test."""
import numpy as np
import pytest
import torch

from paper_2208_10009_gb300 import scenes

pytestmark = pytest.mark.gpu


def _unaligned_copy(t):
    """The same values in a buffer whose data pointer is 4 bytes past a 16-byte boundary."""
    flat = torch.empty(t.numel() + 1, dtype=t.dtype, device=t.device)
    u = flat[1:].view(t.shape)
    u.copy_(t)
    assert u.data_ptr() % 16 == 4
    return u


def test_staged_adjoint_equals_direct(gpu_ctx):
    sc, tx, rx = scenes.urban_canyon()
    scene = gpu_ctx.scene_from(sc)
    rng = np.random.default_rng(11)
    full_tiles = 2 * 152 + 16          # enough tiles for the staged form on a 152-SM GPU
    n = full_tiles * 256 + 37           # and a ragged last tile
    dev = "cuda"
    T = torch.tensor(rng.uniform(0, 1000, (n, 3)), dtype=torch.float32, device=dev)
    R = torch.tensor(rng.uniform(0, 1000, (n, 3)), dtype=torch.float32, device=dev)
    AE = torch.tensor(np.stack([rng.uniform(-np.pi, np.pi, n), rng.uniform(-1.2, 1.2, n)], -1),
                      dtype=torch.float32, device=dev)
    faces = rng.integers(0, sc.nf, (n, 8)).astype(np.int32)
    order = rng.integers(0, 9, n).astype(np.int32)
    faces[5, 0] = sc.nf + 3             # an id out of range: NaN gradients for that path
    order[5] = max(order[5], 1)
    F = torch.tensor(faces, device=dev)
    O = torch.tensor(order, device=dev)
    G = torch.tensor(rng.normal(size=(n, 8)), dtype=torch.float32, device=dev)

    staged = gpu_ctx.unfold_bwd(scene, T, R, AE, F, O, G)
    direct = gpu_ctx.unfold_bwd(scene, _unaligned_copy(T), R, AE, F, O, G)
    whole = gpu_ctx.unfold_bwd(scene, T[: full_tiles * 256], R[: full_tiles * 256], AE[: full_tiles * 256],
                               F[: full_tiles * 256], O[: full_tiles * 256], G[: full_tiles * 256])
    torch.cuda.synchronize()
    for s, d, w in zip(staged, direct, whole):
        s, d, w = s.cpu().numpy(), d.cpu().numpy(), w.cpu().numpy()
        assert np.array_equal(s, d, equal_nan=True)
        assert np.array_equal(s[: full_tiles * 256], w, equal_nan=True)
        assert np.isnan(s[5]).all()
        ok = np.ones(n, bool)
        ok[5] = False
        assert np.isfinite(s[ok]).all()
    scene.close()
