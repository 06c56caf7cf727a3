"""Pins for the oracle's fixed-face-sequence unfolding and its closed-form gradients:
FP64 central finite differences, and agreement with the image method."""
import numpy as np
import pytest

from paper_2208_10009_gb300 import scenes

C0 = 299792458.0


def _paths(oracle_mod):
    sc, tx, rx = scenes.shoebox_config()
    S = oracle_mod.Scene.from_generated(sc)
    im = oracle_mod.image_enumerate(S, tx[0], rx[0], 3)
    return S, tx[0], rx[0], im


def test_unfold_values_match_image_method(oracle_mod):
    S, tx, rx, im = _paths(oracle_mod)
    for p in im:
        d = p["aod_dir"]
        az, el = np.arctan2(d[1], d[0]), np.arctan2(d[2], np.hypot(d[0], d[1]))
        val, _ = oracle_mod.unfold(S, p["faces"], tx, rx, az, el)
        q = oracle_mod.image_path(S, tx, rx, p["faces"])
        assert np.linalg.norm(val[:3]) < 1e-9                  # exact launch hits Rx
        assert abs(val[3] - q["delay"]) < 1e-18
        assert np.allclose(val[4:6], q["aod"], atol=1e-12)
        assert np.allclose(val[6:8], q["aoa"], atol=1e-12)


def test_unfold_miss_is_lateral_offset(oracle_mod):
    """Perturbing the launch by a small angle delta moves the ray past Rx by
    |miss| = |Rx' - Tx| sin(delta)."""
    S, tx, rx, im = _paths(oracle_mod)
    for p in im[::5]:
        d = p["aod_dir"]
        az, el = np.arctan2(d[1], d[0]), np.arctan2(d[2], np.hypot(d[0], d[1]))
        delta = 1e-3
        val, _ = oracle_mod.unfold(S, p["faces"], tx, rx, az, el + delta)
        assert abs(np.linalg.norm(val[:3]) - p["delay"] * C0 * np.sin(delta)) < 1e-9


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_unfold_gradient_central_differences(oracle_mod, seed):
    """Closed-form Jacobian vs FP64 central differences (h = 1e-4 m, 1e-6 rad)."""
    sc, _, _ = scenes.urban_canyon()
    S = oracle_mod.Scene.from_generated(sc)
    rng = np.random.default_rng(seed)
    for _ in range(20):
        k = int(rng.integers(0, 7))
        faces = []
        for _ in range(k):
            f = int(rng.integers(0, sc.nf))
            while faces and f == faces[-1]:
                f = int(rng.integers(0, sc.nf))
            faces.append(f)
        tx = rng.uniform([0, 0, 1], [1000, 1000, 60])
        rx = rng.uniform([0, 0, 1], [1000, 1000, 60])
        az, el = rng.uniform(-np.pi, np.pi), rng.uniform(-1.2, 1.2)
        x0 = np.concatenate([[az, el], tx, rx])

        def f(x):
            return oracle_mod.unfold(S, faces, x[2:5], x[5:8], x[0], x[1])[0]

        _, J = oracle_mod.unfold(S, faces, tx, rx, az, el)
        for c in range(8):
            h = 1e-6 if c < 2 else 1e-4
            e = np.zeros(8)
            e[c] = h
            fd = (f(x0 + e) - f(x0 - e)) / (2 * h)
            fd[4] = (np.angle(np.exp(1j * (f(x0 + e)[4] - f(x0 - e)[4])))) / (2 * h)
            fd[6] = (np.angle(np.exp(1j * (f(x0 + e)[6] - f(x0 - e)[6])))) / (2 * h)
            scale = np.array([1, 1, 1, 1 / C0, 1e-3, 1e-3, 1e-3, 1e-3]) * max(np.abs(J[:, c]).max(), 1e-12)
            err = np.abs(fd - J[:, c])
            assert np.all(err <= 1e-5 * np.maximum(np.abs(J[:, c]), scale)), (faces, c, fd, J[:, c])


def test_unfold_many_equals_unfold(oracle_mod):
    """The batched form returns the one-path values (az = el = 0) for every path, and its
    AOD / AOA / delay equal the image method's on the shoebox's 63 paths."""
    from paper_2208_10009_gb300 import scenes
    sc, tx, rx = scenes.shoebox_config()
    S = oracle_mod.Scene.from_generated(sc)
    im = oracle_mod.image_enumerate(S, tx[0], rx[0], 3)
    assert len(im) == 63
    order = np.array([len(p["faces"]) for p in im])
    faces = np.full((len(im), 8), -1)
    for i, p in enumerate(im):
        faces[i, : order[i]] = p["faces"]
    T, R = np.repeat(tx, len(im), 0), np.repeat(rx, len(im), 0)
    v = oracle_mod.unfold_many(S, order, faces, T, R)
    for i, p in enumerate(im):
        one, _ = oracle_mod.unfold(S, p["faces"], tx[0], rx[0], 0.0, 0.0)
        assert np.array_equal(v[i], one)
        d = np.array([np.cos(v[i, 5]) * np.cos(v[i, 4]), np.cos(v[i, 5]) * np.sin(v[i, 4]), np.sin(v[i, 5])])
        assert np.arctan2(np.linalg.norm(np.cross(d, p["aod_dir"])), d @ p["aod_dir"]) < 1e-12
        assert abs(v[i, 3] / p["delay"] - 1) < 1e-13
