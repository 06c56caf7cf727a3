"""Pins for the oracle's tracing, reception (Eq. 3), image method and validity against
closed forms: one plane, a two-wall corridor, the rectangular room's image lattice."""
import itertools

import numpy as np
import pytest

from paper_2208_10009_gb300 import scenes

C0 = 299792458.0


def _ang(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b)), np.dot(a, b))


def test_single_plane_specular_point_and_delay(oracle_mod):
    S = oracle_mod.Scene.from_generated(scenes.single_plane())
    h1, h2, d = 7.0, 2.0, 30.0
    tx, rx = np.array([0.0, 0.0, h1]), np.array([d, 0.0, h2])
    im = oracle_mod.image_path(S, tx, rx, (0,))
    assert im["valid"]
    # reflection point on line(Tx', Rx) with Tx' = (0, 0, -h1)
    assert np.allclose(im["points"][0], [d * h1 / (h1 + h2), 0.0, 0.0], atol=1e-12)
    assert abs(im["delay"] - np.hypot(d, h1 + h2) / C0) < 1e-18
    los = oracle_mod.image_path(S, tx, rx, ())
    assert los["valid"] and abs(los["delay"] - np.linalg.norm(rx - tx) / C0) < 1e-18
    # exhaustive IM finds exactly LOS + one ground bounce
    paths = oracle_mod.image_enumerate(S, tx, rx, 3)
    assert sorted(p["faces"] for p in paths) == [(), (0,)]


def test_single_plane_power_special_cases(oracle_mod):
    """Free-space loss 20 log10(lambda / (4 pi L)); at normal incidence the perpendicular
    Fresnel coefficient is (1 - sqrt(eps)) / (1 + sqrt(eps)): -1/3 for eps = 4."""
    lam = C0 / 2.4e9
    S = oracle_mod.Scene.from_generated(scenes.single_plane(eps=4.0))
    tx, rx = np.array([0.0, 0.0, 3.0]), np.array([0.0, 0.0, 1.0])
    im = oracle_mod.image_path(S, tx, rx, (0,))
    L = 4.0
    assert abs(im["power"] - (20 * np.log10(lam / (4 * np.pi * L)) + 20 * np.log10(1 / 3))) < 1e-9
    los = oracle_mod.image_path(S, tx, rx, ())
    assert abs(los["power"] - 20 * np.log10(lam / (4 * np.pi * 2.0))) < 1e-9
    # perfect reflector: no reflection loss
    S1 = oracle_mod.Scene.from_generated(scenes.single_plane())
    im1 = oracle_mod.image_path(S1, tx, rx, (0,))
    assert abs(im1["power"] - 20 * np.log10(lam / (4 * np.pi * L))) < 1e-9
    # near grazing |Gamma| -> 1
    txg, rxg = np.array([0.0, 0.0, 0.01]), np.array([1000.0, 0.0, 0.01])
    g = oracle_mod.image_path(S, txg, rxg, (0,))
    Lg = np.hypot(1000.0, 0.02)
    assert abs(g["power"] - 20 * np.log10(lam / (4 * np.pi * Lg))) < 0.01


def test_corridor_images(oracle_mod):
    """Two parallel walls y = 0 and y = W: the order-k images of Tx sit at y = 2mW +- y_Tx and
    exactly two order-k paths exist for every k >= 1."""
    W = 4.0
    S = oracle_mod.Scene.from_generated(scenes.corridor(W))
    tx, rx = np.array([0.0, 1.3, 1.0]), np.array([25.0, 2.9, 1.7])
    paths = oracle_mod.image_enumerate(S, tx, rx, 6)
    for k in range(0, 7):
        got = sorted(p["delay"] for p in paths if p["order"] == k)
        # image set along y: 2mW + y (2|m| reflections), 2mW - y (|2m - 1| reflections)
        ys = []
        for m in range(-8, 9):
            if 2 * abs(m) == k:
                ys.append(2 * m * W + tx[1])
            if abs(2 * m - 1) == k:
                ys.append(2 * m * W - tx[1])
        want = sorted(np.sqrt((rx[0] - tx[0]) ** 2 + (rx[1] - y) ** 2 + (rx[2] - tx[2]) ** 2) / C0 for y in ys)
        assert len(got) == (1 if k == 0 else 2)
        assert np.allclose(got, want, rtol=1e-14, atol=0)


def test_shoebox_image_lattice(oracle_mod):
    """Rectangular room: valid order-k paths = integer points of L1 norm k in 3-D, i.e.
    4k^2 + 2 for k >= 1 (6, 18, 38), with delays from the image lattice."""
    sc, tx, rx = scenes.shoebox_config()
    L, W, H = sc.meta["dims"]
    S = oracle_mod.Scene.from_generated(sc)
    paths = oracle_mod.image_enumerate(S, tx[0], rx[0], 3)
    t, r = tx[0], rx[0]

    def axis_images(p, size):
        out = []
        for m in range(-4, 5):
            out.append((2 * m * size + p, 2 * abs(m)))
            out.append((2 * m * size - p, abs(2 * m - 1)))
        return out

    for k in range(4):
        got = sorted(p["delay"] for p in paths if p["order"] == k)
        want = []
        for (x, a), (y, b), (z, c) in itertools.product(axis_images(t[0], L), axis_images(t[1], W),
                                                         axis_images(t[2], H)):
            if a + b + c == k:
                want.append(np.linalg.norm(r - np.array([x, y, z])) / C0)
        assert len(got) == (1 if k == 0 else 4 * k * k + 2)
        assert np.allclose(got, sorted(want), rtol=1e-13, atol=0)


def test_reception_error_angle_equals_unfolded_angle(oracle_mod):
    """Eq. 3 measured on a received ray equals the angle between that ray's launch direction
    and the exact image-method departure direction of the same face sequence."""
    sc, tx, rx = scenes.shoebox_config()
    S = oracle_mod.Scene.from_generated(sc)
    n = 16
    dirs = oracle_mod.lattice(n)
    tr = oracle_mod.trace(S, tx[0], dirs, rx, 3, np.sqrt(3) * oracle_mod.theta_launch(n))
    assert len(tr.rec_err) > 20
    checked = 0
    for i in range(len(tr.rec_err)):
        k = tr.rec_order[i]
        faces = tuple(tr.rec_faces[i, :k])
        val, _ = oracle_mod.unfold(S, faces, tx[0], rx[0], 0.0, 0.0)
        exact = np.array([np.cos(val[5]) * np.cos(val[4]), np.cos(val[5]) * np.sin(val[4]), np.sin(val[5])])
        assert abs(_ang(dirs[tr.rec_ray[i]], exact) - tr.rec_err[i]) < 1e-12
        # d_ray is the distance along the unfolded ray to the foot of Rx'
        assert abs(tr.rec_dray[i] - val[3] * C0 * np.cos(tr.rec_err[i])) < 1e-9
        im = oracle_mod.image_path(S, tx[0], rx[0], faces)
        if im["status"] >= 0:
            assert abs(_ang(dirs[tr.rec_ray[i]], im["aod_dir"]) - tr.rec_err[i]) < 1e-12
            checked += 1
    assert checked > 20


def test_closed_room_every_ray_bounces(oracle_mod):
    sc, tx, rx = scenes.shoebox_config()
    S = oracle_mod.Scene.from_generated(sc)
    dirs = oracle_mod.lattice(8)
    tr = oracle_mod.trace(S, tx[0], dirs, rx, 3, 0.1)
    assert np.all(tr.ray_nseg == 4) and tr.nsegments == 4 * len(dirs)
    assert np.all(tr.ray_faces >= 0)
    # consecutive faces differ (a ray cannot hit the plane it just left)
    assert np.all(tr.ray_faces[:, 1:] != tr.ray_faces[:, :-1])


def test_open_scene_misses_and_face_skip(oracle_mod):
    """Above a single plane, upward rays miss at once; downward rays bounce once and then
    escape: segments = 1 (up) or 2 (down)."""
    S = oracle_mod.Scene.from_generated(scenes.single_plane())
    dirs = oracle_mod.lattice(6)
    tr = oracle_mod.trace(S, [0, 0, 5.0], dirs, [[10, 0, 1.0]], 4, 0.1)
    down = dirs[:, 2] < -1e-3
    up = dirs[:, 2] > 1e-12
    assert np.all(tr.ray_nseg[down] == 2) and np.all(tr.ray_faces[down, 0] == 0)
    assert np.all(tr.ray_nseg[up] == 1) and np.all(tr.ray_faces[up, 0] == -1)


def test_validity_outside_face(oracle_mod):
    """A face sequence whose image-method bounce point lies off its (finite) face is
    rejected by the validity test, and so is an occluded one."""
    b = scenes._Builder()
    b.quad((0, 0, 0), (1, 0, 0), (0, 1, 0))              # small floor tile, face 0
    b.quad((-5, -5, 1.0), (-5, 5, 1.0), (5, -5, 1.0))    # blocker plane z = 1 (face 1)
    sc = b.finish()
    S = oracle_mod.Scene.from_generated(sc)
    # bounce point at x = 5 is outside the unit tile
    im = oracle_mod.image_path(S, [0, 0.5, 0.5], [10, 0.5, 0.5], (0,))
    assert im["status"] == 0 and not im["valid"]
    # bounce inside the tile but the LOS and the bounce legs stay below z = 1: valid
    im2 = oracle_mod.image_path(S, [0.2, 0.5, 0.5], [0.8, 0.5, 0.5], (0,))
    assert im2["valid"]
    # Rx above the blocker: the last leg crosses z = 1 -> occluded
    im3 = oracle_mod.image_path(S, [0.2, 0.5, 0.5], [0.8, 0.5, 1.5], (0,))
    assert im3["status"] == 0 and not im3["valid"]
