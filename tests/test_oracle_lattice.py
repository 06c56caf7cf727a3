"""Pins for the oracle's equiangular launcher (§II.B, Eq. 1-2, Eq. 8) and sub-ray patterns
(§III.B, Eq. 10) against what the paper prints and what geometry fixes."""
import json
import os

import numpy as np
import pytest
from scipy.spatial import cKDTree

GOLD = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_constants.json")))


def _ang(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


def test_icosahedron_is_regular(oracle_mod):
    v, f, e = oracle_mod.icosahedron()
    assert np.allclose(np.linalg.norm(v, axis=1), 1.0, atol=1e-15)
    assert len(f) == 20 and len(e) == 30 and 12 - 30 + 20 == 2
    # every vertex has 5 neighbours, all edges subtend the same angle theta0
    deg = np.bincount(e.ravel(), minlength=12)
    assert np.all(deg == 5)
    angs = np.degrees(_ang(v[e[:, 0]], v[e[:, 1]]))
    assert np.allclose(angs, GOLD["theta0_deg"]["value"], atol=5e-5)
    assert abs(np.degrees(oracle_mod.theta0()) - GOLD["theta0_deg"]["value"]) < 5e-5
    # faces are outward-oriented triangles of mutually adjacent vertices
    for a, b, c in f:
        nrm = np.cross(v[b] - v[a], v[c] - v[a])
        assert nrm @ (v[a] + v[b] + v[c]) > 0
        assert a < b and a < c


def test_ray_count_and_constants(oracle_mod):
    for n in range(1, 65):
        assert oracle_mod.num_rays(n) == 10 * n * n + 2
    assert oracle_mod.num_rays(21) == GOLD["rays_launched"]["value"]
    for n in (1, 2, 3, 4, 7, 21):
        assert len(oracle_mod.lattice(n)) == 10 * n * n + 2
    # theta_error <= 115.8158 deg / sqrt(N - 2) is Eq. 8 rewritten with N = 10 n^2 + 2
    for n in (5, 21, 64):
        N = oracle_mod.num_rays(n)
        assert abs(np.degrees(oracle_mod.theta_launch(n)) * np.sqrt(N - 2) - GOLD["error_bound_constant_deg"]["value"]) < 5e-4
    # Eq. 10's right-hand side theta_launch / 3^(i/2) == 63.4349 deg / (3^((i+1)/2) n)
    for n, i in ((21, 0), (21, 10), (64, 5)):
        lhs = np.degrees(oracle_mod.theta_launch(n)) / 3 ** (i / 2)
        rhs = GOLD["eq10_constant_deg"]["value"] / (3 ** ((i + 1) / 2) * n)
        assert abs(lhs / rhs - 1) < 1e-5
    # 10 iterations of 1/sqrt(3) shrink: 10 log10(3^5) = 23.86 dB ~ "24 dB"
    assert round(10 * np.log10(np.sqrt(3) ** 10)) == GOLD["reduction_10_iterations_db"]["value"]
    # the printed office result respects the Eq. 10 bound for n = 21, i = 10
    bound = np.degrees(oracle_mod.theta_launch(21)) / 3 ** 5
    assert GOLD["office_mean_aod_error_deg"]["precise_10_iter"] <= bound


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 8, 21, 64])
def test_directions_unit_and_distinct(oracle_mod, n):
    d = oracle_mod.lattice(n)
    assert np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-15
    dist, _ = cKDTree(d).query(d, k=2)
    nn = 2 * np.arcsin(dist[:, 1] / 2)
    # no two rays closer than half the edge spacing; spacing uniform within ~12%
    spacing = oracle_mod.theta0() / n
    assert nn.min() > 0.5 * spacing
    if n >= 8:
        assert nn.max() / nn.min() < 1.12


@pytest.mark.parametrize("n", [1, 2, 3, 4, 5, 6, 7, 9, 10, 21, 64])
def test_face_layers(oracle_mod, n):
    """Per face: (n+1)(n+2)/2 points; layer a has 3(n-3a) = 3n-9a points (3n on layer 0);
    innermost layer: a single centre ray if n = 0 mod 3, three rays if n = 1 mod 3,
    none beyond the last six-point layer if n = 2 mod 3."""
    glob = oracle_mod.lattice(n)
    tree = cKDTree(glob)
    seen = np.zeros(len(glob), int)
    for f in range(20):
        pts, layer, idx = oracle_mod.face_points(n, f)
        assert len(pts) == (n + 1) * (n + 2) // 2
        counts = np.bincount(layer)
        for a, c in enumerate(counts):
            m = n - 3 * a
            assert c == (3 * m if m >= 1 else 1)
        assert counts[0] == 3 * n
        last = n - 3 * (len(counts) - 1)
        inner = counts[-1]
        assert inner == {0: 1, 1: 3, 2: 6}[n % 3] and (last == 0) == (n % 3 == 0)
        # every face point is one of the global rays (shared boundary points coincide)
        dist, j = tree.query(pts)
        assert dist.max() < 1e-14
        seen[j[layer > 0]] += 1
    # interior points belong to exactly one face; vertex/edge rays are not interior
    assert np.all(seen[12 + 30 * (n - 1):] == 1)
    assert np.all(seen[: 12 + 30 * (n - 1)] == 0)


@pytest.mark.parametrize("n", [6, 13, 21])
def test_equal_angles_on_layer_edges(oracle_mod, n):
    """Eq. 1: consecutive points on every layer edge subtend the same angle; on layer 0
    that angle is theta0 / n."""
    for f in (0, 7, 19):
        pts, layer, idx = oracle_mod.face_points(n, f)
        for a in range(layer.max() + 1):
            m = n - 3 * a
            if m < 1:
                continue
            P = pts[layer == a]
            ring = np.vstack([P, P[:1]])
            steps = _ang(ring[:-1], ring[1:])
            for e in range(3):
                s = steps[e * m:(e + 1) * m]
                assert np.ptp(s) < 1e-12
            if a == 0:
                assert np.allclose(steps, oracle_mod.theta0() / n, atol=1e-13)


@pytest.mark.parametrize("n", [5, 9, 22])
def test_face_c3_symmetry(oracle_mod, n):
    """The construction is the same from each of the face's three vertices, so the face's
    point set is invariant under the face's 120-degree rotation."""
    v, F, _ = oracle_mod.icosahedron()
    for f in (0, 11):
        pts, _, _ = oracle_mod.face_points(n, f)
        axis = v[F[f]].sum(0)
        axis /= np.linalg.norm(axis)
        K = np.array([[0, -axis[2], axis[1]], [axis[2], 0, -axis[0]], [-axis[1], axis[0], 0]])
        R = np.eye(3) + np.sin(2 * np.pi / 3) * K + (1 - np.cos(2 * np.pi / 3)) * K @ K
        dist, _ = cKDTree(pts).query(pts @ R.T)
        assert dist.max() < 1e-12


@pytest.mark.parametrize("n", [8, 21])
def test_covering_radius_near_theta_launch(oracle_mod, n):
    """Eq. 8 takes the cone half-angle as theta_launch = theta0 / (sqrt(3) n), the covering
    radius of a perfect triangular lattice of spacing theta0 / n.  The spherical lattice's
    true covering radius is within 15% of it."""
    d = oracle_mod.lattice(n)
    rng = np.random.default_rng(7)
    q = rng.normal(size=(200000, 3))
    q /= np.linalg.norm(q, axis=1)[:, None]
    dist, _ = cKDTree(d).query(q)
    cover = 2 * np.arcsin(dist.max() / 2)
    ratio = cover / oracle_mod.theta_launch(n)
    assert 1.0 < ratio < 1.15


@pytest.mark.parametrize("K", [6, 7, 9, 16])
def test_subray_pattern_covers_cone(oracle_mod, K):
    """§III.B, Fig. 5: the K sub-cones (radius shrink * R around the sub-ray directions) must
    cover the parent cone of radius R; checked by brute force over the unit disc."""
    rho, phi, s = oracle_mod.subray_pattern(K)
    C = np.stack([rho * np.cos(phi), rho * np.sin(phi)], -1)
    rng = np.random.default_rng(K)
    p = rng.uniform(-1, 1, (400000, 2))
    p = p[(p ** 2).sum(1) <= 1]
    t = np.linspace(0, 2 * np.pi, 20000, endpoint=False)
    p = np.vstack([p, np.c_[np.cos(t), np.sin(t)]])
    dmin, _ = cKDTree(C).query(p)
    assert dmin.max() <= s * (1 + 1e-9)
    assert dmin.max() >= s * (1 - 1e-3)  # and the shrink factor is tight
    if K == 6:
        assert abs(s - 1 / np.sqrt(3)) < 1e-15  # the paper's 1/sqrt(3)
    if K == 9:
        assert abs(s - (np.sqrt(2) - 1)) < 1e-15
