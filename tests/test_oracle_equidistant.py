"""Pins for the equidistant launcher of §II.A (ref. 9) and the uniformity comparison of
Fig. 2: equidistant division on an octahedron is the least uniform, on an icosahedron
better, and the paper's equiangular division the most uniform."""
import numpy as np
import pytest
from scipy.spatial import cKDTree


def _ang(a, b):
    return np.arctan2(np.linalg.norm(np.cross(a, b), axis=-1), np.sum(a * b, axis=-1))


@pytest.mark.parametrize("poly,nv,ne,nf", [(20, 12, 30, 20), (8, 6, 12, 8)])
def test_counts_and_flat_geometry(oracle_mod, poly, nv, ne, nf):
    for n in (1, 2, 3, 7, 21):
        d = oracle_mod.equidistant(n, poly)
        assert len(d) == nv + ne * (n - 1) + nf * (n - 1) * (n - 2) // 2
        assert len(d) == (10 if poly == 20 else 4) * n * n + 2
        assert np.abs(np.linalg.norm(d, axis=1) - 1).max() < 1e-15
        dist, _ = cKDTree(d).query(d, k=2)
        assert dist[:, 1].min() > 1e-3 / n          # no duplicates
    # edge points: equal chords on the flat edge, so after projection the angular gaps
    # widen towards the middle of the edge (the spreading described in §II.A)
    n = 12
    d = oracle_mod.equidistant(n, poly)
    e0 = d[nv:nv + n - 1]
    v = d[:nv]
    lo = v[np.argmin(_ang(v, e0[0][None, :]))]
    hi = v[np.argmin(_ang(v, e0[-1][None, :]))]
    pts = np.vstack([lo, e0, hi])
    gaps = _ang(pts[:-1], pts[1:])
    half = len(gaps) // 2
    assert np.all(np.diff(gaps[:half]) > 0) and np.all(np.diff(gaps[-half:]) < 0)


def _density_cv(d, bins=(24, 12)):
    """Fig. 2's map: abscissa azimuth * cos(pitch), ordinate pitch (area preserving); the
    coefficient of variation of the counts in cells that lie inside the map."""
    az = np.arctan2(d[:, 1], d[:, 0])
    el = np.arcsin(np.clip(d[:, 2], -1, 1))
    H, xe, ye = np.histogram2d(az * np.cos(el), el, bins=bins, range=[[-np.pi, np.pi], [-np.pi / 2, np.pi / 2]])
    xc, yc = 0.5 * (xe[1:] + xe[:-1]), 0.5 * (ye[1:] + ye[:-1])
    inside = np.abs(xc)[:, None] + 0.5 * (xe[1] - xe[0]) < np.pi * np.cos(np.abs(yc)[None, :] + 0.5 * (ye[1] - ye[0]))
    return H[inside].std() / H[inside].mean()


def _nn_ratio(d):
    dist, _ = cKDTree(d).query(d, k=2)
    nn = 2 * np.arcsin(dist[:, 1] / 2)
    return nn.max() / nn.min()


def test_fig2_uniformity_ordering(oracle_mod):
    """Fig. 2 at the paper's 4412 rays (n = 21; the octahedron at n = 33, 4358 rays)."""
    ea = oracle_mod.lattice(21)
    ico = oracle_mod.equidistant(21, 20)
    octa = oracle_mod.equidistant(33, 8)
    assert len(ea) == len(ico) == 4412
    cv = [_density_cv(x) for x in (ea, ico, octa)]
    nn = [_nn_ratio(x) for x in (ea, ico, octa)]
    assert cv[0] < cv[1] < cv[2]
    assert nn[0] < nn[1] < nn[2]
    assert nn[0] < 1.1 and nn[1] > 1.3 and nn[2] > 2.0
