"""CPU checks of the CUDA library's boundary: it builds, loads without a GPU, exports
every entry point declared in include/sbr.h, and its host-only functions agree with the
paper's closed forms."""
import os
import re

import numpy as np
import pytest
from scipy.spatial import cKDTree

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "sbr.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"^[A-Za-z_][\w \*]*?\b(sbr_\w+)\s*\(", src, flags=re.M)))


@pytest.fixture(scope="module")
def lib():
    from paper_2208_10009_gb300 import _binding
    return _binding.load()


def test_exports_every_declared_symbol(lib):
    from paper_2208_10009_gb300 import _binding
    names = _declared()
    assert len(names) >= 28
    for n in names:
        assert hasattr(lib, n), n
        assert n in _binding.SIGNATURES, n


def test_host_functions(lib):
    from paper_2208_10009_gb300 import api
    assert lib.sbr_abi_version() == 3
    assert lib.sbr_status_string(0) == b"ok"
    for n in (1, 2, 21, 64, 700, 2200):
        assert api.num_rays(n) == 10 * n * n + 2
    assert api.num_rays(0) == -1
    th0 = np.arccos(1 / np.sqrt(5))
    for n in (1, 21, 700):
        assert abs(api.theta_launch(n) - th0 / (np.sqrt(3) * n)) < 1e-15


@pytest.mark.parametrize("K", [6, 7, 9, 16])
def test_library_subray_patterns_cover(K):
    """The library's own sub-ray constants cover the cone with their shrink factor."""
    from paper_2208_10009_gb300 import api
    rho, phi, s = api.subray_pattern(K)
    C = np.stack([rho * np.cos(phi), rho * np.sin(phi)], -1)
    rng = np.random.default_rng(100 + K)
    p = rng.uniform(-1, 1, (400000, 2))
    p = p[(p ** 2).sum(1) <= 1]
    t = np.linspace(0, 2 * np.pi, 20000, endpoint=False)
    p = np.vstack([p, np.c_[np.cos(t), np.sin(t)]])
    d, _ = cKDTree(C).query(p)
    assert d.max() <= s * (1 + 1e-9)
    if K == 6:
        assert abs(s - 1 / np.sqrt(3)) < 1e-15


def test_bad_pattern_rejected():
    from paper_2208_10009_gb300 import api
    with pytest.raises(api.SbrError):
        api.subray_pattern(8)


def test_oracle_not_imported_by_product():
    """The product package never imports the oracle."""
    pkg = os.path.join(ROOT, "paper_2208_10009_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cpp", ".h", ".cuh")):
                txt = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in txt and "from oracle" not in txt, f
                assert "sbr_oracle" not in txt, f


def _outline_corners(lib, sc):
    import ctypes
    V = np.ascontiguousarray(np.asarray(sc.verts, np.float32))
    T = np.ascontiguousarray(np.asarray(sc.tris, np.int32))
    F = np.ascontiguousarray(np.asarray(sc.tri_face, np.int32))
    nf = int(F.max()) + 1
    out = np.full(nf, -1, np.int32)
    pf, pi = ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_int32)
    st = lib.sbr_face_outline_corners(V.ctypes.data_as(pf), len(V), T.ctypes.data_as(pi), F.ctypes.data_as(pi),
                                      len(T), nf, out.ctypes.data_as(pi))
    assert st == 0
    return out


def test_face_outline_corners(lib):
    """Host logic of the validity test's point-in-face query (§III.A): a face is tested
    against its convex outline exactly when its triangles tile a convex polygon.  Tiled
    rectangles, a triangle and a convex hexagon qualify with their corner counts; an
    L-shape, a ring around a hole, a bent face, a doubled quad and a flipped triangle keep
    the triangle-by-triangle query."""
    from paper_2208_10009_gb300 import scenes
    b = scenes._Builder()
    scenes.box_faces(b, (0, 0, 0), (2, 3, 4), 3)                     # faces 0-5: 3 x 3 tiled rectangles
    tri = b.polygon([(5, 0, 0), (6, 0, 0), (5, 1, 0.5)])
    ang = np.linspace(0, 2 * np.pi, 7)[:-1]
    hexa = b.polygon(np.c_[10 + np.cos(ang), np.sin(ang), np.zeros(6)])
    ell = b.nf
    b.nf += 1
    for (y0, y1, z0, z1) in ((0, 3, 0, 1.5), (3, 6, 0, 1.5), (0, 3, 1.5, 3)):
        b.quad((20, y0, z0), (20, y1, z0), (20, y0, z1), face=ell)
    ring = b.nf
    b.nf += 1
    for i in range(3):
        for j in range(3):
            if (i, j) != (1, 1):
                b.quad((30 + i, j, 0), (31 + i, j, 0), (30 + i, j + 1, 0), face=ring)
    bent = b.nf
    b.nf += 1
    b.polygon([(40, 0, 0), (41, 0, 0), (41, 1, 0)], face=bent)
    b.polygon([(40, 0, 0), (41, 1, 0), (40, 1, 0.3)], face=bent)
    dup = b.nf
    b.nf += 1
    b.quad((50, 0, 0), (51, 0, 0), (50, 1, 0), face=dup)
    b.quad((50, 0, 0), (51, 0, 0), (50, 1, 0), face=dup)
    flip = b.nf
    b.nf += 1
    b.polygon([(60, 0, 0), (61, 0, 0), (61, 1, 0)], face=flip)
    b.polygon([(60, 0, 0), (60, 1, 0), (61, 1, 0)], face=flip)        # wound against the first
    sc = b.finish()
    c = _outline_corners(lib, sc)
    nbox = tri
    assert np.all(c[:nbox] == 4), c[:nbox]
    assert c[tri] == 3 and c[hexa] == 6
    for f in (ell, ring, bent, dup, flip):
        assert c[f] == 0, (f, c[f])
