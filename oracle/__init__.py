"""FP64 CPU oracle for the SBR hot path of arXiv 2208.10009.

TEST INFRASTRUCTURE ONLY.  This package is the independent reference the CUDA library
is checked against.  Only the test suite, ``__graft_entry__.smoke()`` and ``bench.py``'s
CPU-baseline / reference legs may import it.  It shares no code with the CUDA path: the
arithmetic lives in ``sbr_oracle.c`` (plain C, double precision, brute force), and this
module only marshals arrays and groups records.  The one module both sides use is the
seeded scene generator, which holds none of the method's arithmetic.

Parity status: every function is pinned by the tests under ``tests/``.  Two power terms
rest on readings because the paper gives no formula: the reflection power of
:func:`path_eval` (pinned only by single-plane closed forms: free-space loss, the
normal-incidence Fresnel coefficient, the grazing limit) and the diffraction power of
:func:`wedge_eval` / :func:`wedge_image` (free-space loss only, no diffraction
coefficient; pinned by the unrolled-edge closed form around a single wedge).
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sbr_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_SO = os.path.join(_OUT_DIR, "liboracle.so")
MAX_ORDER = 8
C0 = 299792458.0

_lock = threading.Lock()
_lib = None

_d = ctypes.POINTER(ctypes.c_double)
_i32 = ctypes.POINTER(ctypes.c_int32)
_i64 = ctypes.POINTER(ctypes.c_int64)
_vp = ctypes.c_void_p


def build(force: bool = False) -> str:
    """Compile ``sbr_oracle.c`` with gcc (OpenMP when available) into ``_build/``."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if not force and os.path.exists(_SO) and os.path.getmtime(_SO) >= os.path.getmtime(_SRC):
        return _SO
    base = ["gcc", "-O2", "-std=c11", "-D_DEFAULT_SOURCE", "-fPIC", "-shared", _SRC, "-o", _SO + ".tmp", "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True, capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(_SO + ".tmp", _SO)
    return _SO


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        sig = {
            "ora_theta0": (ctypes.c_double, []),
            "ora_theta_launch": (ctypes.c_double, [ctypes.c_int]),
            "ora_num_rays": (ctypes.c_int64, [ctypes.c_int]),
            "ora_icosahedron": (None, [_d, _i32, _i32]),
            "ora_lattice": (ctypes.c_int64, [ctypes.c_int, _d]),
            "ora_lattice_ids": (None, [ctypes.c_int, _i64, ctypes.c_int64, _d]),
            "ora_face_points": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, _d, _i32, _i32]),
            "ora_subray_pattern": (ctypes.c_int, [ctypes.c_int, _d, _d, _d]),
            "ora_scene_new": (_vp, [_d, ctypes.c_int64, _i32, _i32, ctypes.c_int64, _d, ctypes.c_int32]),
            "ora_scene_free": (None, [_vp]),
            "ora_scene_face_plane": (None, [_vp, ctypes.c_int, _d]),
            "ora_scene_scale": (ctypes.c_double, [_vp]),
            "ora_trace": (ctypes.c_int64, [_vp, _d, _d, _i64, ctypes.c_int64, _d, ctypes.c_int32,
                                           ctypes.c_int32, ctypes.c_double, ctypes.c_int32,
                                           _i32, _i32, _d, ctypes.c_int64, _i32, _i64, _i32, _i32,
                                           _d, _d, _i64]),
            "ora_refine": (ctypes.c_int, [_vp, _d, _d, ctypes.c_int, _i32, _d, ctypes.c_double, ctypes.c_int,
                                          ctypes.c_int, ctypes.c_double, _d, _d, _i32, _d]),
            "ora_refine_ex": (ctypes.c_int, [_vp, _d, _d, ctypes.c_int, _i32, _d, ctypes.c_double, ctypes.c_int,
                                             ctypes.c_int, ctypes.c_double, _i32, ctypes.c_int, _d, _d, _i32, _d,
                                             _d, _i32, _d]),
            "ora_path_eval": (ctypes.c_int, [_vp, _d, _d, ctypes.c_int, _i32, _d, ctypes.c_double,
                                             ctypes.c_double, ctypes.c_double, _d, _i32, _d, _d, _d, _d, _d]),
            "ora_image_path": (ctypes.c_int, [_vp, _d, _d, ctypes.c_int, _i32, ctypes.c_double,
                                              ctypes.c_double, _d, _d, _d, _d, _d, _d]),
            "ora_image_enumerate": (ctypes.c_int64, [_vp, _d, _d, ctypes.c_int, ctypes.c_int64, _i32, _i32,
                                                     _d, _d]),
            "ora_unfold": (None, [_vp, ctypes.c_int, _i32, _d, _d, ctypes.c_double, ctypes.c_double, _d, _d]),
            "ora_num_threads": (ctypes.c_int, []),
            "ora_unfold_many": (None, [_vp, ctypes.c_int64, _i32, _i32, _d, _d, _d]),
            "ora_path_errors": (None, [_vp, _d, _d, ctypes.c_int, _i32, _d, _d]),
            "ora_equidistant": (ctypes.c_int64, [ctypes.c_int, ctypes.c_int, _d]),
            "ora_wedges": (ctypes.c_int32, [_vp, _d, _i32]),
            "ora_wedge_exterior": (ctypes.c_int32, [_vp, ctypes.c_int32, _d]),
            "ora_diffract": (ctypes.c_int64, [_vp, _d, _d, _i64, ctypes.c_int64, _d, ctypes.c_int32,
                                              ctypes.c_double, ctypes.c_int64, _i32, _i64, _i32, _d, _d]),
            "ora_refine_wedge": (ctypes.c_int, [_vp, _d, _d, ctypes.c_int32, _d, ctypes.c_double, ctypes.c_int,
                                                ctypes.c_int, ctypes.c_double, _d, _d, _i32, _d]),
            "ora_wedge_eval": (ctypes.c_int, [_vp, _d, _d, ctypes.c_int32, _d, ctypes.c_double, ctypes.c_double,
                                              ctypes.c_double, _d, _i32, _d, _d, _d, _d, _d]),
            "ora_wedge_image": (ctypes.c_int, [_vp, _d, _d, ctypes.c_int32, ctypes.c_double, ctypes.c_double,
                                               _d, _d, _d, _d, _d, _d]),
        }
        for name, (res, args) in sig.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
        return lib


def _p(a, t=_d):
    return None if a is None else a.ctypes.data_as(t)


def _f64(a, shape=None):
    a = np.ascontiguousarray(np.asarray(a, dtype=np.float64))
    return a if shape is None else a.reshape(shape)


def num_threads() -> int:
    return _load().ora_num_threads()


# ----------------------------------------------------------------------------- lattice
def theta0() -> float:
    return _load().ora_theta0()


def theta_launch(n: int) -> float:
    return _load().ora_theta_launch(n)


def num_rays(n: int) -> int:
    return _load().ora_num_rays(n)


def icosahedron():
    v = np.zeros((12, 3))
    f = np.zeros((20, 3), np.int32)
    e = np.zeros((30, 2), np.int32)
    _load().ora_icosahedron(_p(v), _p(f, _i32), _p(e, _i32))
    return v, f, e


def lattice(n: int) -> np.ndarray:
    out = np.zeros((num_rays(n), 3))
    _load().ora_lattice(n, _p(out))
    return out


def equidistant(n: int, poly: int = 20) -> np.ndarray:
    """Equidistant division on the icosahedron (poly = 20) or octahedron (poly = 8)."""
    N = (10 if poly == 20 else 4) * n * n + 2
    out = np.zeros((N, 3))
    c = _load().ora_equidistant(n, poly, _p(out))
    if c != N:
        raise ValueError("unknown polyhedron")
    return out


def lattice_ids(n: int, ids) -> np.ndarray:
    ids = np.ascontiguousarray(np.asarray(ids, dtype=np.int64))
    out = np.zeros((len(ids), 3))
    _load().ora_lattice_ids(n, _p(ids, _i64), len(ids), _p(out))
    return out


def face_points(n: int, f: int):
    cnt = (n + 1) * (n + 2) // 2
    pts = np.zeros((cnt, 3))
    la = np.zeros(cnt, np.int32)
    ix = np.zeros(cnt, np.int32)
    c = _load().ora_face_points(n, f, _p(pts), _p(la, _i32), _p(ix, _i32))
    return pts[:c], la[:c], ix[:c]


def subray_pattern(K: int):
    rho = np.zeros(16)
    phi = np.zeros(16)
    s = np.zeros(1)
    k = _load().ora_subray_pattern(K, _p(rho), _p(phi), _p(s))
    if k != K:
        raise ValueError(f"no sub-ray pattern for K={K}")
    return rho[:K], phi[:K], float(s[0])


# ----------------------------------------------------------------------------- scene
class Scene:
    """A triangle scene: vertices (V,3), triangles (T,3), per-triangle face id, and an
    optional relative permittivity per face (<= 0 or None: perfect reflector)."""

    def __init__(self, verts, tris, tri_face, face_eps=None, nf=None):
        self.verts = _f64(verts, (-1, 3))
        self.tris = np.ascontiguousarray(np.asarray(tris, np.int32).reshape(-1, 3))
        self.tri_face = np.ascontiguousarray(np.asarray(tri_face, np.int32).reshape(-1))
        self.nf = int(nf if nf is not None else (self.tri_face.max() + 1 if len(self.tri_face) else 0))
        self.face_eps = None if face_eps is None else _f64(face_eps)
        self._h = _load().ora_scene_new(_p(self.verts), len(self.verts), _p(self.tris, _i32),
                                        _p(self.tri_face, _i32), len(self.tris), _p(self.face_eps), self.nf)

    @classmethod
    def from_generated(cls, sc):
        return cls(sc.verts, sc.tris, sc.tri_face, sc.face_eps, sc.nf)

    @property
    def handle(self):
        return self._h

    def plane(self, f: int) -> np.ndarray:
        out = np.zeros(4)
        _load().ora_scene_face_plane(self._h, f, _p(out))
        return out

    @property
    def scale(self) -> float:
        return _load().ora_scene_scale(self._h)

    def close(self):
        if self._h:
            _load().ora_scene_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


# ----------------------------------------------------------------------------- tracing
@dataclass
class TraceResult:
    rec_rx: np.ndarray
    rec_ray: np.ndarray
    rec_order: np.ndarray
    rec_faces: np.ndarray
    rec_err: np.ndarray
    rec_dray: np.ndarray
    ray_nseg: np.ndarray
    ray_faces: np.ndarray
    ray_margin: np.ndarray
    nsegments: int


def trace(scene: Scene, tx, dirs, rx, max_order: int, cone: float, ray_ids=None, want_margin=False,
          cap=None) -> TraceResult:
    """Brute-force SBR trace from one Tx (see ``ora_trace``)."""
    lib = _load()
    tx = _f64(tx, (3,))
    dirs = _f64(dirs, (-1, 3))
    rx = _f64(rx, (-1, 3))
    n = len(dirs)
    ids = None if ray_ids is None else np.ascontiguousarray(np.asarray(ray_ids, np.int64))
    nseg = np.zeros(n, np.int32)
    rfaces = np.zeros((n, max_order + 1), np.int32)
    margin = np.zeros(n)
    cap = cap or max(1024, 4 * n)
    while True:
        r_rx = np.zeros(cap, np.int32)
        r_ray = np.zeros(cap, np.int64)
        r_ord = np.zeros(cap, np.int32)
        r_fac = np.zeros((cap, MAX_ORDER), np.int32)
        r_err = np.zeros(cap)
        r_dr = np.zeros(cap)
        nsegs = np.zeros(1, np.int64)
        cnt = lib.ora_trace(scene.handle, _p(tx), _p(dirs), _p(ids, _i64), n, _p(rx), len(rx), max_order,
                            cone, int(want_margin), _p(nseg, _i32), _p(rfaces, _i32), _p(margin), cap,
                            _p(r_rx, _i32), _p(r_ray, _i64), _p(r_ord, _i32), _p(r_fac, _i32), _p(r_err),
                            _p(r_dr), _p(nsegs, _i64))
        if cnt <= cap:
            break
        cap = int(cnt) + 16
    c = int(cnt)
    return TraceResult(r_rx[:c], r_ray[:c], r_ord[:c], r_fac[:c], r_err[:c], r_dr[:c], nseg, rfaces, margin,
                       int(nsegs[0]))


def dedup(tr: TraceResult, tx_id: int = 0):
    """Double-count removal (§III.A, first path test): among records with the same
    (Tx, Rx, face sequence), keep the one with the smallest error angle (Eq. 3); ties go
    to the lowest ray id.  Returns a list of dicts sorted by (tx, rx, order, faces)."""
    best = {}
    for i in range(len(tr.rec_err)):
        k = int(tr.rec_order[i])
        key = (tx_id, int(tr.rec_rx[i]), k, tuple(int(f) for f in tr.rec_faces[i, :k]))
        cand = (float(tr.rec_err[i]), int(tr.rec_ray[i]), float(tr.rec_dray[i]))
        if key not in best or cand[:2] < best[key][:2]:
            best[key] = cand
    out = []
    for key in sorted(best):
        err, ray, dray = best[key]
        out.append(dict(tx=key[0], rx=key[1], order=key[2], faces=key[3], err=err, ray=ray, dray=dray))
    return out


def _faces_arr(faces):
    a = np.full(MAX_ORDER, -1, np.int32)
    a[: len(faces)] = faces
    return a


def refine(scene: Scene, tx, rx, faces, c0, R0: float, K: int, iters: int, target: float = 0.0):
    """The iterative precise algorithm for one path (see ``ora_refine``)."""
    fa = _faces_arr(faces)
    out_dir = np.zeros(3)
    out_err = np.zeros(1)
    choice = np.full(max(iters, 1), -1, np.int32)
    hist = np.full(iters + 1, np.nan)
    it = _load().ora_refine(scene.handle, _p(_f64(tx, (3,))), _p(_f64(rx, (3,))), len(faces), _p(fa, _i32),
                            _p(_f64(c0, (3,))), R0, K, iters, target, _p(out_dir), _p(out_err),
                            _p(choice, _i32), _p(hist))
    if it < 0:
        raise ValueError("bad sub-ray count")
    return dict(dir=out_dir, err=float(out_err[0]), iters=it, choice=choice[:it], err_hist=hist[: it + 1])


def refine_ex(scene: Scene, tx, rx, faces, c0, R0: float, K: int, iters: int, target: float = 0.0, forced=None,
              stall: bool = True):
    """``refine`` with the test hooks of ``ora_refine_ex``: ``forced`` (per iteration the
    sub-ray index in bits 0-3 and the frame axis in bits 4-5, or -1 for the argmin and the
    frame rule) replays another implementation's logged choices; the result adds
    ``sub_err`` (iterations x K: every sub-ray's error angle per iteration), ``axis`` (the
    frame axis the rule picks at each iteration's centre) and ``centre`` (each iteration's
    cone centre).  ``stall=False`` disables the stalled-path exit."""
    fa = _faces_arr(faces)
    out_dir = np.zeros(3)
    out_err = np.zeros(1)
    n = max(iters, 1)
    choice = np.full(n, -1, np.int32)
    hist = np.full(iters + 1, np.nan)
    sub = np.full((n, K), np.nan)
    fz = None
    if forced is not None:
        fz = np.full(n, -1, np.int32)
        f = np.asarray(forced, np.int32)[:n]
        fz[: len(f)] = f
    axis = np.full(n, -1, np.int32)
    centre = np.full((n, 3), np.nan)
    it = _load().ora_refine_ex(scene.handle, _p(_f64(tx, (3,))), _p(_f64(rx, (3,))), len(faces), _p(fa, _i32),
                               _p(_f64(c0, (3,))), R0, K, iters, target, _p(fz, _i32), int(stall), _p(out_dir),
                               _p(out_err), _p(choice, _i32), _p(hist), _p(sub), _p(axis, _i32), _p(centre))
    if it < 0:
        raise ValueError("bad sub-ray count")
    return dict(dir=out_dir, err=float(out_err[0]), iters=it, choice=choice[:it], err_hist=hist[: it + 1],
                sub_err=sub[:it], axis=axis[:it], centre=centre[:it])


def path_errors(scene: Scene, tx, rx, faces, direction):
    """(AOD error, AOA error) of a reflection path launched along ``direction``: the two
    quantities the precise algorithm's early stop compares with its target."""
    fa = _faces_arr(faces)
    out = np.zeros(2)
    _load().ora_path_errors(scene.handle, _p(_f64(tx, (3,))), _p(_f64(rx, (3,))), len(faces), _p(fa, _i32),
                            _p(_f64(direction, (3,))), _p(out))
    return float(out[0]), float(out[1])


def refined_err_bound(R0: float, K: int, iters: int) -> float:
    """Twice the Eq. 10 bound after ``iters`` iterations plus the FP32 evaluation floor: the
    error angle a refined path must not exceed to count as converged."""
    _, _, s = subray_pattern(K)
    return 2.0 * R0 * s ** iters + 1e-7


def path_eval(scene: Scene, tx, rx, faces, direction, freq=2.4e9, ptx_dbm=0.0, err_bound=0.0):
    """Validity test and outputs of one path launched along ``direction`` (err_bound > 0
    adds the convergence condition, see ``ora_path_eval``)."""
    fa = _faces_arr(faces)
    pts = np.zeros((MAX_ORDER, 3))
    valid = np.zeros(1, np.int32)
    delay, power, err = np.zeros(1), np.zeros(1), np.zeros(1)
    aod, aoa = np.zeros(2), np.zeros(2)
    r = _load().ora_path_eval(scene.handle, _p(_f64(tx, (3,))), _p(_f64(rx, (3,))), len(faces), _p(fa, _i32),
                              _p(_f64(direction, (3,))), freq, ptx_dbm, err_bound, _p(pts), _p(valid, _i32),
                              _p(delay),
                              _p(aod), _p(aoa), _p(power), _p(err))
    return dict(ok=(r == 0), valid=bool(valid[0]), points=pts[: len(faces)], delay=float(delay[0]), aod=aod,
                aoa=aoa, power=float(power[0]), err=float(err[0]))


def image_path(scene: Scene, tx, rx, faces, freq=2.4e9, ptx_dbm=0.0):
    """Image-method solution for one face sequence (see ``ora_image_path``)."""
    fa = _faces_arr(faces)
    pts = np.zeros((MAX_ORDER, 3))
    d = np.zeros(3)
    delay, power = np.zeros(1), np.zeros(1)
    aod, aoa = np.zeros(2), np.zeros(2)
    r = _load().ora_image_path(scene.handle, _p(_f64(tx, (3,))), _p(_f64(rx, (3,))), len(faces), _p(fa, _i32),
                               freq, ptx_dbm, _p(pts), _p(d), _p(delay), _p(aod), _p(aoa), _p(power))
    return dict(status=r, valid=(r == 1), points=pts[: len(faces)], aod_dir=d, delay=float(delay[0]), aod=aod,
                aoa=aoa, power=float(power[0]))


def image_enumerate(scene: Scene, tx, rx, max_order: int, cap: int = 1 << 16):
    """All valid image-method paths up to ``max_order`` (exhaustive; small scenes)."""
    order = np.zeros(cap, np.int32)
    faces = np.zeros((cap, MAX_ORDER), np.int32)
    dirs = np.zeros((cap, 3))
    delay = np.zeros(cap)
    c = _load().ora_image_enumerate(scene.handle, _p(_f64(tx, (3,))), _p(_f64(rx, (3,))), max_order, cap,
                                    _p(order, _i32), _p(faces, _i32), _p(dirs), _p(delay))
    c = min(int(c), cap)
    return [dict(order=int(order[i]), faces=tuple(int(f) for f in faces[i, : order[i]]), aod_dir=dirs[i],
                 delay=float(delay[i])) for i in range(c)]


def unfold(scene: Scene, faces, tx, rx, az: float, el: float):
    """Fixed-face-sequence unfolding values (miss[3], delay, AOD az/el, AOA az/el) and
    their closed-form Jacobian w.r.t. (az, el, Tx, Rx)."""
    fa = _faces_arr(faces)
    val = np.zeros(8)
    J = np.zeros((8, 8))
    _load().ora_unfold(scene.handle, len(faces), _p(fa, _i32), _p(_f64(tx, (3,))), _p(_f64(rx, (3,))),
                       float(az), float(el), _p(val), _p(J))
    return val, J


def unfold_many(scene: Scene, order, faces, tx, rx) -> np.ndarray:
    """``unfold`` values (miss[3] at az = el = 0, delay, AOD az/el, AOA az/el) of many
    reflection paths: order (P,), faces (P, 8) -1 padded, tx / rx (P, 3)."""
    order = np.ascontiguousarray(np.asarray(order, np.int32))
    faces = np.ascontiguousarray(np.asarray(faces, np.int32).reshape(-1, MAX_ORDER))
    tx, rx = _f64(tx, (-1, 3)), _f64(rx, (-1, 3))
    out = np.zeros((len(order), 8))
    _load().ora_unfold_many(scene.handle, len(order), _p(order, _i32), _p(faces, _i32), _p(tx), _p(rx), _p(out))
    return out


def az_el(v):
    v = np.asarray(v, np.float64)
    return np.arctan2(v[..., 1], v[..., 0]), np.arctan2(v[..., 2], np.hypot(v[..., 0], v[..., 1]))


# ----------------------------------------------------------------------------- diffraction
def wedges(scene: Scene):
    """Wedges of the scene (see ``wedges_build``): endpoints (W, 2, 3) and face pairs (W, 2)."""
    lib = _load()
    n = lib.ora_wedges(scene.handle, None, None)
    ab = np.zeros((max(n, 1), 6))
    fc = np.zeros((max(n, 1), 2), np.int32)
    lib.ora_wedges(scene.handle, _p(ab), _p(fc, _i32))
    return ab[:n].reshape(-1, 2, 3), fc[:n]


def wedge_exterior(scene: Scene, w: int, p) -> bool:
    return bool(_load().ora_wedge_exterior(scene.handle, int(w), _p(_f64(p, (3,)))))


@dataclass
class DiffractResult:
    rec_rx: np.ndarray
    rec_ray: np.ndarray
    rec_wedge: np.ndarray
    rec_err: np.ndarray
    rec_dray: np.ndarray


def diffract(scene: Scene, tx, dirs, rx, cone: float, ray_ids=None, cap=None) -> DiffractResult:
    """Brute-force rough order-1 diffraction search from one Tx (see ``ora_diffract``);
    records sorted by (ray, wedge, rx)."""
    lib = _load()
    tx = _f64(tx, (3,))
    dirs = _f64(dirs, (-1, 3))
    rx = _f64(rx, (-1, 3))
    ids = None if ray_ids is None else np.ascontiguousarray(np.asarray(ray_ids, np.int64))
    cap = cap or max(1024, len(dirs))
    while True:
        r_rx = np.zeros(cap, np.int32)
        r_ray = np.zeros(cap, np.int64)
        r_w = np.zeros(cap, np.int32)
        r_err = np.zeros(cap)
        r_dr = np.zeros(cap)
        cnt = lib.ora_diffract(scene.handle, _p(tx), _p(dirs), _p(ids, _i64), len(dirs), _p(rx), len(rx), cone, cap,
                               _p(r_rx, _i32), _p(r_ray, _i64), _p(r_w, _i32), _p(r_err), _p(r_dr))
        if cnt <= cap:
            break
        cap = int(cnt) + 16
    c = int(cnt)
    o = np.lexsort((r_rx[:c], r_w[:c], r_ray[:c]))
    return DiffractResult(r_rx[:c][o], r_ray[:c][o], r_w[:c][o], r_err[:c][o], r_dr[:c][o])


def dedup_wedge(dr: DiffractResult, tx_id: int = 0):
    """Double-count removal for diffraction records: one path per (Tx, Rx, wedge), the
    smallest error angle, ties to the lowest ray id."""
    best = {}
    for i in range(len(dr.rec_err)):
        key = (tx_id, int(dr.rec_rx[i]), int(dr.rec_wedge[i]))
        cand = (float(dr.rec_err[i]), int(dr.rec_ray[i]), float(dr.rec_dray[i]))
        if key not in best or cand[:2] < best[key][:2]:
            best[key] = cand
    return [dict(tx=k[0], rx=k[1], wedge=k[2], order=1, faces=(-1 - k[2],), err=v[0], ray=v[1], dray=v[2],
                 diffraction=True) for k, v in sorted(best.items())]


def refine_wedge(scene: Scene, tx, rx, w: int, c0, R0: float, K: int, iters: int, target: float = 0.0):
    """The precise algorithm for a diffraction path (see ``ora_refine_wedge``)."""
    out_dir = np.zeros(3)
    out_err = np.zeros(1)
    choice = np.full(max(iters, 1), -1, np.int32)
    hist = np.full(iters + 1, np.nan)
    it = _load().ora_refine_wedge(scene.handle, _p(_f64(tx, (3,))), _p(_f64(rx, (3,))), int(w),
                                  _p(_f64(c0, (3,))), R0, K, iters, target, _p(out_dir), _p(out_err),
                                  _p(choice, _i32), _p(hist))
    if it < 0:
        raise ValueError("bad sub-ray count or Tx on the edge line")
    return dict(dir=out_dir, err=float(out_err[0]), iters=it, choice=choice[:it], err_hist=hist[: it + 1])


def wedge_eval(scene: Scene, tx, rx, w: int, direction, freq=2.4e9, ptx_dbm=0.0, err_bound=0.0):
    """Validity test and outputs of a diffraction path (see ``ora_wedge_eval``)."""
    q = np.zeros(3)
    valid = np.zeros(1, np.int32)
    delay, power, err = np.zeros(1), np.zeros(1), np.zeros(1)
    aod, aoa = np.zeros(2), np.zeros(2)
    r = _load().ora_wedge_eval(scene.handle, _p(_f64(tx, (3,))), _p(_f64(rx, (3,))), int(w),
                               _p(_f64(direction, (3,))), freq, ptx_dbm, err_bound, _p(q), _p(valid, _i32),
                               _p(delay), _p(aod), _p(aoa), _p(power), _p(err))
    return dict(ok=(r == 0), valid=bool(valid[0]), point=q, delay=float(delay[0]), aod=aod, aoa=aoa,
                power=float(power[0]), err=float(err[0]))


def wedge_image(scene: Scene, tx, rx, w: int, freq=2.4e9, ptx_dbm=0.0):
    """Exact order-1 diffraction path at wedge w (see ``ora_wedge_image``)."""
    q, d = np.zeros(3), np.zeros(3)
    delay, power = np.zeros(1), np.zeros(1)
    aod, aoa = np.zeros(2), np.zeros(2)
    r = _load().ora_wedge_image(scene.handle, _p(_f64(tx, (3,))), _p(_f64(rx, (3,))), int(w), freq, ptx_dbm,
                                _p(q), _p(d), _p(delay), _p(aod), _p(aoa), _p(power))
    return dict(status=r, valid=(r == 1), point=q, aod_dir=d, delay=float(delay[0]), aod=aod, aoa=aoa,
                power=float(power[0]))


def wedge_enumerate(scene: Scene, tx, rx):
    """Every valid exact order-1 diffraction path from tx to rx: {wedge: wedge_image dict}."""
    nw = len(wedges(scene)[1])
    out = {}
    for w in range(nw):
        r = wedge_image(scene, tx, rx, w)
        if r["valid"]:
            out[w] = r
    return out


# ----------------------------------------------------------------------------- pipeline
@dataclass
class PipelineResult:
    paths: list
    nsegments: int
    nrays: int
    nrecords: int
    traces: list = field(default_factory=list)


def sbr_pipeline(scene: Scene, txs, rxs, n: int, max_order: int, alpha: float, K: int, iters: int,
                 target: float = 0.0, ray_ids=None, want_margin=False, freq=2.4e9, keep_traces=False,
                 refine_paths=True, launcher: int = 0, diffraction: bool = False):
    """The whole hot path in the paper's order (Fig. 4): equiangular launch, brute-force
    trace with reception, double-count removal, the precise algorithm, then the validity
    test and outputs.  The reception cone is alpha * theta_launch; the precise algorithm's
    initial cone is the ray cone of Eq. 8, theta_launch, widened to the rough error angle
    when that is larger (alpha > 1 can accept a ray outside its own cone), so the exact
    direction is always inside it.  ``ray_ids`` restricts the launch to a subsample of the
    lattice.  ``diffraction`` adds the order-1 diffraction paths (one per Tx, Rx, wedge)
    after each Tx's reflection paths."""
    txs = _f64(txs, (-1, 3))
    rxs = _f64(rxs, (-1, 3))
    cone = alpha * theta_launch(n)
    all_dirs = equidistant(n, launcher) if launcher else None
    if ray_ids is None:
        dirs = lattice(n) if not launcher else all_dirs
        ids = None
    else:
        ids = np.asarray(ray_ids, np.int64)
        dirs = lattice_ids(n, ids) if not launcher else all_dirs[ids]
    paths, traces = [], []
    nseg = nrec = 0
    for t, tx in enumerate(txs):
        tr = trace(scene, tx, dirs, rxs, max_order, cone, ray_ids=ids, want_margin=want_margin)
        nseg += tr.nsegments
        nrec += len(tr.rec_err)
        if keep_traces:
            traces.append(tr)
        for p in dedup(tr, t):
            c0 = lattice_ids(n, [p["ray"]])[0] if not launcher else all_dirs[p["ray"]]
            p["rough_dir"] = c0
            if refine_paths:
                R0 = max(theta_launch(n), p["err"])
                r = refine(scene, tx, rxs[p["rx"]], p["faces"], c0, R0, K, iters, target)
                p.update(ref_dir=r["dir"], ref_err=r["err"], iters=r["iters"], choice=r["choice"],
                         err_hist=r["err_hist"])
                bound = refined_err_bound(R0, K, r["iters"]) if r["iters"] > 0 else 0.0
                ev = path_eval(scene, tx, rxs[p["rx"]], p["faces"], r["dir"], freq, err_bound=bound)
                p.update(valid=ev["valid"], delay=ev["delay"], aod=ev["aod"], aoa=ev["aoa"], power=ev["power"],
                         points=ev["points"])
            paths.append(p)
        if not diffraction:
            continue
        dr = diffract(scene, tx, dirs, rxs, cone, ray_ids=ids)
        nrec += len(dr.rec_err)
        for p in dedup_wedge(dr, t):
            c0 = lattice_ids(n, [p["ray"]])[0] if not launcher else all_dirs[p["ray"]]
            p["rough_dir"] = c0
            if refine_paths:
                R0 = max(theta_launch(n), p["err"])
                r = refine_wedge(scene, tx, rxs[p["rx"]], p["wedge"], c0, R0, K, iters, target)
                p.update(ref_dir=r["dir"], ref_err=r["err"], iters=r["iters"], choice=r["choice"],
                         err_hist=r["err_hist"])
                bound = refined_err_bound(R0, K, r["iters"]) if r["iters"] > 0 else 0.0
                ev = wedge_eval(scene, tx, rxs[p["rx"]], p["wedge"], r["dir"], freq, err_bound=bound)
                p.update(valid=ev["valid"], delay=ev["delay"], aod=ev["aod"], aoa=ev["aoa"], power=ev["power"],
                         points=ev["point"][None, :])
            paths.append(p)
    return PipelineResult(paths, nseg, len(dirs) * len(txs), nrec, traces)
