"""Shared comparison helpers for the GPU-vs-oracle parity tests (test code only)."""
import numpy as np

DEG = np.pi / 180.0
# tolerances (the benchmark spec): delays 1e-6 relative, angles 1e-4 degree
TOL_DELAY_REL = 1e-6
TOL_ANGLE_RAD = 1e-4 * DEG
# grazing / edge exclusion margin for per-ray face-sequence parity (rad)
EDGE_MARGIN = 1e-6


def ang(a, b):
    a, b = np.asarray(a, np.float64), np.asarray(b, np.float64)
    return float(np.arctan2(np.linalg.norm(np.cross(a, b)), np.dot(a, b)))


def dir_of(az, el):
    return np.array([np.cos(el) * np.cos(az), np.cos(el) * np.sin(az), np.sin(el)])


def key_of(rec):
    return (int(rec["tx"]), int(rec["rx"]), int(rec["order"]), tuple(int(f) for f in rec["faces"][: rec["order"]]))


def gpu_paths_by_key(recs):
    out = {}
    for r in recs:
        k = key_of(r)
        assert k not in out, f"duplicate path {k}"
        out[k] = r
    return out


def oracle_paths_by_key(paths):
    return {(p["tx"], p["rx"], p["order"], tuple(p["faces"])): p for p in paths}
