"""Shared comparison helpers for the GPU-vs-oracle parity tests (test code only)."""
import numpy as np

DEG = np.pi / 180.0
# parity tolerances of the GPU path against the oracle: delays 1e-6 relative, angles 1e-4 degree
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


def in_key_order(recs, *aligned):
    """Query output sorted by path key (Tx, Rx, order, face sequence), with arrays aligned to
    it (e.g. the choice log, indexed like the records) reordered the same way.  The order of
    sbr_query's output follows the double-count removal's atomics and varies from run to
    run; a test that samples from it by position samples the same paths only in key order."""
    o = np.lexsort(tuple(recs["faces"][:, j] for j in range(recs["faces"].shape[1] - 1, -1, -1)) +
                   (recs["order"], recs["rx"], recs["tx"]))
    return (recs[o],) + tuple(a[: len(recs)][o] for a in aligned)


def oracle_paths_by_key(paths):
    return {(p["tx"], p["rx"], p["order"], tuple(p["faces"])): p for p in paths}


# ----------------------------------------------------------------------------- refinement
U32 = 2.0 ** -24          # FP32 unit roundoff
PATH_TRACE_FAIL, PATH_STALLED = 4, 16


def replay_refinement(oracle_mod, S, tx, rx, faces, c0, R0, K, rec, log, cap, target=0.0, fp64_below=1e-5):
    """Check one GPU-refined path decision by decision against the oracle (§III.B).

    The oracle replays the GPU's logged decisions (argmin sub-ray and frame axis of every
    iteration) in FP64, so each decision is judged on the cone the GPU actually had:
      - the GPU's final direction equals the replay's within 1e-4 deg: the arithmetic
        along the same decisions agrees;
      - every decision is the oracle's own for that cone, or a tie within the GPU's
        rounding.  With u = 2^-24 and D = 4 max(drift, u) (drift = the final angle between
        the GPU's and the replay's direction: how far rounding has moved the GPU's centre),
        the chosen sub-ray's FP64 error may exceed the best one's by at most 6 u + 2 D in an
        FP32 iteration (each sub-ray's error is evaluated within 3 u) and 2 D + 1e-12 R in
        an FP64 one; a different frame axis needs the two candidate |c_i| within 4 u + D;
      - the stop: a path that stopped before the cap met the target (AOD and AOA errors)
        at its last iteration and not one iteration earlier, a stalled path had left the
        stall bound, a path at the cap never met the target earlier -- each within the
        same rounding (AOA errors with up to 50x amplification of it).
    Returns dict(drift, ties, axis_ties, max_gap) for reporting."""
    it = int(rec["iters"])
    forced = np.asarray(log[:it], np.int32)
    rep = oracle_mod.refine_ex(S, tx, rx, faces, c0, R0, K, it, forced=forced, stall=False)
    assert rep["iters"] == it, ("replay ended early: a logged sub-ray is invalid in FP64", faces, it, rep["iters"])
    drift = ang(rec["dir"], rep["dir"])
    assert drift < TOL_ANGLE_RAD, ("GPU state differs from the replay of its own decisions", faces, drift)
    _, _, s = oracle_mod.subray_pattern(K)
    D = 4.0 * max(drift, U32)
    ties = axis_ties = 0
    max_gap = 0.0
    for i in range(it):
        R = R0 * s ** i
        k, axis = int(forced[i]) & 15, (int(forced[i]) >> 4) & 3
        fp64 = R < fp64_below
        if axis != rep["axis"][i]:
            c = np.abs(rep["centre"][i])
            tol = (2 * D + 1e-15) if fp64 else (4 * U32 + D)
            assert abs(c[axis] - c[rep["axis"][i]]) <= tol, ("frame axis differs without a tie", faces, i, c, axis)
            axis_ties += 1
        e = rep["sub_err"][i]
        gap = float(e[k] - np.min(e))
        tol = (2 * D + 1e-12 * R) if fp64 else (6 * U32 + 2 * D)
        assert gap <= tol, ("argmin differs beyond rounding", faces, i, gap, tol, e.tolist(), k)
        ties += gap > 0
        max_gap = max(max_gap, gap)
    flags = int(rec["flags"])
    tolA = 50.0 * (6 * U32 + 2 * D)

    def errs(j):   # AOD / AOA errors of the replay's state after j iterations
        d = rep["centre"][j] if j < it else rep["dir"]
        return oracle_mod.path_errors(S, tx, rx, faces, d)

    def reached(j, slack):
        a, b = errs(j)
        t_a = target * (1 + slack * 1e-4) + slack * (6 * U32 + 2 * D)
        t_b = target * (1 + slack * 1e-2) + slack * tolA
        return a <= t_a and (len(faces) == 0 or b <= t_b)

    if flags & PATH_TRACE_FAIL:
        nxt = oracle_mod.refine_ex(S, tx, rx, faces, c0, R0, K, it + 1, forced=list(forced) + [-1], stall=False)
        assert nxt["iters"] == it, ("GPU found every sub-ray invalid, the oracle did not", faces, it)
    elif flags & PATH_STALLED:
        R = R0 * s ** it
        stall = 1.0 / (1.0 - s) + 2.0 * s
        assert rep["err_hist"][it] > R * stall + 1e-6 - (6 * U32 + 2 * D), ("stall exit without a stall", faces)
    elif target > 0:
        if it < cap:
            assert reached(it, +1), ("stopped before the target was met", faces, it, errs(it))
        for j in range(it):
            assert not reached(j, -1), ("the target was met earlier", faces, j, errs(j))
    else:
        assert it == cap
    return dict(drift=drift, ties=ties, axis_ties=axis_ties, max_gap=max_gap)
