"""GPU test of sbr_dedup_noalloc, the entry point for callers that cannot let the library
allocate device memory (e.g. processes whose device memory is reserved by another
framework's pool).

It is called straight through the C ABI and must reproduce the double-count removal that
sbr_launch performed on the same reception records, on two calls in a row (the fixed
scratch array keeps the previous call's contents, so each call has to clear it), without
requesting memory from the context's allocator.  This file sorts last so that a run that
stops at the first failure has run every other test already."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2208_10009_gb300 import _binding as B
from paper_2208_10009_gb300 import api, scenes

pytestmark = pytest.mark.gpu


def _by_key(recs):
    return {(int(r["tx"]), int(r["rx"]), int(r["order"]), tuple(int(f) for f in r["faces"][: r["order"]])): r
            for r in recs}


def test_dedup_noalloc_matches_launch():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    ctx = api.Context(0)

    sc, tx, rx = scenes.shoebox_config()
    scene = ctx.scene_from(sc)
    rxs = ctx.rx_upload(rx)
    paths = ctx.paths_create(1 << 16, 1 << 12)
    ctx.launch(scene, tx, rxs, paths, 64, 3, rx_angle_scale=float(np.sqrt(3.0)), sync=True)
    want = _by_key(ctx.query(paths))
    assert len(want) == 63

    cap = 256
    out = torch.zeros(cap * 128, dtype=torch.uint8, device="cuda")
    counts = torch.full((2,), -1, dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    before = torch.cuda.memory_allocated()
    for _ in range(2):
        out.zero_()
        st = ctx.lib.sbr_dedup_noalloc(ctx.handle, paths.handle, out.data_ptr(), cap, counts.data_ptr())
        assert st == 0, ctx.lib.sbr_last_error(ctx.handle)
        torch.cuda.synchronize()
        n, collisions = (int(v) for v in counts.cpu())
        assert collisions == 0 and n == len(want)
        got = _by_key(out.cpu().numpy().view(B.PATH_DTYPE)[:n])
        assert set(got) == set(want)
        for k, r in got.items():
            w = want[k]
            assert int(r["ray"]) == int(w["ray"])
            assert r["rough_err"] == w["rough_err"] and r["rough_dray"] == w["rough_dray"]
            assert np.array_equal(r["dir"], w["dir"])
    assert torch.cuda.memory_allocated() == before

    # a launch with more records (the canyon's ~1.5k: a larger part of the table in use),
    # right after the shoebox's calls, at the largest accepted record capacity
    sc2, tx2, rx2 = scenes.urban_canyon()
    scene2 = ctx.scene_from(sc2)
    rxs2 = ctx.rx_upload(rx2)
    paths2 = ctx.paths_create(131072, 1 << 14)
    ctx.launch(scene2, tx2, rxs2, paths2, 700, 6, rx_angle_scale=float(np.sqrt(3.0)), sync=True)
    want2 = _by_key(ctx.query(paths2))
    assert len(want2) > 300
    out2 = torch.zeros((1 << 14) * 128, dtype=torch.uint8, device="cuda")
    for _ in range(2):
        st = ctx.lib.sbr_dedup_noalloc(ctx.handle, paths2.handle, out2.data_ptr(), 1 << 14, counts.data_ptr())
        assert st == 0, ctx.lib.sbr_last_error(ctx.handle)
        torch.cuda.synchronize()
        n, collisions = (int(v) for v in counts.cpu())
        assert collisions == 0 and n == len(want2)
        got = _by_key(out2.cpu().numpy().view(B.PATH_DTYPE)[:n])
        assert set(got) == set(want2)
        assert all(int(got[k]["ray"]) == int(w["ray"]) and got[k]["rough_err"] == w["rough_err"]
                   for k, w in want2.items())
    for h in (paths2, rxs2, scene2):
        h.close()

    # a container larger than the fixed maximum is refused with a clear message
    big = ctx.paths_create(131072 + 1, 16)
    ctx.launch(scene, tx, rxs, big, 8, 1, rx_angle_scale=float(np.sqrt(3.0)), sync=True)
    st = ctx.lib.sbr_dedup_noalloc(ctx.handle, big.handle, out.data_ptr(), cap, counts.data_ptr())
    assert st == 1 and b"exceeds the fixed maximum" in ctx.lib.sbr_last_error(ctx.handle)
    for h in (big, paths, rxs, scene):
        h.close()
    ctx.close()
