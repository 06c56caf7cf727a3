"""CPU tests of the parity helpers' own logic (no GPU)."""
import numpy as np

from paper_2208_10009_gb300 import _binding as B
from parity_util import in_key_order


def test_in_key_order_sorts_by_path_key_and_carries_aligned_arrays():
    rng = np.random.default_rng(3)
    n = 200
    recs = np.zeros(n, dtype=B.PATH_DTYPE)
    recs["tx"] = rng.integers(0, 3, n)
    recs["rx"] = rng.integers(0, 4, n)
    recs["order"] = rng.integers(0, 3, n)
    recs["faces"] = -1
    for i in range(n):
        recs["faces"][i, : recs["order"][i]] = rng.integers(0, 5, recs["order"][i])
    recs["ray"] = np.arange(n)                 # identifies the record after the sort
    log = np.arange(n)[:, None] * 10 + np.arange(4)[None, :]   # one row per record
    got, lg = in_key_order(recs, np.concatenate([log, log[:7]]))
    keys = [(int(r["tx"]), int(r["rx"]), int(r["order"]), tuple(int(f) for f in r["faces"])) for r in got]
    assert keys == sorted(keys)
    assert sorted(got["ray"].tolist()) == list(range(n))
    assert np.array_equal(lg[:, 0] // 10, got["ray"])   # the aligned rows travel with their records
