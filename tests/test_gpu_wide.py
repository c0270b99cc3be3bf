"""128-bit keys (state vectors wider than 64 bits) in the bucket scheme:
parity with the 128-bit oracle set, exactly as for 64-bit keys."""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import keys as wk

from gpu_util import assert_flags_per_key

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


def _pairs(n, seed, start=0, share=None):
    """n distinct 128-bit keys (low, high); share='lo' makes many keys share
    their low word, 'hi' their high word."""
    lo = wk.distinct_keys(n, 64, seed=seed, start=start)
    hi = wk.distinct_keys(n, 64, seed=seed + 1000, start=start)
    if share == "lo":
        lo = lo % np.uint64(7)
    elif share == "hi":
        hi = hi % np.uint64(5)
    return np.stack([lo, hi], axis=1)


def _dev(pairs):
    return torch.from_numpy(np.ascontiguousarray(pairs).view(np.int64)).cuda()


def _ids(pairs):
    """A scalar id per pair for flag-count comparisons."""
    return pairs[:, 0].astype(object) * (1 << 64) + pairs[:, 1].astype(object)


@pytest.mark.parametrize("lanes", [2, 4])
@pytest.mark.parametrize("share", [None, "lo", "hi"])
def test_find_or_put_lookup_export_match_oracle(oracle_lib, lanes, share):
    rng = np.random.default_rng(5)
    n = 120_000
    pool = _pairs(n, seed=40, share=share)
    t = ht.HashTable(int(n / 0.85), "bucket", 128, dict(bucket_slots=8, lanes_per_key=lanes))
    orc = oracle_lib.OracleTable128()
    issued = 0
    while issued < n:
        fresh = pool[issued:issued + 20_000]
        issued += len(fresh)
        rep = pool[rng.integers(0, issued, size=7000)]
        b = np.concatenate([fresh, rep])[rng.permutation(len(fresh) + 7000)]
        got = t.find_or_put(_dev(b)).cpu().numpy()
        exp = orc.find_or_put(b)
        assert_flags_per_key(_ids(b), got, exp)
    assert t.sync() == 0 and t.size() == orc.size() == n
    k, _ = t.export()
    got = set(map(tuple, k.cpu().numpy().view(np.uint64).tolist()))
    assert got == set(map(tuple, orc.export().tolist()))
    absent = _pairs(5000, seed=40, start=n + 10, share=share)
    q = np.concatenate([pool[:5000], absent])
    f, _ = t.lookup(_dev(q))
    np.testing.assert_array_equal(f.cpu().numpy(), orc.lookup(q))


def test_edge_keys_and_reserved(oracle_lib):
    # Words that are all ones except the reserved bit, zeros, and a key with
    # an all-ones low word (a legal key that reads like a half-written slot).
    ones = np.uint64(2 ** 64 - 1)
    top = np.uint64(2 ** 63 - 1)
    keys = np.array([[0, 0], [ones, 0], [0, top], [ones, top], [1, 2], [ones, 0]], dtype=np.uint64)
    t = ht.HashTable(64, "bucket", 128)
    got = t.find_or_put(_dev(keys)).cpu().numpy()
    np.testing.assert_array_equal(got, [1, 1, 1, 1, 1, 0])
    f, _ = t.lookup(_dev(keys))
    assert f.cpu().numpy().all()
    assert t.size() == 5 and t.sync() == 0
    bad = np.array([[3, 2 ** 63]], dtype=np.uint64)                  # reserved bit set
    t.find_or_put(_dev(bad))
    assert t.sync() == 1


def test_overflow_grow_and_full(oracle_lib):
    # A small table spills into its overflow set, reports full beyond it,
    # and growth moves every key to the new storage.
    keys = _pairs(3000, seed=77)
    t = ht.HashTable(64, "bucket", 128, dict(num_hashes=2))
    t.find_or_put(_dev(keys[:600]))
    assert t.sync() == 0 and t.size() == 600
    assert t.stats()["overflow_used"] > 0
    t.grow(8192)
    assert t.size() == 600
    f, _ = t.lookup(_dev(keys[:600]))
    assert f.cpu().numpy().all()
    orc = oracle_lib.OracleTable128()
    orc.find_or_put(keys[:600])
    more = keys[400:3000]
    assert_flags_per_key(_ids(more), t.find_or_put(_dev(more)).cpu().numpy(), orc.find_or_put(more))
    assert t.sync() == 0 and t.size() == 3000
    small = ht.HashTable(8, "bucket", 128, dict(num_hashes=1))
    small.find_or_put(_dev(_pairs(5000, seed=78)))
    assert small.sync() == 3


def test_unsupported_uses_are_rejected():
    with pytest.raises(ht.HtError):
        ht.HashTable(64, "cuckoo", 128)
    with pytest.raises(ht.HtError):
        ht.HashTable(64, "bucket", 128, dict(bucket_slots=16))
