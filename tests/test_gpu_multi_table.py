"""ht_multi_find_or_put: many tables, one call.  Results per table equal the
oracle's, whatever mix of schemes, key widths and bucket shapes the call
holds; items naming the same table act as one batch."""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import keys as wk

from gpu_util import assert_flags_per_key, assert_same_set, keys_np, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


def _tables():
    specs = [("bucket", 64, None), ("bucket", 32, None), ("bucket", 64, dict(bucket_slots=8, lanes_per_key=4)),
             ("bucket", 64, dict(bucket_slots=32, lanes_per_key=8)), ("cuckoo", 64, None), ("cuckoo", 32, None),
             ("bucket", 64, None), ("bucket", 32, dict(bucket_slots=8, lanes_per_key=2))]
    return specs, [ht.HashTable(60_000, s, kw, p) for s, kw, p in specs]


def test_many_tables_one_call_match_oracle(oracle_lib):
    rng = np.random.default_rng(4)
    specs, tabs = _tables()
    orcs = [oracle_lib.OracleTable() for _ in tabs]
    issued = [0] * len(tabs)
    for rnd in range(3):
        items, hostk = [], []
        order = rng.permutation(len(tabs))
        for ti in order:
            kw = specs[ti][1]
            n = int(rng.integers(0, 9000))          # includes empty and ragged items
            fresh = wk.distinct_keys(n, kw, seed=300 + int(ti), start=issued[ti])
            if issued[ti] and n:
                old = wk.distinct_keys(issued[ti], kw, seed=300 + int(ti))
                pick = rng.random(n) < 0.3
                fresh[pick] = old[rng.integers(0, issued[ti], size=int(pick.sum()))]
            issued[ti] += n
            k = to_dev(fresh)
            items.append((int(ti), k, torch.empty(n, dtype=torch.uint8, device="cuda")))
            hostk.append(fresh)
        ht.ht_multi_find_or_put([t.handle for t in tabs], items)
        torch.cuda.synchronize()
        for (ti, _, flags), k in zip(items, hostk):
            assert_flags_per_key(k, to_np(flags), orcs[ti].find_or_put(k))
    for t, o, (s, kw, _) in zip(tabs, orcs, specs):
        assert t.sync() == 0 and t.size() == o.size()
        got, _ = t.export()
        assert_same_set(keys_np(got, kw), o.export()[0])
        t.close()


def test_items_on_the_same_table_act_as_one_batch(oracle_lib):
    t = ht.HashTable(100_000, "bucket", 64)
    a = wk.distinct_keys(20_000, 64, seed=41)
    b = np.concatenate([a[:10_000], wk.distinct_keys(5000, 64, seed=42)])
    fa = torch.empty(len(a), dtype=torch.uint8, device="cuda")
    fb = torch.empty(len(b), dtype=torch.uint8, device="cuda")
    ht.ht_multi_find_or_put([t.handle], [(0, to_dev(a), fa), (0, to_dev(b), fb)])
    both = np.concatenate([a, b])
    flags = np.concatenate([to_np(fa), to_np(fb)])
    assert_flags_per_key(both, flags, oracle_lib.OracleTable().find_or_put(both))
    assert t.size() == 25_000
    t.close()


def test_invalid_items_are_rejected():
    t = ht.HashTable(1000, "bucket", 64)
    k = to_dev(wk.distinct_keys(10, 64, seed=1))
    with pytest.raises(ht.HtError):
        ht.ht_multi_find_or_put([t.handle], [(1, k, None)])
    ht.ht_multi_find_or_put([t.handle], [])                    # nothing to do
    ht.ht_multi_find_or_put([t.handle], [(0, k, None)])        # flags optional
    assert t.size() == 10
    t.close()
