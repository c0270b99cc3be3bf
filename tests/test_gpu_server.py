"""The serving loop: results in the mix equal results alone, admission by
free device memory, bounded waits.

"Alone" means the same requests of each table run one after another through
plain ht_find_or_put on a fresh table; "in the mix" means all requests of all
tables submitted at once and batched by the server.  Per request the number
of is_new flags of every distinct key must agree (and with the oracle).
"""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import keys as wk

from gpu_util import assert_flags_per_key, to_dev, to_np

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


def _trace(seed, n_tables, n_req, max_n=20000):
    rng = np.random.default_rng(seed)
    pools = [wk.distinct_keys(30000, 64, seed=seed * 100 + t) for t in range(n_tables)]
    reqs = []
    for _ in range(n_req):
        t = int(rng.integers(0, n_tables))
        n = int(np.exp(rng.uniform(0, np.log(max_n))))
        keys = pools[t][rng.integers(0, len(pools[t]), size=n)]
        reqs.append((t, keys))
    return reqs


def _alone(reqs, schemes, caps):
    tables = [ht.HashTable(c, s, 64) for c, s in zip(caps, schemes)]
    out = []
    for t, keys in reqs:
        out.append(to_np(tables[t].find_or_put(to_dev(keys))))
    return out


@pytest.mark.parametrize("pack,inflight", [(1, 4), (1, 1), (0, 2)])
def test_results_in_the_mix_equal_results_alone(oracle_lib, pack, inflight):
    schemes = ["bucket"] * 6 + ["cuckoo"] * 3
    caps = [40000, 50000, 60000, 45000, 70000, 38000, 40000, 52000, 64000]
    reqs = _trace(3, len(schemes), 250)
    srv = ht.Server(pack=pack, max_inflight=inflight, hbm_reserve_bytes=0)
    ids = [srv.open_table(c, s) for c, s in zip(caps, schemes)]
    rids = [srv.submit(ids[t], keys) for t, keys in reqs]
    mixed = []
    for r in rids:
        st, lat, flags = srv.wait(r, timeout_ms=60000)
        assert st == 0 and lat is not None and lat >= 0
        mixed.append(flags.copy())
    alone = _alone(reqs, schemes, caps)
    oracles = [oracle_lib.OracleTable() for _ in schemes]
    for (t, keys), m, a in zip(reqs, mixed, alone):
        exp = oracles[t].find_or_put(keys)
        assert_flags_per_key(keys, m, a)
        assert_flags_per_key(keys, m, exp)
    stats = srv.stats()
    assert stats["requests"] == len(reqs) and stats["status"] == 0
    assert stats["keys"] == sum(len(k) for _, k in reqs)
    assert 0 <= stats["p50_us"] <= stats["p99_us"] <= stats["max_us"]
    for i, o in zip(ids, oracles):
        adm, size = srv.table_state(i)
        assert adm == 1 and size == o.size()
    srv.close()


def test_admission_waits_for_free_memory():
    # Pretend 3.5 tables' worth of memory is free: the 4th table waits until
    # another closes; its requests time out meanwhile, then complete.
    cap = 1 << 20
    one = cap * 8 + 4096 * 8 + (1 << 16) * 8 + 4096
    srv = ht.Server(fake_free_bytes=int(one * 3.5), hbm_reserve_bytes=0)
    ids = [srv.open_table(cap, "bucket") for _ in range(4)]
    keys = [wk.distinct_keys(5000, 64, seed=70 + i) for i in range(4)]
    rids = [srv.submit(ids[i], keys[i]) for i in range(4)]
    for i in range(3):
        st, _, flags = srv.wait(rids[i], timeout_ms=30000)
        assert st == 0 and flags.sum() == 5000
    assert srv.table_state(ids[3])[0] == 0
    st, _, _ = srv.wait(rids[3], timeout_ms=200)
    assert st == 5                                  # HT_ERR_TIMEOUT: still waiting for admission
    srv.close_table(ids[0])
    st, _, flags = srv.wait(rids[3], timeout_ms=30000)
    assert st == 0 and flags.sum() == 5000
    assert srv.table_state(ids[0])[0] == -1 and srv.table_state(ids[3])[0] == 1
    srv.close()


def test_submit_rejects_bad_requests():
    srv = ht.Server(batch_key_budget=1024, hbm_reserve_bytes=0)
    t = srv.open_table(4096, "bucket")
    with pytest.raises(ht.HtError):
        srv.submit(t, np.arange(2000, dtype=np.uint64))
    with pytest.raises(ht.HtError):
        srv.submit(t + 5, np.arange(10, dtype=np.uint64))
    srv.close_table(t)
    with pytest.raises(ht.HtError):
        srv.submit(t, np.arange(10, dtype=np.uint64))
    srv.close()


def test_admission_with_real_free_memory_after_close():
    # Reserve all but ~1.5 tables of the real free memory: the second table
    # is admitted only once the first one's memory is back with the driver.
    cap = 1 << 26
    one = cap * 8 + 4096 * 8 + (1 << 16) * 8 + 4096
    torch.cuda.synchronize()
    free, _ = torch.cuda.mem_get_info()
    srv = ht.Server(hbm_reserve_bytes=int(free - 1.5 * one))
    a = srv.open_table(cap, "bucket")
    b = srv.open_table(cap, "bucket")
    ka, kb = wk.distinct_keys(1000, 64, seed=81), wk.distinct_keys(1000, 64, seed=82)
    ra, rb = srv.submit(a, ka), srv.submit(b, kb)
    st, _, flags = srv.wait(ra, timeout_ms=30000)
    assert st == 0 and flags.sum() == 1000
    assert srv.wait(rb, timeout_ms=300)[0] == 5       # b waits for memory
    srv.close_table(a)
    st, _, flags = srv.wait(rb, timeout_ms=30000)
    assert st == 0 and flags.sum() == 1000
    srv.close()


def test_overfull_table_reports_full_and_others_stay_exact(oracle_lib):
    # A 64-slot table cannot hold 5000 keys (table + stash + overflow set):
    # its request reports HT_ERR_FULL (3), sticky for its later requests;
    # requests of another table in the same batches stay exact.
    srv = ht.Server(hbm_reserve_bytes=0)
    small = srv.open_table(64, "bucket")
    big = srv.open_table(100_000, "bucket")
    ks, kb = wk.distinct_keys(5000, 64, seed=91), wk.distinct_keys(20_000, 64, seed=92)
    r1, r2 = srv.submit(small, ks), srv.submit(big, kb)
    assert srv.wait(r1, timeout_ms=30000)[0] == 3
    st, _, flags = srv.wait(r2, timeout_ms=30000)
    assert st == 0 and flags.sum() == 20_000
    assert srv.wait(srv.submit(small, ks[:10]), timeout_ms=30000)[0] == 3
    st, _, flags = srv.wait(srv.submit(big, kb[:100]), timeout_ms=30000)
    assert st == 0 and flags.sum() == 0
    srv.close()


def test_pinned_requests_match_pageable(oracle_lib):
    # Large requests whose keys sit in page-locked memory are copied to the
    # device straight from the caller's buffer; results are the same.
    reqs = [wk.distinct_keys(n, 64, seed=95 + i) for i, n in enumerate([70_000, 1000, 200_000, 65_536])]
    reqs[2][:50_000] = reqs[0][:50_000]                 # repeats across requests of one table
    pinned = [torch.from_numpy(k.view(np.int64)).pin_memory() for k in reqs]
    srv = ht.Server(hbm_reserve_bytes=0)
    t_pin, t_page = srv.open_table(600_000, "bucket"), srv.open_table(600_000, "bucket")
    rp = [srv.submit(t_pin, p.numpy().view(np.uint64)) for p in pinned]
    rq = [srv.submit(t_page, k) for k in reqs]
    orc = oracle_lib.OracleTable()
    for k, a, b in zip(reqs, rp, rq):
        sa, _, fa = srv.wait(a, timeout_ms=30000)
        sb, _, fb = srv.wait(b, timeout_ms=30000)
        assert sa == sb == 0
        exp = orc.find_or_put(k)
        assert_flags_per_key(k, fa, exp)
        assert_flags_per_key(k, fb, exp)
    srv.close()
