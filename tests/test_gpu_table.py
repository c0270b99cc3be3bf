"""Parity of the CUDA find-or-put / insert / lookup path with the CPU oracle.

Every comparison is exact (integer work): per distinct key of a batch the
number of is_new flags equals the oracle's, the stored set equals the
oracle's set, found flags are identical and values are the oracle's (or, for
a key first inserted by a batch that held it several times, one of the
values supplied for it in that batch).
"""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import keys as wk

from gpu_util import assert_flags_per_key, assert_same_set, keys_np, to_dev, to_np

pytestmark = pytest.mark.gpu
SCHEMES = ["bucket", "cuckoo"]


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


def _fill_and_check(oracle_lib, scheme, kw, n_distinct, batch, dup, lf, params=None, seed=1):
    fs = wk.fill_stream(n_distinct, batch, dup, kw, seed=seed)
    cap = int(np.ceil(n_distinct / lf))
    t = ht.HashTable(cap, scheme, kw, params)
    orc = oracle_lib.OracleTable()
    for b in range(fs.n_batches):
        kb = fs.batch(b)
        got = to_np(t.find_or_put(to_dev(kb)))
        exp = orc.find_or_put(kb)
        assert_flags_per_key(kb, got, exp)
        assert got.sum() == fs.fresh_counts[b]
    assert t.sync() == 0
    assert t.size() == orc.size() == n_distinct
    k, _ = t.export()
    assert_same_set(keys_np(k, kw), orc.export()[0])
    return t, orc, fs


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("kw", [32, 64])
@pytest.mark.parametrize("dup", [0.0, 0.25, 0.5])
def test_find_or_put_parity(oracle_lib, scheme, kw, dup):
    # Several batches, a ragged last batch, load 0.8.
    _fill_and_check(oracle_lib, scheme, kw, n_distinct=100_003, batch=1 << 15, dup=dup, lf=0.8)


@pytest.mark.parametrize("kw", [32, 64])
@pytest.mark.parametrize("lf", [0.8, 0.9])
def test_cuckoo_paper_insertion_rule_parity(oracle_lib, kw, lf):
    # cuckoo_chain_h1 = 1: Section 4.1's rule, every insertion starting at
    # h_1 (a CAS in the probe only when h_1 was empty, else a claim and an
    # eviction chain from h_1), with many keys finding h_1 taken at these
    # loads; results equal the oracle's like the default rule's.
    t, _, fs = _fill_and_check(oracle_lib, "cuckoo", kw, n_distinct=100_003, batch=1 << 15, dup=0.25, lf=lf,
                               params=dict(cuckoo_chain_h1=1), seed=17)
    st = t.stats()
    assert st["exchanges"] > 0 and st["probe_cas"] > 0


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("lf", [0.5, 0.9])
def test_find_or_put_loads(oracle_lib, scheme, lf):
    _fill_and_check(oracle_lib, scheme, 64, n_distinct=(1 << 18) + 77, batch=1 << 16, dup=0.25, lf=lf, seed=7)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("slots,lanes", [(8, 4), (8, 8), (16, 4), (16, 16), (32, 8), (32, 16), (32, 32)])
def test_bucket_shapes_and_cuckoo_hashes(oracle_lib, scheme, slots, lanes):
    if scheme == "bucket":
        params = dict(bucket_slots=slots, lanes_per_key=lanes)
    else:
        params = dict(num_hashes=2 + (slots * lanes) % 7, bucket_slots=slots)
    _fill_and_check(oracle_lib, scheme, 64, n_distinct=50_000, batch=20_000, dup=0.5, lf=0.8, params=params)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("n,kw", [(30_000, 32), (300_000, 64)])
def test_l2_persisting_tables_stay_exact(oracle_lib, scheme, n, kw):
    # l2_persist attaches an access-policy window (the slots, or Cuckoo's
    # claim set) to every launch of the table; results must not change.
    _fill_and_check(oracle_lib, scheme, kw, n_distinct=n, batch=1 << 14, dup=0.3, lf=0.8,
                    params=dict(l2_persist=1), seed=13)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_single_key_repeated(oracle_lib, scheme):
    keys = np.full(1 << 16, 12345, dtype=np.uint64)
    t = ht.HashTable(1024, scheme, 64)
    got = to_np(t.find_or_put(to_dev(keys)))
    assert got.sum() == 1
    got = to_np(t.find_or_put(to_dev(keys)))
    assert got.sum() == 0
    assert t.size() == 1


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("kw", [32, 64])
def test_empty_and_tiny_batches(oracle_lib, scheme, kw):
    t = ht.HashTable(64, scheme, kw)
    dt = torch.int32 if kw == 32 else torch.int64
    empty = torch.empty(0, dtype=dt, device="cuda")
    assert t.find_or_put(empty).numel() == 0
    f, _ = t.lookup(empty)
    assert f.numel() == 0
    one = torch.tensor([5], dtype=dt, device="cuda")
    assert to_np(t.find_or_put(one)).tolist() == [1]
    assert to_np(t.lookup(one)[0]).tolist() == [1]
    assert t.size() == 1


@pytest.mark.parametrize("scheme", SCHEMES)
def test_map_insert_lookup_parity(oracle_lib, scheme):
    rng = np.random.default_rng(5)
    n = 60_000
    t = ht.HashTable(int(n / 0.8), scheme, 32)
    orc = oracle_lib.OracleTable()
    pool = wk.distinct_keys(n, 32, seed=11)
    first_batch_vals = {}
    for b in range(3):
        kb = pool[rng.integers(0, n, size=40_000)]
        vb = rng.integers(0, 2**32 - 1, size=len(kb), dtype=np.uint64).astype(np.uint32)
        absent_before = {int(k) for k in np.unique(kb)} - set(orc.export()[0].tolist())
        for k, v in zip(kb.tolist(), vb.tolist()):
            if k in absent_before:
                first_batch_vals.setdefault(k, set()).add(v)
        t.insert(to_dev(kb), to_dev(vb))
        orc.insert(kb, vb)
        q = np.concatenate([pool, wk.distinct_keys(5000, 32, seed=11, start=n + 10)])
        found, vals = t.lookup(to_dev(q))
        of, ov = orc.lookup(q)
        np.testing.assert_array_equal(to_np(found), of)
        gv = to_np(vals, np.uint32)
        # Every found key's value: one of the values its first inserting
        # batch supplied for it (which one is unspecified); absent keys read 0.
        bad = [int(q[i]) for i in np.nonzero(of)[0] if int(gv[i]) not in first_batch_vals[int(q[i])]]
        assert not bad, (len(bad), bad[:3])
        assert not gv[of == 0].any()
        assert t.size() == orc.size()
    # A second insert of present keys keeps the first values.
    before = to_np(t.lookup(to_dev(pool))[1], np.uint32)
    t.insert(to_dev(pool), to_dev(np.zeros(n, dtype=np.uint32)))
    after = to_np(t.lookup(to_dev(pool))[1], np.uint32)
    np.testing.assert_array_equal(before, after)


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("kw", [32, 64])
def test_lookup_half_present(oracle_lib, scheme, kw):
    n = 1 << 17
    t = ht.HashTable(int(n / 0.8), scheme, kw)
    t.insert(to_dev(wk.distinct_keys(n, kw, seed=2)))
    q, present = wk.lookup_batch(n, (1 << 17) + 5, kw, seed=2)
    found, _ = t.lookup(to_dev(q))
    np.testing.assert_array_equal(to_np(found), present)


@pytest.mark.parametrize("scheme", SCHEMES)
def test_reserved_key_reports_invalid(oracle_lib, scheme):
    t = ht.HashTable(256, scheme, 32)
    keys = np.array([1, 2, 0xFFFFFFFF, 3, 2], dtype=np.uint32)
    got = to_np(t.find_or_put(to_dev(keys)))
    assert got.tolist()[2] == 0 and got.sum() == 3
    assert t.sync() == 1          # HT_ERR_INVALID, reported once
    assert t.sync() == 0
    assert t.size() == 3
    t64 = ht.HashTable(256, scheme, 64)
    k64 = np.array([1, 1 << 63, 7], dtype=np.uint64)
    assert to_np(t64.find_or_put(to_dev(k64))).tolist() == [1, 0, 1]
    assert t64.sync() == 1


@pytest.mark.parametrize("scheme", SCHEMES)
def test_stash_overflow_and_rebuild(oracle_lib, scheme):
    # A small table with one hash function per bucket (or two for Cuckoo), a
    # 4-slot stash and one eviction: many keys spill, the overflow set asks
    # for a rebuild and the next synchronising call runs it.  Results stay
    # exact throughout.
    if scheme == "bucket":
        params = dict(num_hashes=1, bucket_slots=8, lanes_per_key=4, stash_slots=4)
    else:
        params = dict(num_hashes=2, max_evictions=1, stash_slots=4)
    n = 700
    fs = wk.fill_stream(n, 256, 0.3, 64, seed=4)
    t = ht.HashTable(1024, scheme, 64, params)
    orc = oracle_lib.OracleTable()
    for b in range(fs.n_batches):
        kb = fs.batch(b)
        got = to_np(t.find_or_put(to_dev(kb)))
        assert_flags_per_key(kb, got, orc.find_or_put(kb))
        q = fs.keys[:fs.offsets[b + 1]]
        np.testing.assert_array_equal(to_np(t.lookup(to_dev(q))[0]), np.ones(len(q), np.uint8))
    assert t.sync() == 0
    assert t.info()["rebuilds"] >= 1
    assert t.size() == n
    k, _ = t.export()
    assert_same_set(keys_np(k, 64), orc.export()[0])
    absent = wk.distinct_keys(1000, 64, seed=4, start=n + 1)
    assert to_np(t.lookup(to_dev(absent))[0]).sum() == 0


@pytest.mark.parametrize("scheme", SCHEMES)
def test_small_table_large_batches_with_repeats(oracle_lib, scheme):
    # Batches far larger than the table (each key repeated ~40 times): a
    # Cuckoo launch takes max_batch keys while its dedup set and winner list
    # are sized by the table; results stay exact.
    rng = np.random.default_rng(8)
    pool = wk.distinct_keys(50_000, 64, seed=61)
    t = ht.HashTable(65_000, scheme, 64)
    orc = oracle_lib.OracleTable()
    for b in range(3):
        kb = pool[rng.integers(0, len(pool), size=(1 << 21) + 12345)]
        got = to_np(t.find_or_put(to_dev(kb)))
        assert_flags_per_key(kb, got, orc.find_or_put(kb))
    assert t.sync() == 0 and t.size() == orc.size()


def test_cuckoo_batch_with_more_distinct_keys_than_the_table_holds():
    # 200k distinct keys into ~1300 places: the table reports HT_ERR_FULL and
    # counts what it dropped; nothing is written out of bounds; every stored
    # key was reported new (a new key may still be dropped: the table is full).
    keys = wk.distinct_keys(200_000, 64, seed=62)
    t = ht.HashTable(128, "cuckoo", 64)
    flags = to_np(t.find_or_put(to_dev(keys))).astype(bool)
    assert t.sync() == 3
    found = to_np(t.lookup(to_dev(keys))[0]).astype(bool)
    st = t.stats()
    assert 0 < found.sum() == st["size"] <= 128 + 101 + 1024
    assert not (found & ~flags).any()
    assert st["dropped"] > 0 and st["dropped"] + st["size"] >= flags.sum()


@pytest.mark.parametrize("scheme", SCHEMES)
def test_overfull_table_reports_full(oracle_lib, scheme):
    # 3000 keys into 64 slots + 4 stash + 1024 overflow: keys are dropped and
    # the table reports HT_ERR_FULL; nothing hangs.
    params = dict(num_hashes=2, stash_slots=4, max_rebuilds=2, max_evictions=8)
    t = ht.HashTable(64, scheme, 64, params)
    t.find_or_put(to_dev(wk.distinct_keys(3000, 64, seed=9)))
    assert t.sync() == 3


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("kw", [32, 64])
def test_find_or_put_append_and_compact(oracle_lib, scheme, kw):
    fs = wk.fill_stream(30_000, 1 << 14, 0.5, kw, seed=8)
    t = ht.HashTable(40_000, scheme, kw)
    dt = torch.int32 if kw == 32 else torch.int64
    for b in range(fs.n_batches):
        kb = to_dev(fs.batch(b))
        out = torch.empty(kb.numel(), dtype=dt, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        is_new = torch.empty(kb.numel(), dtype=torch.uint8, device="cuda")
        ht.ht_find_or_put_append(t.handle, kb, out, cnt, is_new)
        c = int(cnt.item())
        assert c == fs.fresh_counts[b]
        exp = np.unique(keys_np(kb[is_new.bool()], kw))
        assert_same_set(keys_np(out[:c], kw), exp)
        out2 = torch.empty_like(out)
        cnt2 = torch.zeros(1, dtype=torch.int64, device="cuda")
        ht.ht_compact(kb, is_new, out2, cnt2)
        assert int(cnt2.item()) == c
        assert_same_set(keys_np(out2[:c], kw), exp)


def test_compact_matches_numpy():
    rng = np.random.default_rng(3)
    for n in [0, 1, 31, 33, 1000, 123_457]:
        keys = rng.integers(0, 2**63 - 1, size=n, dtype=np.uint64)
        flags = (rng.random(n) < 0.3).astype(np.uint8)
        out = torch.empty(max(n, 1), dtype=torch.int64, device="cuda")
        cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
        ht.ht_compact(to_dev(keys), to_dev(flags), out, cnt)
        c = int(cnt.item())
        assert c == flags.sum()
        np.testing.assert_array_equal(np.sort(to_np(out[:c], np.uint64)), np.sort(keys[flags == 1]))


@pytest.mark.parametrize("scheme", SCHEMES)
def test_stats_counters(oracle_lib, scheme):
    # size and the stash/overflow counts agree with the table; Cuckoo makes
    # at least one table atomic per new key (a CAS into the first empty slot
    # its probe saw or, with all k slots full, a chain's exchanges) and the
    # bucket scheme none; ht_clear zeroes them.
    t, orc, fs = _fill_and_check(oracle_lib, scheme, 64, n_distinct=200_000, batch=1 << 15, dup=0.25, lf=0.85,
                                 seed=31)
    st = t.stats()
    assert st["size"] == orc.size() == t.size()
    assert st["dropped"] == 0 and st["flags"] == 0
    if scheme == "cuckoo":
        atomics = st["probe_cas"] + st["exchanges"]
        assert atomics >= fs.n_distinct - st["stash_used"] - st["overflow_used"]
        assert atomics < 50 * fs.n_distinct
        assert st["probe_cas"] <= 4 * (fs.n_issued - fs.n_distinct) + 4 * fs.n_distinct
        assert st["exchanges"] > 0                            # at load 0.85 some keys find k slots full
        # Every key reads h_1; a key reads all k slots only when h_1 is occupied.
        assert fs.n_issued <= st["probes"] <= 4 * fs.n_issued
        assert st["probes"] < 4 * fs.n_issued * 0.9           # early exits happen at load 0.85
    else:
        assert st["exchanges"] == st["probe_cas"] == 0
        assert st["probes"] == 0                              # not counted for the bucket scheme
    t.clear()
    st = t.stats()
    assert st["size"] == st["exchanges"] == st["probe_cas"] == st["stash_used"] == st["overflow_used"] == 0


def test_cuckoo_probe_miss_counters():
    """The probe's miss counters: n distinct keys into an empty table all
    miss (each read at least h_1, at most k slots); the same keys again all
    hit, adding reads but no misses."""
    n = 100_000
    keys = wk.distinct_keys(n, 64, seed=44)
    t = ht.HashTable(int(n / 0.8), "cuckoo", 64)
    t.find_or_put(to_dev(keys))
    st = t.stats()
    assert st["probe_misses"] == n
    assert n <= st["probe_miss_reads"] <= 4 * n and st["probe_miss_reads"] == st["probes"]
    t.find_or_put(to_dev(keys))
    st2 = t.stats()
    assert st2["probe_misses"] == n and st2["probe_miss_reads"] == st["probe_miss_reads"]
    assert st2["probes"] - st["probes"] >= n                   # every hit read h_1 at least
    assert st2["probe_cas"] == st["probe_cas"] and st2["exchanges"] == st["exchanges"]   # hits store nothing


def test_cuckoo_probe_stores_at_low_load():
    """Distinct keys into a table at load 0.05: nearly every key sees an
    empty slot, so the probe stores it with one CAS and almost no key needs
    an eviction chain; the set stays exact."""
    n = 100_000
    keys = wk.distinct_keys(n, 64, seed=45)
    t = ht.HashTable(n * 20, "cuckoo", 64)
    flags = to_np(t.find_or_put(to_dev(keys)))
    assert flags.sum() == n and t.size() == n
    st = t.stats()
    # Keys of one batch whose first empty slot coincides (about n^2 / 2m
    # pairs, 2.5% of n here) race on it; the loser's CAS moves on to its
    # next slot.
    assert n <= st["probe_cas"] <= n + n // 20
    assert st["exchanges"] <= n // 1000
    assert to_np(t.lookup(to_dev(keys))[0]).all()
    found, _ = t.lookup(to_dev(wk.distinct_keys(1000, 64, seed=44, start=n + 5)))
    assert int(found.sum()) == 0
    assert t.stats()["probe_misses"] == n                     # lookups are not counted


@pytest.mark.parametrize("scheme", SCHEMES)
def test_clear_empties(oracle_lib, scheme):
    t = ht.HashTable(4096, scheme, 64)
    k = to_dev(wk.distinct_keys(3000, 64, seed=1))
    assert to_np(t.find_or_put(k)).sum() == 3000
    t.clear()
    assert t.size() == 0
    assert to_np(t.find_or_put(k)).sum() == 3000


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("kw", [32, 64])
def test_grow_keeps_contents_and_values(oracle_lib, scheme, kw):
    n = 50_000
    keys = wk.distinct_keys(n, kw, seed=71)
    t = ht.HashTable(70_000, scheme, kw)
    orc = oracle_lib.OracleTable()
    if kw == 32:
        vals = ((np.arange(n, dtype=np.uint64) * 2654435761) & 0xFFFFFFFF).astype(np.uint32)
        t.insert(to_dev(keys), to_dev(vals))
    else:
        t.find_or_put(to_dev(keys))
    orc.find_or_put(keys)
    t.grow(300_000)
    assert t.info()["slots"] >= 300_000 and t.size() == n
    f, v = t.lookup(to_dev(keys))
    assert to_np(f).all()
    if kw == 32:
        np.testing.assert_array_equal(to_np(v, np.uint32), vals)
    more = wk.distinct_keys(150_000, kw, seed=71, start=n - 10_000)       # 10k repeats, 140k new
    assert_flags_per_key(more, to_np(t.find_or_put(to_dev(more))), orc.find_or_put(more))
    assert t.sync() == 0 and t.size() == orc.size()
    k, _ = t.export()
    assert_same_set(keys_np(k, kw), orc.export()[0])


@pytest.mark.parametrize("scheme", SCHEMES)
def test_grow_too_small_reports_full_and_keeps_the_table(oracle_lib, scheme):
    keys = wk.distinct_keys(20_000, 64, seed=72)
    t = ht.HashTable(30_000, scheme, 64)
    t.find_or_put(to_dev(keys))
    slots = t.info()["slots"]
    with pytest.raises(ht.HtError) as e:
        t.grow(1000)
    assert e.value.status == 3
    assert t.info()["slots"] == slots and t.size() == 20_000 and t.sync() == 0
    assert to_np(t.lookup(to_dev(keys))[0]).all()


@pytest.mark.parametrize("scheme", SCHEMES)
def test_auto_grow_at_synchronising_calls(oracle_lib, scheme):
    # Starts at 4096 slots, grows whenever a sync finds it above load 0.8.
    fs = wk.fill_stream(200_000, 1024, 0.25, 64, seed=73)
    t = ht.HashTable(4096, scheme, 64, dict(grow_load_permille=800))
    orc = oracle_lib.OracleTable()
    for b in range(fs.n_batches):
        kb = fs.batch(b)
        assert_flags_per_key(kb, to_np(t.find_or_put(to_dev(kb))), orc.find_or_put(kb))
        assert t.sync() == 0
    assert t.size() == 200_000 and t.info()["slots"] >= 200_000 / 0.8
    k, _ = t.export()
    assert_same_set(keys_np(k, 64), orc.export()[0])


@pytest.mark.parametrize("scheme", SCHEMES)
@pytest.mark.parametrize("kw", [32, 64, 128])
def test_checkpoint_save_and_load(oracle_lib, scheme, kw, tmp_path):
    n = 30_000
    if kw == 128:
        lo = wk.distinct_keys(n, 64, seed=81)
        keys = torch.from_numpy(np.stack([lo, lo ^ np.uint64(12345)], axis=1).view(np.int64)).cuda()
        vals = None
    else:
        keys = to_dev(wk.distinct_keys(n, kw, seed=81))
        vals = to_dev(np.arange(n, dtype=np.uint32)) if kw == 32 else None
    t = ht.HashTable(40_000, scheme, kw)
    t.insert(keys, vals)
    path = str(tmp_path / "table.npz")
    t.save(path)
    r = ht.HashTable.load(path)
    assert r.size() == n and r.info()["slots"] == t.info()["slots"] and r.key_width == kw
    f, v = r.lookup(keys)
    assert to_np(f).all()
    if kw == 32:
        np.testing.assert_array_equal(to_np(v, np.uint32), np.arange(n, dtype=np.uint32))
