"""128-bit keys (state vectors wider than 64 bits) in both schemes: parity
with the 128-bit oracle set, exactly as for 64-bit keys."""
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


# (scheme, params): the bucket scheme at 2 and 4 lanes per key, Cuckoo (k=4).
TABLES = [("bucket", dict(bucket_slots=8, lanes_per_key=2)), ("bucket", dict(bucket_slots=8, lanes_per_key=4)),
          ("cuckoo", None)]
TABLE_IDS = ["bucket_g2", "bucket_g4", "cuckoo"]


@pytest.mark.parametrize("table", TABLES, ids=TABLE_IDS)
@pytest.mark.parametrize("share", [None, "lo", "hi"])
def test_find_or_put_lookup_export_match_oracle(oracle_lib, table, share):
    rng = np.random.default_rng(5)
    n = 120_000
    pool = _pairs(n, seed=40, share=share)
    t = ht.HashTable(int(n / 0.85), table[0], 128, table[1])
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


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_edge_keys_and_reserved(oracle_lib, scheme):
    # Words that are all ones except the reserved bit, zeros, and a key with
    # an all-ones low word (a legal key that reads like a half-written slot).
    ones = np.uint64(2 ** 64 - 1)
    top = np.uint64(2 ** 63 - 1)
    keys = np.array([[0, 0], [ones, 0], [0, top], [ones, top], [1, 2], [ones, 0]], dtype=np.uint64)
    t = ht.HashTable(64, scheme, 128)
    got = t.find_or_put(_dev(keys)).cpu().numpy()
    np.testing.assert_array_equal(got, [1, 1, 1, 1, 1, 0])
    f, _ = t.lookup(_dev(keys))
    assert f.cpu().numpy().all()
    assert t.size() == 5 and t.sync() == 0
    bad = np.array([[3, 2 ** 63]], dtype=np.uint64)                  # reserved bit set
    t.find_or_put(_dev(bad))
    assert t.sync() == 1


def test_cuckoo_keys_with_an_all_ones_low_word(oracle_lib):
    # A key whose low word is all ones reads like a half-written slot, so the
    # Cuckoo probe settles such a slot with its CAS, never by the read.  Many
    # such keys, repeated within and across batches, stay exact.
    ones = np.uint64(2 ** 64 - 1)
    keys = np.stack([np.full(4000, ones, dtype=np.uint64), wk.distinct_keys(4000, 64, seed=81)], axis=1)
    t = ht.HashTable(8000, "cuckoo", 128)
    orc = oracle_lib.OracleTable128()
    rng = np.random.default_rng(5)
    for lo in range(0, 4000, 1000):
        b = np.concatenate([keys[lo:lo + 1000], keys[rng.integers(0, lo + 1000, size=1000)]])
        b = b[rng.permutation(len(b))]
        assert_flags_per_key(_ids(b), t.find_or_put(_dev(b)).cpu().numpy(), orc.find_or_put(b))
    assert t.sync() == 0 and t.size() == 4000
    f, _ = t.lookup(_dev(keys))
    assert f.cpu().numpy().all()


def test_cuckoo_paper_insertion_rule_parity(oracle_lib):
    # cuckoo_chain_h1 = 1 (Section 4.1's start at h_1) for 128-bit keys, at
    # load 0.85 with repeats within and across batches, against the oracle.
    keys = _pairs(20_000, seed=83)
    t = ht.HashTable(int(20_000 / 0.85), "cuckoo", 128, dict(cuckoo_chain_h1=1))
    orc = oracle_lib.OracleTable128()
    rng = np.random.default_rng(9)
    for lo in range(0, 20_000, 5000):
        b = np.concatenate([keys[lo:lo + 5000], keys[rng.integers(0, lo + 5000, size=2000)]])
        b = b[rng.permutation(len(b))]
        assert_flags_per_key(_ids(b), t.find_or_put(_dev(b)).cpu().numpy(), orc.find_or_put(b))
    assert t.sync() == 0 and t.size() == 20_000
    assert t.stats()["exchanges"] > 0


def test_cuckoo_probe_stores_at_low_load():
    # At load 0.05 nearly every key sees an empty slot: the probe stores it
    # with one 16-byte CAS (a few more where keys of the batch race for a
    # slot) and almost no key runs an eviction chain; a second pass finds
    # every key and stores nothing.
    n = 50_000
    keys = _pairs(n, seed=82)
    t = ht.HashTable(n * 20, "cuckoo", 128)
    assert t.find_or_put(_dev(keys)).cpu().numpy().sum() == n and t.size() == n
    st = t.stats()
    assert n <= st["probe_cas"] <= n + n // 20
    assert st["exchanges"] <= n // 1000
    assert t.find_or_put(_dev(keys)).cpu().numpy().sum() == 0
    assert t.stats()["probe_cas"] == st["probe_cas"]


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_overflow_grow_and_full(oracle_lib, scheme):
    # A small table spills into its overflow set, reports full beyond it,
    # and growth moves every key to the new storage.
    keys = _pairs(3000, seed=77)
    params = dict(num_hashes=2) if scheme == "bucket" else dict(num_hashes=2, max_evictions=4)
    t = ht.HashTable(64, scheme, 128, params)
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
    small = ht.HashTable(8, scheme, 128, dict(num_hashes=1) if scheme == "bucket" else dict(num_hashes=2))
    small.find_or_put(_dev(_pairs(5000, seed=78)))
    assert small.sync() == 3


def test_unsupported_uses_are_rejected():
    with pytest.raises(ht.HtError):
        ht.HashTable(64, "bucket", 128, dict(bucket_slots=16))
    t = ht.HashTable(1024, "bucket", 128)
    from workloads import statespace as ss
    m = ss.random_model(1, C=3, L=8, R=5)
    with pytest.raises(ht.HtError):
        ht.ht_bfs(t.handle, _hmodel(m), 0, 16, torch.empty((1024, 2), dtype=torch.int64, device="cuda"), fused=True)


WIDE_MODELS = [
    dict(seed=31, C=16, L=32, R=[2, 3, 2, 2, 3, 2, 2, 2, 2, 2, 2, 2, 3, 2, 2, 2], p_sync=0.0, P=0),
    dict(seed=32, C=16, L=32, R=[3, 2, 3, 2, 2, 3, 2, 2, 3, 2, 2, 2, 2, 2, 3, 2], p_sync=0.4, P=4),
    dict(seed=33, C=14, L=[32] * 8 + [16] * 6, R=[4, 3, 3, 2, 3, 2, 2, 3, 2, 2, 3, 2, 2, 3], p_sync=0.3, P=5),
]


def _hmodel(m):
    return ht.make_model(m.C, m.bits, m.deg, m.tgt, m.lab, m.pairs)


@pytest.mark.parametrize("spec", WIDE_MODELS)
def test_wide_successors_match_oracle(oracle_lib, spec):
    from workloads import statespace as ss
    m = ss.random_model(spec["seed"], C=spec["C"], L=spec["L"], R=spec["R"], p_sync=spec["p_sync"], P=spec["P"])
    assert m.key_width == 128
    ref = oracle_lib.bfs(m, max_states=1 << 20, wide=True)
    states = ref.states[: min(5000, ref.total)]
    d = torch.from_numpy(np.ascontiguousarray(states).view(np.int64)).cuda()
    succ = torch.empty((len(states) * 64, 2), dtype=torch.int64, device="cuda")
    cnt = torch.zeros(1, dtype=torch.int64, device="cuda")
    ht.ht_successors(_hmodel(m), d, succ, cnt)
    c = int(cnt.item())
    exp = np.concatenate([oracle_lib.successors128(m, int(a) | (int(b) << 64)) for a, b in states.tolist()])
    assert c == len(exp)
    got = succ[:c].cpu().numpy().view(np.uint64)
    assert sorted(map(tuple, got.tolist())) == sorted(map(tuple, exp.tolist()))


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
@pytest.mark.parametrize("spec", WIDE_MODELS)
def test_wide_bfs_matches_oracle_levels(oracle_lib, spec, scheme):
    from workloads import statespace as ss
    m = ss.random_model(spec["seed"], C=spec["C"], L=spec["L"], R=spec["R"], p_sync=spec["p_sync"], P=spec["P"])
    ref = oracle_lib.bfs(m, max_states=1 << 22, wide=True)
    assert ref.rc == 0
    t = ht.HashTable(max(64, int(ref.total / 0.7)), scheme, 128)
    states = torch.empty((ref.total + 16, 2), dtype=torch.int64, device="cuda")
    res, sizes = ht.ht_bfs(t.handle, _hmodel(m), 0, 4096, states)
    assert res.complete == 1 and res.states == ref.total
    assert res.successors == int(ref.level_succ.sum())
    np.testing.assert_array_equal(np.array(sizes), ref.level_sizes)
    got = states[:res.states].cpu().numpy().view(np.uint64)
    off = 0
    for d, n_d in enumerate(sizes):
        assert set(map(tuple, got[off:off + n_d].tolist())) == set(map(tuple, ref.level(d).tolist())), d
        off += n_d
    assert t.size() == ref.total
