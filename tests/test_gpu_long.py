"""Keys of 3 to 8 64-bit words (192 to 512 bits) in both schemes: parity with
the oracle's set of word vectors, exactly as for one- and two-word keys.

The bucket scheme claims a header word and publishes the key's words after
writing them; Cuckoo keeps (digest, row) entries pointing into a key store.
Tests with a shortened digest make distinct keys share digests, so the
full-key comparisons that tell them apart run on most probes."""
import ctypes

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


def _dev(rows):
    return torch.from_numpy(np.ascontiguousarray(rows, dtype=np.uint64).view(np.int64)).cuda()


def _ids(rows):
    """A scalar id per distinct row, for per-key flag counts."""
    _, inv = np.unique(rows, axis=0, return_inverse=True)
    return inv.reshape(-1)


def _rows(t):
    return set(map(tuple, t.cpu().numpy().view(np.uint64).tolist()))


def _stream_check(t, orc, pool, rng, fresh_per_batch, repeats):
    issued = 0
    while issued < len(pool):
        fresh = pool[issued:issued + fresh_per_batch]
        issued += len(fresh)
        rep = pool[rng.integers(0, issued, size=repeats)]
        b = np.concatenate([fresh, rep])[rng.permutation(len(fresh) + repeats)]
        got = t.find_or_put(_dev(b)).cpu().numpy()
        assert_flags_per_key(_ids(b), got, orc.find_or_put(b))


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
@pytest.mark.parametrize("width", [192, 256, 512])
@pytest.mark.parametrize("shared", [False, True])
def test_find_or_put_lookup_export_match_oracle(oracle_lib, scheme, width, shared):
    rng = np.random.default_rng(width + shared)
    w = width // 64
    n = 60_000
    pool = wk.distinct_keys(n, width, seed=50, shared_prefix=shared)
    t = ht.HashTable(int(n / 0.8), scheme, width)
    orc = oracle_lib.OracleTableLong(w)
    _stream_check(t, orc, pool, rng, 15_000, 5_000)
    assert t.sync() == 0 and t.size() == orc.size() == n
    k, _ = t.export()
    assert k.shape == (n, w)
    assert _rows(k) == set(map(tuple, orc.export().tolist()))
    absent = wk.distinct_keys(7000, width, seed=50, start=n + 5, shared_prefix=shared)
    q = np.concatenate([pool[rng.integers(0, n, size=7000)], absent])
    f, _ = t.lookup(_dev(q))
    np.testing.assert_array_equal(f.cpu().numpy(), orc.lookup(q))
    # A second pass over the whole pool finds every key and adds none.
    again = t.find_or_put(_dev(pool)).cpu().numpy()
    assert not again.any() and t.size() == n


@pytest.mark.parametrize("scheme,bits", [("bucket", 6), ("bucket", 12), ("cuckoo", 12), ("cuckoo", 16)])
def test_shared_digests_are_told_apart(oracle_lib, scheme, bits):
    # Keys reduced to `bits`-bit digests: thousands of distinct keys share
    # tags and hash positions, and only the word comparisons separate them.
    rng = np.random.default_rng(bits)
    n = 4000
    pool = wk.distinct_keys(n, 256, seed=61, shared_prefix=True)
    params = dict(digest_bits=bits)
    t = ht.HashTable(1 << 15, scheme, 256, params)
    orc = oracle_lib.OracleTableLong(4)
    _stream_check(t, orc, pool, rng, 1000, 700)
    assert t.sync() == 0 and t.size() == orc.size() == n
    assert _rows(t.export()[0]) == set(map(tuple, pool.tolist()))
    absent = wk.distinct_keys(3000, 256, seed=61, start=n, shared_prefix=True)
    q = np.concatenate([pool[:3000], absent])
    f, _ = t.lookup(_dev(q))
    np.testing.assert_array_equal(f.cpu().numpy(), orc.lookup(q))


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
@pytest.mark.parametrize("width", [192, 512])
def test_edge_keys(oracle_lib, scheme, width):
    # No key value is reserved: all zeros, all ones, and keys one word apart.
    w = width // 64
    ones = 2 ** 64 - 1
    rows = [[0] * w, [ones] * w, [ones] * (w - 1) + [0], [0] * (w - 1) + [ones], [1] + [0] * (w - 1),
            [0] * (w - 1) + [1], [ones] * w, list(range(w)), list(range(w))[::-1]]
    keys = np.array(rows, dtype=np.uint64)
    t = ht.HashTable(64, scheme, width)
    got = t.find_or_put(_dev(keys)).cpu().numpy()
    orc = oracle_lib.OracleTableLong(w)
    assert_flags_per_key(_ids(keys), got, orc.find_or_put(keys))
    assert t.sync() == 0 and t.size() == orc.size() == 8
    f, _ = t.lookup(_dev(keys))
    assert f.cpu().numpy().all()
    assert not t.find_or_put(_dev(keys)).cpu().numpy().any()
    assert _rows(t.export()[0]) == set(map(tuple, keys.tolist()))
    t.clear()
    assert t.size() == 0 and not t.lookup(_dev(keys))[0].cpu().numpy().any()


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_single_key_repeated(scheme):
    # 2^16 copies of one key in one batch: exactly one copy is new.  In the
    # bucket scheme every other copy meets the one claimed header and waits
    # for its publish before comparing.
    key = np.array([[2 ** 64 - 1, 0, 12345, 2 ** 63]], dtype=np.uint64)
    keys = np.repeat(key, 1 << 16, axis=0)
    t = ht.HashTable(1024, scheme, 256)
    assert int(t.find_or_put(_dev(keys)).sum()) == 1
    assert int(t.find_or_put(_dev(keys)).sum()) == 0
    assert t.sync() == 0 and t.size() == 1
    assert t.lookup(_dev(keys))[0].cpu().numpy().all()


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_full_grow_and_checkpoint(oracle_lib, scheme, tmp_path):
    keys = wk.distinct_keys(6000, 320, seed=70)
    # Too small: keys are dropped and the table reports full.
    small = ht.HashTable(16, scheme, 320, dict(num_hashes=1) if scheme == "bucket" else dict(num_hashes=2))
    small.find_or_put(_dev(keys[:2000]))
    assert small.sync() == 3
    # Growth moves every key to new storage; later batches stay exact.
    t = ht.HashTable(2048, scheme, 320)
    orc = oracle_lib.OracleTableLong(5)
    assert_flags_per_key(_ids(keys[:1500]), t.find_or_put(_dev(keys[:1500])).cpu().numpy(),
                         orc.find_or_put(keys[:1500]))
    assert t.sync() == 0 and t.size() == 1500
    t.grow(16384)
    assert t.size() == 1500 and t.lookup(_dev(keys[:1500]))[0].cpu().numpy().all()
    more = keys[1000:6000]
    assert_flags_per_key(_ids(more), t.find_or_put(_dev(more)).cpu().numpy(), orc.find_or_put(more))
    assert t.sync() == 0 and t.size() == orc.size() == 6000
    path = str(tmp_path / "long.npz")
    t.save(path)
    u = ht.HashTable.load(path)
    assert u.key_width == 320 and u.size() == 6000
    assert _rows(u.export()[0]) == set(map(tuple, keys.tolist()))


def test_cuckoo_past_the_key_store_keeps_a_consistent_set():
    # More distinct keys than the key store has rows: winners past its last
    # row give their claims back and leave list records that the insert
    # kernel skips, so every stored key is stored once, came from the input
    # and is found, and the size counts exactly the stored keys.
    keys = wk.distinct_keys(3000, 256, seed=73)
    t = ht.HashTable(64, "cuckoo", 256)
    for lo in range(0, 3000, 1000):
        t.find_or_put(_dev(keys[lo:lo + 1000]))
    assert t.sync() == 3
    # Export into room for four times the size: a key stored twice, or an
    # entry left by a stale list record, would show up as extra entries.
    lib, stream = ht.load(), ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    size = ctypes.c_uint64()
    assert lib.ht_size(t.handle, ctypes.byref(size), stream) == 3       # the size still reads out
    n = size.value
    buf = torch.empty((4 * n + 64, 4), dtype=torch.int64, device="cuda")
    cnt = ctypes.c_uint64()
    st = lib.ht_export(t.handle, ctypes.c_void_p(buf.data_ptr()), None, buf.shape[0], ctypes.byref(cnt), stream)
    assert st == 3 and 0 < cnt.value == n
    ex = buf[:n]
    rows = _rows(ex)
    assert len(rows) == n
    assert rows <= set(map(tuple, keys.tolist()))
    assert t.lookup(ex)[0].cpu().numpy().all()


def test_cuckoo_overflow_and_rebuild_stay_exact(oracle_lib):
    # Three hash functions and short eviction chains at load 0.85: entries
    # spill to the overflow set, synchronising calls rebuild the table with
    # new constants, and the set stays exact throughout.
    keys = wk.distinct_keys(8500, 256, seed=71)
    t = ht.HashTable(10_000, "cuckoo", 256, dict(num_hashes=3, max_evictions=16))
    orc = oracle_lib.OracleTableLong(4)
    rng = np.random.default_rng(3)
    for lo in range(0, 8500, 1700):
        b = np.concatenate([keys[lo:lo + 1700], keys[rng.integers(0, lo + 1700, size=600)]])
        b = b[rng.permutation(len(b))]
        assert_flags_per_key(_ids(b), t.find_or_put(_dev(b)).cpu().numpy(), orc.find_or_put(b))
        assert t.sync() == 0
    assert t.size() == orc.size() == 8500
    assert t.lookup(_dev(keys))[0].cpu().numpy().all()
    st = t.stats()
    assert st["overflow_used"] > 0 or st["rebuilds"] > 0


def test_cuckoo_paper_insertion_rule_parity(oracle_lib):
    # cuckoo_chain_h1 = 1: every long-key chain starts at h_1 (Section 4.1).
    keys = wk.distinct_keys(6000, 256, seed=74)
    t = ht.HashTable(int(6000 / 0.85), "cuckoo", 256, dict(cuckoo_chain_h1=1))
    orc = oracle_lib.OracleTableLong(4)
    rng = np.random.default_rng(4)
    for lo in range(0, 6000, 1500):
        b = np.concatenate([keys[lo:lo + 1500], keys[rng.integers(0, lo + 1500, size=500)]])
        b = b[rng.permutation(len(b))]
        assert_flags_per_key(_ids(b), t.find_or_put(_dev(b)).cpu().numpy(), orc.find_or_put(b))
    assert t.sync() == 0 and t.size() == orc.size() == 6000


def test_large_batch_parity(oracle_lib):
    # 2^21 keys of 256 bits in batches of 2^19, both schemes, against the oracle.
    n = 1 << 21
    fs = wk.fill_stream(n, 1 << 19, 0.25, 256, seed=72)
    for scheme in ("bucket", "cuckoo"):
        t = ht.HashTable(int(n / 0.8), scheme, 256)
        orc = oracle_lib.OracleTableLong(4)
        for b in range(fs.n_batches):
            kb = fs.batch(b)
            got = t.find_or_put(_dev(kb)).cpu().numpy()
            assert_flags_per_key(_ids(kb), got, orc.find_or_put(kb))
        assert t.sync() == 0 and t.size() == n


def test_unsupported_uses_are_rejected():
    for bad in (160, 576, 1024):
        with pytest.raises(ht.HtError):
            ht.HashTable(64, "bucket", bad)
    with pytest.raises(ht.HtError):
        ht.HashTable(64, "bucket", 64, dict(digest_bits=8))          # a long-key knob only
    with pytest.raises(ht.HtError):
        ht.HashTable(64, "bucket", 256, dict(bucket_slots=8))
    t = ht.HashTable(1024, "bucket", 256)
    keys = _dev(wk.distinct_keys(10, 256, seed=1))
    with pytest.raises(ht.HtError):
        ht.ht_find_or_put_append(t.handle, keys, torch.empty((10, 4), dtype=torch.int64, device="cuda"),
                                 torch.zeros(1, dtype=torch.int64, device="cuda"),
                                 torch.empty(10, dtype=torch.uint8, device="cuda"))
    with pytest.raises(ht.HtError):
        ht.ht_multi_find_or_put([t.handle], [(0, keys, torch.empty(10, dtype=torch.uint8, device="cuda"))])


class _DeviceWords:
    """A view of device memory the library owns, for torch to write into."""

    def __init__(self, ptr, nwords):
        self.__cuda_array_interface__ = {"shape": (nwords,), "typestr": "<i8", "data": (ptr, False),
                                         "version": 3, "strides": None}


def test_publish_wait_runs_out_and_reports_timeout():
    """Section 4.2: a reader that meets a claimed, unpublished slot of its
    key's tag must wait for the writer.  Here no writer exists: every header
    of the table is claimed (busy) and never published, with tags 0..3, and
    the digest is cut to 2 bits so every key's tag matches some of them.  The
    wait is bounded by the table's publish_wait_polls: the kernel gives up,
    the lookup finishes, and the next synchronising call returns
    HT_ERR_TIMEOUT.  Nothing on the device waits without a bound."""
    import time
    busy = 1 << 62
    t = ht.HashTable(1024, "bucket", 256, dict(digest_bits=2, publish_wait_polls=64))
    ptr, nbytes = ht.ht_table_words(t.handle)
    nwords = nbytes // 8
    words = torch.as_tensor(_DeviceWords(ptr, nwords), device="cuda")
    words.copy_(busy | (torch.arange(nwords, device="cuda", dtype=torch.int64) & 3))
    torch.cuda.synchronize()
    keys = _dev(wk.distinct_keys(256, 256, seed=5))
    t0 = time.time()
    found, _ = t.lookup(keys)
    torch.cuda.synchronize()
    assert time.time() - t0 < 30
    assert int(found.sum()) == 0
    assert t.sync() == 5                                      # HT_ERR_TIMEOUT
    assert ht.ht_stats(t.handle)["flags"] & 8
    # find-or-put meets the same claimed headers: bounded again, no key stored.
    flags = t.find_or_put(keys)
    torch.cuda.synchronize()
    assert int(flags.sum()) == 0 and t.sync() == 5
    # Cleared, the table works normally again.
    t.clear()
    assert int(t.find_or_put(keys).sum()) == 256
    assert t.sync() == 0 and t.size() == 256
    found, _ = t.lookup(keys)
    assert int(found.sum()) == 256
