"""The allocation-free Cuckoo find-or-put matches the regular one.

ht_cuckoo_find_or_put_noalloc serves callers that cannot call cudaMalloc
(all device memory reserved up front, or a path where allocation is not
allowed): they pass the table memory, and the per-call scratch comes from a
static device array inside the library.  Here it is called through the C ABI
on caller-owned torch buffers, twice in a row on the same table, and each
call's flags and the stored set are compared with ht_find_or_put on a
regular Cuckoo table given the same keys.  The comparison is the one every
parity test uses: per distinct key, the same number of is_new flags.  Further
cases cover what only the caller's state block reports: a table too small for
its keys (keys dropped, none invented), a reserved key (skipped, status bit
set) and a second table with another seed after the first.

This file is collected last on purpose, so that a run stopping at the first
failure has already run every other test.
"""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import keys as wk

from gpu_util import assert_flags_per_key, assert_same_set, keys_np, to_dev, to_np

pytestmark = pytest.mark.gpu

EMPTY = np.uint64(0xFFFFFFFFFFFFFFFF)
# State block layout (include/ht.h): counters, then a 101-word stash at byte
# 128 and a 64-word overflow area at byte 1152.
STASH_AT, STASH_WORDS = 128, 101
OVF_AT, OVF_WORDS = 1152, 64
FLAG_INVALID, FLAG_OVERFLOW, FLAG_DROPPED = 1, 2, 4


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


def _state_counters(state):
    c = to_np(state[:32].clone(), np.uint64)
    w = to_np(state[16:32].clone(), np.uint32)
    return dict(size=int(c[0]), dropped=int(c[1]), stash_used=int(w[0]), ovf_used=int(w[1]), flags=int(w[2]))


def _held_keys(slots, state):
    words = to_np(slots, np.uint64)
    stash = to_np(state[STASH_AT:STASH_AT + STASH_WORDS * 8].clone(), np.uint64)
    overflow = to_np(state[OVF_AT:OVF_AT + OVF_WORDS * 8].clone(), np.uint64)
    held = np.concatenate([words, stash, overflow])
    return held[held != EMPTY]


def _noalloc(slots, state, seed, keys, is_new=None, reset=False):
    ht.ht_cuckoo_find_or_put_noalloc(slots, state, seed, keys, is_new, reset=reset)


def test_noalloc_matches_find_or_put_on_two_calls():
    n_distinct = 150_000
    fs = wk.fill_stream(n_distinct, 120_000, 0.4, 64, seed=21)
    assert fs.n_batches >= 2
    nslots = int(n_distinct / 0.8)
    slots = torch.empty(nslots, dtype=torch.int64, device="cuda")
    state = torch.empty(ht.NOALLOC_STATE_BYTES, dtype=torch.uint8, device="cuda")
    ref = ht.HashTable(nslots, "cuckoo", 64)
    for call in range(2):
        kb = to_dev(fs.batch(call))
        assert kb.numel() <= ht.NOALLOC_MAX_BATCH
        got = torch.empty(kb.numel(), dtype=torch.uint8, device="cuda")
        _noalloc(slots, state, 12345, kb, got, reset=(call == 0))
        exp = ref.find_or_put(kb)
        torch.cuda.synchronize()
        kn = fs.batch(call)
        assert_flags_per_key(kn, to_np(got), to_np(exp))
        assert int(got.sum()) == fs.fresh_counts[call]
        c = _state_counters(state)
        assert c["size"] == ref.size()       # stored keys
        assert c["dropped"] == 0 and c["flags"] == 0
    # The stored sets agree: read the caller's table words directly.
    k, _ = ref.export()
    assert_same_set(_held_keys(slots, state), keys_np(k, 64))
    # A third call without flags (is_new = NULL) stores the same keys.
    kb = to_dev(fs.batch(2))
    _noalloc(slots, state, 12345, kb)
    ref.find_or_put(kb)
    torch.cuda.synchronize()
    k, _ = ref.export()
    assert_same_set(_held_keys(slots, state), keys_np(k, 64))
    assert _state_counters(state)["size"] == ref.size()


def test_noalloc_second_table_and_seed_after_the_first():
    """Each call starts from an empty dedup set whatever the previous call on
    another table left: a second table with another seed matches a regular
    table given the same keys."""
    for seed, tseed in ((7, 901), (8, 902)):
        keys = wk.distinct_keys(60_000, 64, seed=tseed)
        rng = np.random.default_rng(tseed)
        batch = np.concatenate([keys, keys[rng.integers(0, len(keys), 20_000)]])
        rng.shuffle(batch)
        nslots = 80_000
        slots = torch.empty(nslots, dtype=torch.int64, device="cuda")
        state = torch.empty(ht.NOALLOC_STATE_BYTES, dtype=torch.uint8, device="cuda")
        got = torch.empty(len(batch), dtype=torch.uint8, device="cuda")
        _noalloc(slots, state, seed, to_dev(batch), got, reset=True)
        ref = ht.HashTable(nslots, "cuckoo", 64)
        exp = ref.find_or_put(to_dev(batch))
        torch.cuda.synchronize()
        assert_flags_per_key(batch, to_np(got), to_np(exp))
        assert_same_set(_held_keys(slots, state), keys)


def test_noalloc_tiny_table_drops_keys_and_invents_none():
    """More distinct keys than slots + stash + overflow: the surplus is
    counted as dropped, every held key is one of the inputs, held once, and
    the per-key flags count each held key exactly once."""
    nslots = 512
    keys = wk.distinct_keys(2000, 64, seed=77)
    assert nslots + STASH_WORDS + OVF_WORDS < len(keys)
    slots = torch.empty(nslots, dtype=torch.int64, device="cuda")
    state = torch.empty(ht.NOALLOC_STATE_BYTES, dtype=torch.uint8, device="cuda")
    got = torch.empty(len(keys), dtype=torch.uint8, device="cuda")
    _noalloc(slots, state, 3, to_dev(keys), got, reset=True)
    torch.cuda.synchronize()
    c = _state_counters(state)
    held = _held_keys(slots, state)
    assert len(np.unique(held)) == len(held), "a key is held twice"
    assert np.isin(held, keys).all(), "a held key is not an input"
    assert c["size"] == len(held)
    assert c["dropped"] == len(keys) - len(held) > 0
    assert c["flags"] & FLAG_DROPPED and c["flags"] & FLAG_OVERFLOW
    # Every input was flagged new once (all distinct, all absent before);
    # a dropped key keeps its flag: it was new, but could not be stored.
    assert int(got.sum()) == len(keys)


def test_noalloc_reserved_key_is_skipped_and_reported_in_the_state():
    keys = wk.distinct_keys(5000, 64, seed=78)
    batch = keys.copy()
    batch[17] = np.uint64(1 << 63) | np.uint64(5)       # top bit set: reserved
    slots = torch.empty(8192, dtype=torch.int64, device="cuda")
    state = torch.empty(ht.NOALLOC_STATE_BYTES, dtype=torch.uint8, device="cuda")
    got = torch.empty(len(batch), dtype=torch.uint8, device="cuda")
    _noalloc(slots, state, 4, to_dev(batch), got, reset=True)
    torch.cuda.synchronize()
    c = _state_counters(state)
    assert c["flags"] & FLAG_INVALID
    g = to_np(got)
    assert g[17] == 0 and int(g.sum()) == len(batch) - 1
    assert_same_set(_held_keys(slots, state), np.delete(keys, 17))
    # The status bit is sticky until a reset clears it.
    _noalloc(slots, state, 4, to_dev(keys[:10]), None)
    torch.cuda.synchronize()
    assert _state_counters(state)["flags"] & FLAG_INVALID
    _noalloc(slots, state, 4, to_dev(keys[:0]), None, reset=True)
    torch.cuda.synchronize()
    assert _state_counters(state) == dict(size=0, dropped=0, stash_used=0, ovf_used=0, flags=0)


def test_noalloc_rejects_oversized_batch_and_bad_arguments():
    slots = torch.empty(1024, dtype=torch.int64, device="cuda")
    state = torch.empty(ht.NOALLOC_STATE_BYTES, dtype=torch.uint8, device="cuda")
    big = torch.zeros(ht.NOALLOC_MAX_BATCH + 1, dtype=torch.int64, device="cuda")
    with pytest.raises(ValueError):
        _noalloc(slots, state, 1, big)
    lib = ht.load()
    # The C entry point rejects the same sizes on its own.
    assert lib.ht_cuckoo_find_or_put_noalloc(slots.data_ptr(), 1024, state.data_ptr(), 1, big.data_ptr(),
                                             big.numel(), None, 0, None) == 1
    assert lib.ht_cuckoo_find_or_put_noalloc(None, 1024, None, 1, None, 0, None, 1, None) == 1
    # An empty batch with reset only clears.
    _noalloc(slots, state, 1, big[:0], reset=True)
    torch.cuda.synchronize()
    assert _state_counters(state)["size"] == 0
