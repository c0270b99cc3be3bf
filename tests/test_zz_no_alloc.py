"""The allocation-free Cuckoo find-or-put matches the regular one.

ht_cuckoo_find_or_put_noalloc serves callers that cannot call cudaMalloc
(all device memory reserved up front, or a path where allocation is not
allowed): they pass the table memory, and the per-call scratch comes from a
static device array inside the library.  Here it is called through the C ABI
on caller-owned torch buffers, twice in a row on the same table, and each
call's flags and the stored set are compared with ht_find_or_put on a
regular Cuckoo table given the same keys.  The comparison is the one every
parity test uses: per distinct key, the same number of is_new flags.

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


@pytest.fixture(scope="module", autouse=True)
def _lib():
    from paper_1712_09494_gb300 import _build
    _build.build()
    assert torch.cuda.is_available()
    ht.load()


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
        rc = ht.ht_cuckoo_find_or_put_noalloc(slots, state, 12345, kb, got, reset=(call == 0))
        assert rc == 0
        exp = ref.find_or_put(kb)
        torch.cuda.synchronize()
        kn = fs.batch(call)
        assert_flags_per_key(kn, to_np(got), to_np(exp))
        assert int(got.sum()) == fs.fresh_counts[call]
        counters = to_np(state[:16].clone(), np.uint64)
        assert int(counters[0]) == ref.size()      # stored keys
        assert int(counters[1]) == 0                # nothing dropped
    # The stored sets agree: read the caller's table words directly.
    words = to_np(slots, np.uint64)
    stash = to_np(state[128:128 + 101 * 8].clone(), np.uint64)
    overflow = to_np(state[1152:1152 + 64 * 8].clone(), np.uint64)
    held = np.concatenate([words, stash, overflow])
    held = held[held != np.uint64(0xFFFFFFFFFFFFFFFF)]
    k, _ = ref.export()
    assert_same_set(held, keys_np(k, 64))


def test_noalloc_rejects_oversized_batch_and_bad_arguments():
    slots = torch.empty(1024, dtype=torch.int64, device="cuda")
    state = torch.empty(ht.NOALLOC_STATE_BYTES, dtype=torch.uint8, device="cuda")
    big = torch.zeros(ht.NOALLOC_MAX_BATCH + 1, dtype=torch.int64, device="cuda")
    assert ht.ht_cuckoo_find_or_put_noalloc(slots, state, 1, big) == 1
    lib = ht.load()
    assert lib.ht_cuckoo_find_or_put_noalloc(None, 1024, None, 1, None, 0, None, 1, None) == 1
    # An empty batch with reset only clears.
    assert ht.ht_cuckoo_find_or_put_noalloc(slots, state, 1, big[:0], reset=True) == 0
    torch.cuda.synchronize()
    assert int(to_np(state[:8].clone(), np.uint64)[0]) == 0
