"""The benchmark's headline fill at full size, in the launch configuration the
benchmark times: 2^27 distinct random 64-bit keys (seed 2024) into a table of
ceil(2^27 / 0.8) slots, find-or-put batches of 2^24 keys with 25% repeats,
both schemes, default parameters, one ht_find_or_put per batch.

Replaying the oracle over the whole history takes minutes, so the check uses
what holds at any size (gpu_util.check_batch_flags): every batch flags
exactly as many keys as the generator issued fresh in it, and in three
batches, for 4096 sampled keys each, the flags over all of a key's
occurrences are 1 for a key fresh in that batch and 0 otherwise.  The table
ends with exactly 2^27 keys, and sampled lookups of issued and never-issued
keys are exact.
"""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import keys as wk

from gpu_util import check_batch_flags

pytestmark = pytest.mark.gpu

N, B, DUP, SEED, LF = 1 << 27, 1 << 24, 0.25, 2024, 0.8
M = 1 << 20           # sampled lookups of each kind
DEV = "cuda"


@pytest.fixture(scope="module")
def stream():
    from paper_1712_09494_gb300 import _build
    _build.build()
    ht.load()
    return wk.fill_stream(N, B, DUP, 64, seed=SEED)


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_full_size_fill_is_exactly_once(stream, scheme):
    fs = stream
    dev = torch.device(DEV)
    keys_d = torch.from_numpy(fs.keys.view(np.int64)).to(dev)
    t = ht.HashTable(int(np.ceil(N / LF)), scheme, 64)
    flags = torch.empty(B, dtype=torch.uint8, device=dev)
    rng = np.random.default_rng(7)
    checked = {0, fs.n_batches // 2, fs.n_batches - 1}
    issued = 0
    for b in range(fs.n_batches):
        lo, hi = int(fs.offsets[b]), int(fs.offsets[b + 1])
        ht.ht_find_or_put(t.handle, keys_d[lo:hi], flags[:hi - lo])
        f = flags[:hi - lo].cpu().numpy()
        nf = int(fs.fresh_counts[b])
        if b in checked:
            fresh = wk.distinct_keys(nf, 64, seed=SEED, start=issued)
            problems = check_batch_flags(fs.keys[lo:hi], f, fresh, rng.integers(0, hi - lo, size=4096))
            assert not problems, (scheme, b, problems)
        else:
            assert int(f.sum()) == nf, (scheme, b)
        issued += nf
    assert issued == N
    assert t.sync() == 0 and t.size() == N
    m = M
    present = wk.distinct_keys(m, 64, seed=SEED, start=int(rng.integers(0, N - m)))
    absent = wk.distinct_keys(m, 64, seed=SEED, start=N + 1)
    q = torch.from_numpy(np.concatenate([present, absent]).view(np.int64)).to(dev)
    found, _ = t.lookup(q)
    found = found.cpu().numpy()
    assert found[:m].all() and not found[m:].any()
    t.close()
