"""The benchmark's headline fill at full size, in the launch configuration the
benchmark times: 2^27 distinct random 64-bit keys (seed 2024) into a table of
ceil(2^27 / 0.8) slots, find-or-put batches of 2^24 keys with 25% repeats,
both schemes, default parameters, one ht_find_or_put per batch.

Replaying the oracle over the whole history takes minutes, so the check uses
what the generator knows exactly: the keys it issues for the first time in
each batch.  For EVERY batch, the flagged keys, sorted, must equal that
batch's fresh keys, sorted (gpu_util.check_batch_flags_exact): each key new
to the table is flagged exactly once and no other key is flagged -- the
oracle's per-key flag counts, for every key of every batch.  At the end the
table holds exactly 2^27 keys, its export (sorted) equals all 2^27 generated
keys (sorted), and lookups of 2^20 issued and 2^20 never-issued keys are
exact.
"""
import numpy as np
import pytest
import torch

import paper_1712_09494_gb300 as ht
from workloads import keys as wk

from gpu_util import check_batch_flags_exact

pytestmark = pytest.mark.gpu

N, B, DUP, SEED, LF = 1 << 27, 1 << 24, 0.25, 2024, 0.8
M = 1 << 20           # lookups of each kind
DEV = "cuda"


@pytest.fixture(scope="module")
def stream():
    from paper_1712_09494_gb300 import _build
    _build.build()
    ht.load()
    return wk.fill_stream(N, B, DUP, 64, seed=SEED)


@pytest.fixture(scope="module")
def all_keys_sorted():
    return np.sort(wk.distinct_keys(N, 64, seed=SEED))


@pytest.mark.parametrize("scheme", ["bucket", "cuckoo"])
def test_full_size_fill_is_exactly_once(stream, all_keys_sorted, scheme):
    fs = stream
    dev = torch.device(DEV)
    keys_d = torch.from_numpy(fs.keys.view(np.int64)).to(dev)
    t = ht.HashTable(int(np.ceil(N / LF)), scheme, 64)
    flags = torch.empty(B, dtype=torch.uint8, device=dev)
    issued = 0
    for b in range(fs.n_batches):
        lo, hi = int(fs.offsets[b]), int(fs.offsets[b + 1])
        ht.ht_find_or_put(t.handle, keys_d[lo:hi], flags[:hi - lo])
        f = flags[:hi - lo].cpu().numpy()
        nf = int(fs.fresh_counts[b])
        fresh = fs.keys[lo:hi][:0] if nf == 0 else wk.distinct_keys(nf, 64, seed=SEED, start=issued)
        problems = check_batch_flags_exact(fs.keys[lo:hi], f, fresh)
        assert not problems, (scheme, b, problems)
        issued += nf
    del keys_d
    assert issued == N
    assert t.sync() == 0 and t.size() == N
    exported, _ = t.export()
    got = np.sort(exported.cpu().numpy().view(np.uint64))
    del exported
    assert len(got) == N and np.array_equal(got, all_keys_sorted), scheme
    del got
    rng = np.random.default_rng(7)
    present = wk.distinct_keys(M, 64, seed=SEED, start=int(rng.integers(0, N - M)))
    absent = wk.distinct_keys(M, 64, seed=SEED, start=N + 1)
    q = torch.from_numpy(np.concatenate([present, absent]).view(np.int64)).to(dev)
    found, _ = t.lookup(q)
    found = found.cpu().numpy()
    assert found[:M].all() and not found[M:].any()
    t.close()
