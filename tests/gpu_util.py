"""Helpers for the GPU parity tests: marshal numpy inputs to CUDA tensors and
compare CUDA results with the oracle under the rules of a set/map."""
import numpy as np
import torch


def to_dev(a):
    a = np.ascontiguousarray(a)
    if a.dtype == np.uint64:
        a = a.view(np.int64)
    elif a.dtype == np.uint32:
        a = a.view(np.int32)
    return torch.from_numpy(a).cuda()


def to_np(t, dtype=None):
    a = t.cpu().numpy()
    if dtype is not None:
        a = a.view(dtype)
    return a


def keys_np(t, key_width):
    return to_np(t, np.uint32 if key_width == 32 else np.uint64)


def assert_flags_per_key(keys, got, expected):
    """Among equal keys of one batch exactly as many flags as the oracle's
    (which flags the first occurrence); which occurrence is unspecified."""
    got = np.asarray(got).astype(np.int64)
    expected = np.asarray(expected).astype(np.int64)
    assert set(np.unique(got).tolist()) <= {0, 1}
    uk, inv = np.unique(np.asarray(keys), return_inverse=True)
    sg = np.bincount(inv, weights=got, minlength=len(uk))
    se = np.bincount(inv, weights=expected, minlength=len(uk))
    bad = np.nonzero(sg != se)[0]
    assert len(bad) == 0, "per-key flag counts differ for %d keys, e.g. %s: gpu %s oracle %s" % (
        len(bad), uk[bad[:3]], sg[bad[:3]], se[bad[:3]])


def assert_same_set(gpu_keys, oracle_keys):
    a = np.sort(np.asarray(gpu_keys).astype(np.uint64))
    b = np.sort(np.asarray(oracle_keys).astype(np.uint64))
    assert len(a) == len(b), "sizes differ: gpu %d oracle %d" % (len(a), len(b))
    assert len(np.unique(a)) == len(a), "a key is stored twice"
    assert np.array_equal(a, b)


def check_batch_flags(batch, flags, fresh, sample_pos):
    """Exactly-once check of one find-or-put batch at any size, without the
    oracle's whole history: `fresh` holds the keys issued for the first time
    in this batch (from the generator), `sample_pos` positions of the batch
    to check.  For each sampled key the flags over all its occurrences in the
    batch must sum to 1 if it is fresh, else 0; and the batch's flags must
    sum to the number of fresh keys.  Returns a list of problems."""
    batch = np.asarray(batch)
    flags = np.asarray(flags).astype(np.int64)
    bad = []
    if set(np.unique(flags).tolist()) - {0, 1}:
        bad.append("flags other than 0/1")
    if int(flags.sum()) != len(fresh):
        bad.append("batch flags %d, fresh keys %d" % (int(flags.sum()), len(fresh)))
    # Membership by binary search in sorted arrays (np.isin of a small array
    # in a large one is far slower): each batch element's sampled key, if
    # any, then the flag count per sampled key; fresh keys likewise.
    kk = np.unique(batch[np.asarray(sample_pos)])
    at = np.minimum(np.searchsorted(kk, batch), len(kk) - 1)
    hit = kk[at] == batch
    per_key = np.bincount(at[hit], weights=flags[hit], minlength=len(kk)).astype(np.int64)
    sf = np.sort(np.asarray(fresh))
    if len(sf):
        want = (sf[np.minimum(np.searchsorted(sf, kk), len(sf) - 1)] == kk).astype(np.int64)
    else:
        want = np.zeros(len(kk), dtype=np.int64)
    wrong = np.nonzero(per_key != want)[0]
    if len(wrong):
        bad.append("%d sampled keys with wrong flag counts, e.g. %s: %s (want %s)" % (
            len(wrong), kk[wrong[:3]], per_key[wrong[:3]], want[wrong[:3]]))
    return bad


def check_batch_flags_exact(batch, flags, fresh):
    """The complete exactly-once check of one find-or-put batch, for every key
    of it: the flagged keys, sorted, must equal the batch's fresh keys
    (those issued for the first time in it), sorted.  Since the fresh keys
    are distinct, that says each fresh key is flagged exactly once and no
    other key is flagged -- the same facts as the oracle's per-key flag
    counts, for a stream whose earlier batches were exact.  Returns a list
    of problems."""
    batch = np.asarray(batch)
    flags = np.asarray(flags)
    bad = []
    if set(np.unique(flags).tolist()) - {0, 1}:
        bad.append("flags other than 0/1")
    flagged = np.sort(batch[flags.astype(bool)])
    want = np.sort(np.asarray(fresh))
    if len(flagged) != len(want):
        bad.append("batch flags %d, fresh keys %d" % (len(flagged), len(want)))
    elif not np.array_equal(flagged, want):
        at = np.nonzero(flagged != want)[0]
        bad.append("%d flagged keys differ from the fresh keys, e.g. %s vs %s" % (
            len(at), flagged[at[:3]], want[at[:3]]))
    return bad
