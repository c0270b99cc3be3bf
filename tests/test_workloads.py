"""The seeded input generators produce what their docstrings promise."""
import numpy as np
import pytest

from workloads import keys as wk
from workloads import statespace as ss


@pytest.mark.parametrize("width", [32, 64])
def test_distinct_keys_are_distinct_and_valid(width):
    k = wk.distinct_keys(1 << 16, width, seed=5)
    assert len(np.unique(k)) == len(k)
    if width == 32:
        assert k.dtype == np.uint32 and not (k == np.uint32(wk.EMPTY32)).any()
    else:
        assert k.dtype == np.uint64 and (k >> np.uint64(63) == 0).all()
    other = wk.distinct_keys(1 << 12, width, seed=5, start=1 << 16)
    assert len(np.intersect1d(k, other)) == 0


def test_mix32_perm_is_a_bijection_on_a_small_domain():
    # The cycle-walking permutation maps [0, 2^32-1) onto itself; check the
    # top of the domain explicitly (where the reserved value lives).
    x = np.arange((1 << 32) - (1 << 16), (1 << 32) - 1, dtype=np.uint64)
    y = wk.mix32_perm(x, seed=9)
    assert len(np.unique(y)) == len(y)
    assert not (y == wk.EMPTY32).any()


@pytest.mark.parametrize("d", [0.0, 0.25, 0.5])
@pytest.mark.parametrize("width", [32, 64])
def test_fill_stream_shape(d, width):
    n, B = 5000, 1024
    fs = wk.fill_stream(n, B, d, width, seed=3)
    assert len(np.unique(fs.keys)) == n
    assert fs.fresh_counts.sum() == n
    seen = set()
    for b in range(fs.n_batches):
        kb = fs.batch(b).tolist()
        first = set(kb) - seen
        assert len(first) == fs.fresh_counts[b]
        seen |= set(kb)
    if d == 0.0:
        assert fs.n_issued == n
    else:
        assert abs(fs.n_issued - n / (1 - d)) < fs.n_batches + 2


@pytest.mark.parametrize("nb", [1, 2, 5, 100])
def test_fill_stream_prefix_matches_full(nb):
    full = wk.fill_stream(5000, 1024, 0.25, 64, seed=7)
    pre = wk.fill_stream(5000, 1024, 0.25, 64, seed=7, max_batches=nb)
    m = min(nb, full.n_batches)
    assert pre.n_batches == m
    assert np.array_equal(pre.offsets, full.offsets[:m + 1])
    assert np.array_equal(pre.keys, full.keys[:full.offsets[m]])
    assert np.array_equal(pre.fresh_counts, full.fresh_counts[:m])


@pytest.mark.parametrize("width", [192, 256, 512])
@pytest.mark.parametrize("shared", [False, True])
def test_long_keys_distinct_and_span_every_bit(width, shared):
    w = width // 64
    k = wk.distinct_keys(20000, width, seed=4, shared_prefix=shared)
    assert k.shape == (20000, w) and k.dtype == np.uint64
    assert len(np.unique(k, axis=0)) == 20000
    other = wk.distinct_keys(5000, width, seed=4, start=20000, shared_prefix=shared)
    both = np.concatenate([k, other])
    assert len(np.unique(both, axis=0)) == 25000           # disjoint index ranges, disjoint keys
    assert (k[:, -1] >> np.uint64(63)).any()                 # the top bit of the last word is used
    if shared:
        assert len(np.unique(k[:, :-1], axis=0)) <= 4 ** (w - 1)   # many keys share every word but the last
        assert set(np.unique(k[:, 0]).tolist()) <= {0, 1, 2, 3}
    else:
        assert (k[:, 0] >> np.uint64(63)).any()


def test_long_fill_stream_rows():
    fs = wk.fill_stream(3000, 512, 0.4, 256, seed=6)
    assert fs.keys.shape[1] == 4
    assert len(np.unique(fs.keys, axis=0)) == 3000 and fs.fresh_counts.sum() == 3000
    with pytest.raises(ValueError):
        wk.distinct_keys(10, 160, seed=1)


def test_lookup_batch_split():
    keys, present = wk.lookup_batch(1000, 2001, 64, seed=1)
    stored = set(wk.distinct_keys(1000, 64, seed=1).tolist())
    assert present.sum() == 1000
    for k, p in zip(keys.tolist(), present.tolist()):
        assert (k in stored) == bool(p)


def test_models_fit_their_format():
    m = ss.config3_model()
    assert m.C == 12 and m.total_bits == 60 and m.key_width == 64 and m.P == 4
    assert (m.deg[:12, :32] >= 1).all() and (m.deg[:12, :32] <= 3).all()
    for c in range(m.C):
        for u in range(32):
            for j in range(m.deg[c, u]):
                lab = int(m.lab[c, u, j])
                assert lab == 0 or c in m.pairs[lab - 1]
    ms = ss.batched_models(16, seed=2)
    for mm in ms:
        assert 6 <= mm.C <= 10 and mm.total_bits <= 63


def test_device_keys_match_the_host_stream():
    torch = pytest.importorskip("torch")
    from workloads import device_keys as dk
    for seed, start, n in [(0, 0, 1000), (7, 123456789, 5000), (2 ** 40 + 3, 2 ** 62 - 10, 10)]:
        host = wk.distinct_keys(n, 64, seed, start=start)
        dev = dk.distinct_keys_dev(n, seed, start=start).numpy().view(np.uint64)
        np.testing.assert_array_equal(dev, host)


def test_device_fill_batches_shape():
    torch = pytest.importorskip("torch")
    from workloads import device_keys as dk
    n, B, d = 10_000, 1024, 0.25
    batches, fresh = dk.fill_batches_dev(n, B, d, seed=3, device="cpu")
    assert sum(fresh) == n
    allk = torch.cat(batches).numpy()
    assert len(np.unique(allk)) == n
    assert all(len(b) == B for b in batches[:-1])
    seen = set()
    for b, f in zip(batches, fresh):
        s = set(b.tolist())
        assert len(s - seen) == f             # exactly f keys new to the stream
        seen |= s


def test_device_mix32_matches_the_host_permutation():
    torch = pytest.importorskip("torch")
    from workloads import device_keys as dk
    for seed in (0, 1, 12345):
        x = np.concatenate([np.arange(0, 5000), np.arange(2 ** 32 - 5000, 2 ** 32 - 1)]).astype(np.uint64)
        host = wk.mix32_perm(x, seed)
        dev = dk.mix32_perm_dev(torch.from_numpy(x.astype(np.int64)), seed).numpy().astype(np.uint64)
        np.testing.assert_array_equal(dev, host)


def test_multiplicity_sequence_shape():
    torch = pytest.importorskip("torch")
    from workloads import device_keys as dk
    n = 200_000
    for mult in (1, 10, 100):
        k = dk.multiplicity_sequence_dev(n, mult, seed=5, device="cpu")
        assert k.dtype == torch.int32 and k.numel() == n
        u = np.unique(k.numpy().view(np.uint32))
        assert 0xFFFFFFFF not in u
        rng = round(n / mult)
        assert len(u) <= rng
        # Uniform draws: the expected number of distinct values is rng (1 - e^-mult).
        exp = rng * (1 - np.exp(-mult))
        assert abs(len(u) - exp) < 5 * np.sqrt(exp) + 10


def test_batch_flag_check_accepts_exactly_once_and_catches_mistakes():
    # The full-size fill test's checker, on a small stream with flags made
    # from the generator's fresh keys (first occurrence flagged).
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from gpu_util import check_batch_flags
    fs = wk.fill_stream(20_000, 4096, 0.25, 64, seed=5)
    rng = np.random.default_rng(0)
    issued = 0
    for b in range(fs.n_batches):
        kb = fs.batch(b)
        nf = int(fs.fresh_counts[b])
        fresh = wk.distinct_keys(nf, 64, seed=5, start=issued)
        issued += nf
        flags = np.zeros(len(kb), dtype=np.uint8)
        _, first = np.unique(kb, return_index=True)
        flags[first[np.isin(kb[first], fresh)]] = 1
        pos = rng.integers(0, len(kb), size=500)
        assert check_batch_flags(kb, flags, fresh, pos) == []
        if b == 1:
            f2 = flags.copy()
            f2[np.nonzero(f2)[0][0]] = 0                       # a new key left unflagged
            assert check_batch_flags(kb, f2, fresh, np.arange(len(kb)))
            f3 = flags.copy()
            dup = np.nonzero(~np.isin(kb, fresh))[0][0]          # an old key flagged new
            f3[dup] = 1
            assert check_batch_flags(kb, f3, fresh, np.array([dup]))


def test_exact_batch_flag_check_accepts_exactly_once_and_catches_mistakes():
    # The full-size fill test's checker of every key of every batch, on a
    # small stream with flags made from the generator's fresh keys.
    import sys, os
    sys.path.insert(0, os.path.dirname(os.path.abspath(__file__)))
    from gpu_util import check_batch_flags_exact
    fs = wk.fill_stream(20_000, 4096, 0.25, 64, seed=6)
    issued = 0
    for b in range(fs.n_batches):
        kb = fs.batch(b)
        nf = int(fs.fresh_counts[b])
        fresh = wk.distinct_keys(nf, 64, seed=6, start=issued)
        issued += nf
        flags = np.zeros(len(kb), dtype=np.uint8)
        _, first = np.unique(kb, return_index=True)
        flags[first[np.isin(kb[first], fresh)]] = 1
        # any occurrence may carry the flag: move some to the last occurrence
        _, last = np.unique(kb[::-1], return_index=True)
        last = len(kb) - 1 - last
        fl2 = flags.copy()
        moved = first[np.isin(kb[first], fresh)][:50]
        fl2[moved] = 0
        fl2[last[np.searchsorted(np.unique(kb), kb[moved])]] = 1
        assert check_batch_flags_exact(kb, flags, fresh) == []
        assert check_batch_flags_exact(kb, fl2, fresh) == []
        if b == 1:
            f2 = flags.copy()
            f2[np.nonzero(f2)[0][0]] = 0                        # a new key left unflagged
            assert check_batch_flags_exact(kb, f2, fresh)
            f3 = flags.copy()
            f3[np.nonzero(~np.isin(kb, fresh))[0][0]] = 1       # an old key flagged new
            assert check_batch_flags_exact(kb, f3, fresh)
            f4 = f3.copy()
            f4[np.nonzero(flags)[0][0]] = 0                     # both at once: the count still matches
            assert int(f4.sum()) == nf and check_batch_flags_exact(kb, f4, fresh)
            rep = np.nonzero(np.isin(kb, fresh) & (flags == 0))[0][0]
            f5 = flags.copy()
            f5[rep] = 1                                         # a fresh key flagged twice ...
            other = np.nonzero(flags & (kb != kb[rep]))[0][0]
            f5[other] = 0                                       # ... and another left out
            assert int(f5.sum()) == nf and check_batch_flags_exact(kb, f5, fresh)
