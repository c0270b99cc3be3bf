"""Seeded key streams.

The paper benchmarks sequences of integers in which each value may occur
several times (Section 5.2: random sequences of 10^8 integers whose value
range sets the mean multiplicity; model-checking sequences with mean
multiplicity 5-8, Section 6).  Those files are not available, so these
generators produce streams of the same shape:

* ``distinct_keys`` -- n distinct pseudo-random keys, from a bijection of the
  index range, so disjoint index ranges give disjoint key sets.
* ``fill_stream``   -- a stream of find-or-put batches that fills a table
  with exactly ``n_distinct`` keys; each batch holds (1-d)*B fresh keys and
  d*B repeats drawn uniformly from the keys issued so far (earlier batches
  and this batch's fresh keys), shuffled.
* ``lookup_batch``  -- a query batch, half keys present and half absent.

Reserved words: for 32-bit keys 0xFFFFFFFF is the empty marker; for 64-bit
keys the top bit is reserved.  No generator here ever emits them.
"""
import numpy as np

EMPTY32 = 0xFFFFFFFF
KEY_MASK63 = (1 << 63) - 1

_M63 = np.uint64(KEY_MASK63)
_M32 = np.uint64(0xFFFFFFFF)


def mix63_perm(x, seed=0):
    """A bijection of [0, 2^63): odd multiplies mod 2^63 and xor-shifts.

    Each step is invertible on 63-bit words, so distinct inputs give distinct
    outputs.  Used only to make seeded, distinct, uniform-looking keys.
    """
    x = np.asarray(x, dtype=np.uint64)
    s = np.uint64((seed * 0x9E3779B97F4A7C15 + 0x632BE59BD9B4E019) & KEY_MASK63)
    with np.errstate(over="ignore"):
        z = (x + s) & _M63
        z = (z * np.uint64(0xD6E8FEB86659FD93)) & _M63
        z ^= z >> np.uint64(29)
        z = (z * np.uint64(0xA0761D6478BD642F)) & _M63
        z ^= z >> np.uint64(32)
        z = (z * np.uint64(0xE7037ED1A0B428DB)) & _M63
        z ^= z >> np.uint64(29)
    return z


def _perm32_once(z, s):
    with np.errstate(over="ignore"):
        z = (z + s) & _M32
        z = (z * np.uint64(0x7FEB352D)) & _M32
        z ^= z >> np.uint64(15)
        z = (z * np.uint64(0x846CA68B)) & _M32
        z ^= z >> np.uint64(16)
    return z


def mix32_perm(x, seed=0):
    """A bijection of [0, 2^32 - 1) (0xFFFFFFFF excluded by cycle walking).

    A 32-bit permutation is applied until the result leaves the reserved
    value; restricted to a subset, cycle walking stays a bijection.
    """
    x = np.asarray(x, dtype=np.uint64) & _M32
    s = np.uint64((seed * 0x9E3779B9 + 0x85EBCA6B) & 0xFFFFFFFF)
    z = _perm32_once(x, s)
    bad = z == np.uint64(EMPTY32)
    while bad.any():
        z[bad] = _perm32_once(z[bad], s)
        bad = z == np.uint64(EMPTY32)
    return z


def _word_mix(x, salt):
    """SplitMix64-style finaliser over the full 64-bit range (not a bijection
    requirement here: these words only fill out long keys)."""
    with np.errstate(over="ignore"):
        z = np.asarray(x, dtype=np.uint64) + np.uint64(salt)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        return z ^ (z >> np.uint64(31))


def long_words(width):
    """Words per key of a long-key width (64 * W, W = 3..8), else None."""
    if width % 64 == 0 and 3 <= width // 64 <= 8:
        return width // 64
    return None


def distinct_keys(n, width, seed, start=0, shared_prefix=False):
    """Keys ``start .. start+n-1`` of the seeded stream; all distinct.

    width 64 -> uint64 in [0, 2^63); width 32 -> uint32 != 0xFFFFFFFF
    (indices must stay below 2^32 - 1).  width 64*W (W = 3..8) -> (n, W)
    uint64 rows over the full 64-bit range of every word: the last word is
    a bijection of the index (so rows are distinct) and the others are
    mixed from the index -- or, with ``shared_prefix``, drawn from 4 values
    each, so that many keys agree on every word but the last.
    """
    idx = np.arange(start, start + n, dtype=np.uint64)
    if width == 64:
        return mix63_perm(idx, seed)
    if width == 32:
        if start + n > EMPTY32:
            raise ValueError("32-bit key stream holds at most 2^32-1 keys")
        return mix32_perm(idx, seed).astype(np.uint32)
    w = long_words(width)
    if w is None:
        raise ValueError("width must be 32, 64 or 64*W with W in 3..8")
    out = np.empty((n, w), dtype=np.uint64)
    for j in range(w - 1):
        v = _word_mix(idx, (seed * 0x632BE59BD9B4E019 + 0x9E3779B97F4A7C15 * (j + 1)) & ((1 << 64) - 1))
        out[:, j] = v & np.uint64(3) if shared_prefix else v
    # Bit 63 of the last word comes from the index too, so every word spans 64 bits.
    last = mix63_perm(idx, seed + 17)
    top = (_word_mix(idx, seed ^ 0x5851F42D4C957F2D) >> np.uint64(63)) << np.uint64(63)
    out[:, w - 1] = last | top
    return out


class FillStream:
    """A find-or-put stream: concatenated keys plus per-batch bookkeeping."""

    def __init__(self, keys, offsets, fresh_counts, n_distinct, width):
        self.keys = keys                    # all batches, issue order
        self.offsets = offsets              # batch b is keys[offsets[b]:offsets[b+1]]
        self.fresh_counts = fresh_counts    # number of first-time keys per batch
        self.n_distinct = n_distinct
        self.width = width

    @property
    def n_batches(self):
        return len(self.offsets) - 1

    def batch(self, b):
        return self.keys[self.offsets[b]:self.offsets[b + 1]]

    @property
    def n_issued(self):
        return int(self.offsets[-1])


def fill_stream(n_distinct, batch, dup_rate, width, seed, max_batches=None):
    """Batches that take an empty table to exactly ``n_distinct`` keys.

    Batch b holds f = round((1-d)*B) fresh keys (fewer in the last batch) and
    round(f*d/(1-d)) repeats drawn uniformly from every key issued up to and
    including this batch's fresh ones, so repeats occur both across and
    within batches.  Each batch is shuffled.

    ``max_batches`` stops after that many batches; the batches made are the
    same as the full stream's first ones (fresh key i depends only on i and
    the random draws come in the same order), so a CPU sample of a large
    stream need not generate all of it.
    """
    if not 0.0 <= dup_rate < 1.0:
        raise ValueError("dup_rate must be in [0, 1)")
    rng = np.random.Generator(np.random.PCG64(seed))
    per_batch_fresh = max(1, int(round(batch * (1.0 - dup_rate))))
    n_fresh = n_distinct if max_batches is None else min(n_distinct, max_batches * per_batch_fresh)
    fresh = distinct_keys(n_fresh, width, seed)
    parts, offsets, fresh_counts = [], [0], []
    issued = 0
    while issued < n_fresh:
        nf = min(per_batch_fresh, n_fresh - issued)
        nd = batch - nf if nf == per_batch_fresh else int(round(nf * dup_rate / (1.0 - dup_rate)))
        end = issued + nf
        b = np.empty((nf + nd,) + fresh.shape[1:], dtype=fresh.dtype)
        b[:nf] = fresh[issued:end]
        if nd:
            b[nf:] = fresh[rng.integers(0, end, size=nd)]
        rng.shuffle(b)
        parts.append(b)
        offsets.append(offsets[-1] + len(b))
        fresh_counts.append(nf)
        issued = end
    keys = np.concatenate(parts) if parts else np.empty((0,) + fresh.shape[1:], dtype=fresh.dtype)
    return FillStream(keys, np.asarray(offsets, dtype=np.int64),
                      np.asarray(fresh_counts, dtype=np.int64), n_distinct, width)


def lookup_batch(n_present_pool, n_query, width, seed, present_frac=0.5):
    """A query batch over a table holding keys 0..n_present_pool-1 of the stream.

    Returns (keys, expected_present) where the first round(present_frac*n)
    drawn keys come from the stored range and the rest from a disjoint
    index range, then shuffled together.
    """
    rng = np.random.Generator(np.random.PCG64(seed ^ 0x5EED))
    n_in = int(round(present_frac * n_query))
    n_out = n_query - n_in
    stored = distinct_keys(n_present_pool, width, seed)
    pick = stored[rng.integers(0, n_present_pool, size=n_in)] if n_in else stored[:0]
    absent = distinct_keys(n_out, width, seed, start=n_present_pool + 1)
    keys = np.concatenate([pick, absent])
    present = np.concatenate([np.ones(n_in, dtype=np.uint8), np.zeros(n_out, dtype=np.uint8)])
    order = rng.permutation(n_query)
    return keys[order], present[order]
