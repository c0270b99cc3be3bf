"""Every interleaving of the long-key bucket protocol, on a small model (no GPU).

The long-key bucket kernel claims a slot's header word (EMPTY -> BUSY|tag by
compare-and-swap), writes the key's words to the slot's row, and publishes
the header (-> tag) with a release store; a thread whose tag matches a header
waits for the publish, then compares the row with its key.  Claims go in slot
order over the slots read as EMPTY, bucket after bucket (Section 4.2's "next
free slot", then the next hash function).

This model runs that protocol with each memory access as one atomic step and
explores every interleaving of a few threads (depth-first, over distinct
states).  In every final state each key new to the table is claimed by
exactly one of its threads and found by the others, no key is stored twice,
and no state is stuck.  The same model with the key as the slot word (one CAS
stores it whole, no publish) is the 64-bit kernels' protocol.  Planted
mistakes in the model -- skipping the tag check of the snapshot, or
publishing before the row is written -- must be caught, so that the checker
is known to see such bugs.
"""
import pytest

EMPTY = ("empty",)


def _busy(tag):
    return ("busy", tag)


def _ready(tag):
    return ("ready", tag)


class Model:
    """keys: one key per thread; tag[key]: its tag (equal tags model digest
    collisions); seq[key]: its buckets h_1, h_2, ... ; S: slots per bucket;
    pre: {slot: key} stored (published) before the threads start; rows: the
    initial row contents (stale words left from earlier use)."""

    def __init__(self, keys, tag, seq, S, nbuckets, pre=None, rows=None,
                 skip_match=False, publish_first=False, one_word=False):
        self.keys, self.tag, self.seq, self.S = list(keys), tag, seq, S
        self.one_word = one_word
        self.nslots = S * nbuckets
        self.skip_match, self.publish_first = skip_match, publish_first
        hdr = [EMPTY] * self.nslots
        row = list(rows) if rows is not None else [None] * self.nslots
        for s, k in (pre or {}).items():
            hdr[s] = _ready(tag[k])
            row[s] = k
        self.pre = dict(pre or {})
        # thread state: (pc, f, snapshot, todo, result)
        threads = tuple(("read", 0, 0, (), (), None) for _ in self.keys)
        self.start = (tuple(hdr), tuple(row), threads)

    # One step of thread i, or None if it cannot move (done, or waiting).
    def step(self, state, i):
        hdr, row, threads = state
        pc, f, pos, snap, todo, res = threads[i]
        key = self.keys[i]
        tag = self.tag[key]
        seq = self.seq[key]
        hdr, row = list(hdr), list(row)

        def put(new):
            t = list(threads)
            t[i] = new
            return (tuple(hdr), tuple(row), tuple(t))

        if pc == "done":
            return None
        base = seq[f] * self.S if f < len(seq) else 0
        if pc == "read":                      # read header pos of bucket h_f
            snap2 = snap + (hdr[base + pos],)
            if pos + 1 < self.S:
                return put(("read", f, pos + 1, snap2, (), None))
            match = tuple(s for s, h in enumerate(snap2)
                          if h != EMPTY and h[1] == tag and not self.skip_match)
            empty = tuple(s for s, h in enumerate(snap2) if h == EMPTY)
            return put(("match", f, 0, snap2, (match, empty), None))
        if pc == "match":                     # check tag matches in slot order
            match, empty = todo
            if pos < len(match):
                return put(("wait", f, match[pos], snap, todo, ("match", pos + 1)))
            return put(("claim", f, 0, snap, todo, None))
        if pc == "wait":                      # wait for the publish, then compare the row
            s = base + pos
            if hdr[s][0] == "busy":
                return None
            if row[s] == key:
                return put(("done", f, 0, (), (), "found"))
            nxt, p = res
            return put((nxt, f, p, snap, todo, None))
        if pc == "claim":                     # claim the slots read as EMPTY, in slot order
            match, empty = todo
            if pos >= len(empty):             # bucket full: the next function, if any
                if f + 1 < len(seq):
                    return put(("read", f + 1, 0, (), (), None))
                return put(("done", f, 0, (), (), "full"))
            s = base + empty[pos]
            old = hdr[s]
            if old == EMPTY:
                if self.one_word:             # the word is the key: stored whole by the CAS
                    hdr[s] = _ready(tag)
                    row[s] = key
                    return put(("done", f, 0, (), (), "claimed"))
                if self.publish_first:
                    hdr[s] = _ready(tag)
                    return put(("write", f, empty[pos], snap, todo, None))
                hdr[s] = _busy(tag)
                return put(("write", f, empty[pos], snap, todo, None))
            if old[1] == tag:
                return put(("wait", f, empty[pos], snap, todo, ("claim", pos + 1)))
            return put(("claim", f, pos + 1, snap, todo, None))
        if pc == "write":                     # the key's words into the slot's row
            row[base + pos] = key
            if self.publish_first:
                return put(("done", f, 0, (), (), "claimed"))
            return put(("publish", f, pos, snap, todo, None))
        if pc == "publish":                   # release store of the tag
            hdr[base + pos] = _ready(tag)
            return put(("done", f, 0, (), (), "claimed"))
        raise AssertionError(pc)

    def explore(self, limit=2_000_000):
        """All reachable final states; raises on a stuck state."""
        seen, finals, stack = {self.start}, [], [self.start]
        while stack:
            st = stack.pop()
            moved = False
            for i in range(len(self.keys)):
                nxt = self.step(st, i)
                if nxt is None:
                    continue
                moved = True
                if nxt not in seen:
                    seen.add(nxt)
                    stack.append(nxt)
                    assert len(seen) < limit, "state space too large for the test"
            if not moved:
                if any(t[0] != "done" for t in st[2]):
                    raise AssertionError("stuck state: %r" % (st,))
                finals.append(st)
        return finals, len(seen)

    def violations(self, final):
        """What is wrong with a final state (empty list: nothing)."""
        hdr, row, threads = final
        out = []
        stored = [row[s] for s in range(self.nslots) if hdr[s][0] == "ready"]
        if len(stored) != len(set(stored)):
            out.append("a key is stored twice: %r" % stored)
        if any(h[0] == "busy" for h in hdr):
            out.append("a claimed header was never published")
        for k in set(self.keys):
            res = [threads[i][5] for i in range(len(self.keys)) if self.keys[i] == k]
            if k in self.pre.values():
                if any(r != "found" for r in res):
                    out.append("stored key %r not found by every copy: %r" % (k, res))
            elif "full" not in res:
                if res.count("claimed") != 1 or res.count("found") != len(res) - 1:
                    out.append("key %r: %r (want one claim, the rest found)" % (k, res))
                if k not in stored:
                    out.append("key %r is not stored" % k)
        return out


def _check(model):
    finals, n = model.explore()
    bad = [(f, v) for f in finals for v in [model.violations(f)] if v]
    return finals, n, bad


# Tags: 'a' and 'b' collide (same tag, different keys); 'c' differs.
TAG = {"a": 1, "b": 1, "c": 2}


@pytest.mark.parametrize("keys", [("a", "a", "a"), ("a", "a", "b"), ("a", "b", "a"), ("a", "c", "a")])
def test_one_bucket_every_interleaving(keys):
    m = Model(keys, TAG, {"a": [0], "b": [0], "c": [0]}, S=3, nbuckets=1)
    finals, n, bad = _check(m)
    assert not bad, bad[0]
    assert n > 100 and finals


def test_full_buckets_move_on_in_order():
    # One slot per bucket: copies of 'a' and a colliding 'b' race for bucket
    # 0, the loser of each key moves on to its next bucket.
    seq = {"a": [0, 1, 2], "b": [0, 2, 1]}
    m = Model(("a", "b", "a", "b"), TAG, seq, S=1, nbuckets=3)
    finals, n, bad = _check(m)
    assert not bad, bad[0]


@pytest.mark.parametrize("keys,seq,rows", [
    (("a", "a", "b", "b"), {"a": [0, 1], "b": [1, 0]}, None),
    (("a", "b", "a", "c"), {"a": [0, 1], "b": [0, 1], "c": [1, 0]}, ["a", "a", "b", "b"]),
])
def test_two_buckets_of_two(keys, seq, rows):
    m = Model(keys, TAG, seq, S=2, nbuckets=2, rows=rows)
    finals, n, bad = _check(m)
    assert not bad, bad[0]


def test_key_behind_a_full_bucket_is_found():
    # Bucket 0 is full of other keys (one with a colliding tag); 'a' sits in
    # bucket 1.  Its copies compare, move on and find it; a new colliding
    # 'd' lands in bucket 1's free slot.
    tag = dict(TAG, d=1, e=3)
    m = Model(("a", "a", "d"), tag, {"a": [0, 1], "d": [0, 1], "b": [0], "e": [0]}, S=2, nbuckets=2,
              pre={0: "b", 1: "e", 2: "a"})
    finals, n, bad = _check(m)
    assert not bad, bad[0]
    for f in finals:
        assert [t[5] for t in f[2]] == ["found", "found", "claimed"]


def test_stored_keys_and_stale_rows():
    # 'c' is already stored in slot 0; every row holds a stale 'a' left from
    # before a clear, so a reader that compared a row before its publish
    # would "find" 'a' where 'b' is being written.
    m = Model(("a", "b", "c", "a"), TAG, {"a": [0], "b": [0], "c": [0]}, S=3, nbuckets=1,
              pre={0: "c"}, rows=["c", "a", "a"])
    finals, n, bad = _check(m)
    assert not bad, bad[0]


@pytest.mark.parametrize("keys,pre", [
    (("a", "a", "b", "b"), None),
    (("a", "b", "c", "a"), {1: "c"}),
])
def test_one_word_claims(keys, pre):
    # The 64-bit kernels' protocol: the slot word is the key, so a claim
    # stores it whole and there is no publish step (each key its own tag).
    tag = {"a": 1, "b": 2, "c": 3}
    seq = {"a": [0, 1], "b": [1, 0], "c": [0, 1]}
    m = Model(keys, tag, seq, S=2, nbuckets=2, pre=pre, one_word=True)
    finals, n, bad = _check(m)
    assert not bad, bad[0]
    assert n > 100


def test_claim_set_with_colliding_digests():
    # The long-key Cuckoo claim set: linear probing (one-slot buckets in
    # probe order, wrapping) over entries that one 16-byte CAS writes whole;
    # 'a' and 'b' share a digest and are told apart by comparing batch keys.
    seq = {"a": [0, 1, 2], "b": [1, 2, 0]}
    m = Model(("a", "b", "a", "b"), TAG, seq, S=1, nbuckets=3, one_word=True)
    finals, n, bad = _check(m)
    assert not bad, bad[0]
    assert n > 100


def test_checker_catches_a_skipped_tag_check():
    # Planted: the snapshot's tag matches are ignored, so a copy that sees
    # its key already published claims another slot -- a key stored twice.
    m = Model(("a", "a"), TAG, {"a": [0]}, S=2, nbuckets=1, pre=None, skip_match=True)
    finals, n, bad = _check(m)
    assert bad and any("twice" in v for _, vs in bad for v in vs)


def test_checker_catches_publish_before_write():
    # Planted: the header is published before the row is written; with a
    # stale 'a' in the row, a colliding 'a' reads the half-made slot of 'b'
    # as its own key and is lost.
    m = Model(("b", "a"), TAG, {"a": [0], "b": [0]}, S=2, nbuckets=1, rows=["a", "a"], publish_first=True)
    finals, n, bad = _check(m)
    assert bad
