"""Every interleaving of the 128-bit Cuckoo probe's stores under torn reads (no GPU).

A 128-bit slot is written by one 16-byte compare-and-swap, but the probe
reads slots with plain 16-byte loads, which the memory model does not make
atomic with respect to that CAS: a read may see one word of a key being
stored and the other word still all ones (EMPTY is all ones in both words).
The probe therefore counts a read as a complete key only when neither word
is all ones; any other read is a candidate that the CAS settles, and the CAS
always returns the slot's true content.  A key whose low word is all ones is
legal and always reads as a candidate.

The model gives each slot a true content (what a CAS sees) and a visible
content (what a plain read sees).  A successful CAS sets the true content at
once; the storing thread then makes the key visible in two further steps,
one word first (either word) and then both.  Each copy of a key reads
h_1, h_2, ... until it finds the key complete or meets a candidate, CASes
from EMPTY in slot order from there (a CAS that returns the key: found; one
that returns another key: next slot), and claims in the dedup set when every
slot held another key.  Checked in every reachable state: no key is stored
twice (true contents) and a key stored at h_j has h_1 .. h_{j-1} occupied;
in every final state each absent key is new for exactly one copy and each
present key is found by all its copies.

The planted mistake -- a torn read taken as another key's slot, so the copy
reads on past it -- must be caught: a copy then stores its key a second time
behind a slot where another copy's store of it is still half visible.
"""
import pytest

ONES = "1"                     # an all-ones word
E = (ONES, ONES)               # an empty slot


def _class(v):
    """2: a complete key (neither word all ones); 1: a candidate."""
    return 2 if v[0] != ONES and v[1] != ONES else 1


class WideStores:
    """Copies of 128-bit keys probing and storing concurrently.

    State: (true slots, visible slots, claims, copies).  A copy is
    (phase, a, ...): "R" reading h_a, "C" CASing h_a, "V1"/"V2" making its
    stored key visible (one word, then both), "L" claiming, and the outcomes
    "F" found, "S" stored, "W" won the claim, "X" lost it."""

    def __init__(self, h, table, batch, mistake=None):
        self.h = h
        self.k = len(next(iter(h.values())))
        self.batch = list(batch)
        self.mistake = mistake
        self.before = {x for x in table if x != E}
        self.start = (tuple(table), tuple(table), frozenset(), tuple(("R", 0) for _ in self.batch))

    def moves(self, state, i):
        """The states copy i can move the system to (several where the
        visible word order is a choice)."""
        true, vis, claims, copies = state
        x, hs, st = self.batch[i], self.h[self.batch[i]], copies[i]
        ph = st[0]
        out = []
        if ph in ("F", "S", "W", "X"):
            return out

        def put(new_st, t=true, v=vis, c=claims):
            cp = list(copies)
            cp[i] = new_st
            out.append((t, v, c, tuple(cp)))

        if ph == "R":
            a = st[1]
            v = vis[hs[a]]
            if _class(v) == 2 and v == x:
                put(("F",))
            elif _class(v) == 1 and not (self.mistake == "torn_as_occupied" and v != E):
                put(("C", a))
            else:
                put(("L",) if a + 1 == self.k else ("R", a + 1))
        elif ph == "C":
            a = st[1]
            s = hs[a]
            if true[s] == E:
                t = list(true)
                t[s] = x
                put(("V1", s), t=tuple(t))
            elif true[s] == x:
                put(("F",))
            else:
                put(("L",) if a + 1 == self.k else ("C", a + 1))
        elif ph == "V1":                        # one word of the key becomes visible
            s = st[1]
            for half in ((x[0], ONES), (ONES, x[1])):
                v = list(vis)
                v[s] = half
                put(("V2", s), v=tuple(v))
        elif ph == "V2":                        # both words visible
            s = st[1]
            v = list(vis)
            v[s] = x
            put(("S",), v=tuple(v))
        elif ph == "L":
            if x in claims:
                put(("X",))
            else:
                put(("W",), c=claims | {x})
        return out

    def check_state(self, state):
        true = state[0]
        stored = [x for x in true if x != E]
        if len(stored) != len(set(stored)):
            return "a key in two slots: %r" % (true,)
        for s, x in enumerate(true):
            if x == E:
                continue
            hs = self.h[x]
            j = hs.index(s)
            for i in range(j):
                if true[hs[i]] == E:
                    return "key %r at h_%d with h_%d empty: %r" % (x, j + 1, i + 1, true)
        return None

    def check_final(self, state):
        copies = state[3]
        for x in set(self.batch):
            outs = [copies[i][0] for i in range(len(self.batch)) if self.batch[i] == x]
            new = sum(o in ("S", "W") for o in outs)
            if x in self.before:
                if any(o != "F" for o in outs):
                    return "key %r present before, not found by every copy: %r" % (x, outs)
            elif new != 1:
                return "key %r new for %d copies: %r" % (x, new, outs)
        return None

    def explore(self, limit=2_000_000):
        seen, stack, n_final = {self.start}, [self.start], 0
        while stack:
            st = stack.pop()
            bad = self.check_state(st)
            if bad:
                return bad, len(seen), n_final
            moved = False
            for i in range(len(self.batch)):
                for nxt in self.moves(st, i):
                    moved = True
                    if nxt not in seen:
                        seen.add(nxt)
                        stack.append(nxt)
                        assert len(seen) < limit
            if not moved:
                bad = self.check_final(st)
                if bad:
                    return bad, len(seen), n_final
                n_final += 1
        return None, len(seen), n_final


# Keys as (low word, high word); "L" is a legal key whose low word is all ones.
P, Q, R, S, T = ("p", "P"), ("q", "Q"), ("r", "R"), ("s", "S"), ("t", "T")
L = (ONES, "L")
H = {  # 5 slots, k = 3
    P: [0, 2, 4], Q: [1, 3, 1], R: [0, 1, 4], S: [2, 3, 0], T: [0, 4, 2], L: [0, 1, 3],
}


def _table(stored):
    """A table holding `stored` keys, each at the first slot of its own that
    is empty (as the probe stores them one at a time)."""
    t = [E] * 5
    for x in stored:
        for s in H[x]:
            if t[s] == E:
                t[s] = x
                break
        else:
            raise AssertionError("no room for %r" % (x,))
    return t


@pytest.mark.parametrize("pre,batch", [
    ([], [R, R, T]),                    # two copies race on h_1 while a third key shares it
    ([P], [R, R, L]),                   # a key with an all-ones low word among them
    ([P, Q], [L, L, R]),                # copies of the all-ones-low key, and a fuller table
    ([L], [L, R, R]),                   # the all-ones-low key present before: found by its copy
    ([P, Q, S], [T, T]),                # every slot of T full: the claim set decides
])
def test_wide_stores_are_exact_under_torn_reads(pre, batch):
    m = WideStores(H, _table(pre), batch)
    bad, n, n_final = m.explore()
    assert bad is None, bad
    assert n_final > 0 and n > 20


def test_checker_catches_a_torn_read_taken_as_another_key():
    # Copy 1 stores R at h_1 and has made only one word visible; copy 2 reads
    # that half-written slot, takes it as another key's and stores R again at
    # its next empty slot.
    m = WideStores(H, _table([]), [R, R], mistake="torn_as_occupied")
    bad, _, _ = m.explore()
    assert bad is not None and ("two slots" in bad or "new for 2" in bad)
