"""Every interleaving of the Cuckoo probe kernel's stores, on a small model (no GPU).

In a find-or-put batch each copy of a key is probed by its own thread.  The
probe reads h_1, h_2, ... one slot at a time and stops at the key (found) or
at the first EMPTY slot.  An absent copy that saw an EMPTY slot stores
itself there with a CAS from EMPTY; a CAS that returns the key means another
copy stored it first (found), and one that returns another key moves on to
the next slot, which the CAS reads as well (the bucket scheme's claim in
slot order, Section 4.2, over h_a .. h_k).  A copy whose k slots are all full
claims its key in the dedup set; the one claimant wins and its eviction
chain runs in the insert kernel, after the probe kernel has ended.  With the
paper's rule (Section 4.1: every insertion starts at h_1) a copy CASes only
an EMPTY h_1 and otherwise claims.

Each memory access is one atomic step.  Checked in every reachable state:
no key sits in two slots, and a key stored at h_j (j the smallest index
naming its slot) has h_1 .. h_{j-1} occupied -- the probe's early exit.
Checked in every final state: each key absent before the batch is new for
exactly one of its copies (a CAS that stored it, or the claim), every other
copy is not new, and each key present before is found by all its copies.
The claim winners' chains then run concurrently from h_1 (the chain model
of test_cuckoo_chain_model.py) and every key ends in exactly one place,
found by a probe with the early exit.

Three planted mistakes must each be caught: a copy whose CAS lost to another
key claiming at once instead of trying its next slot; copies with all slots
full inserting without the dedup claim; and a CAS at the last EMPTY slot
seen instead of the first.
"""
import pytest

from test_cuckoo_chain_model import Chains, _sequential_table

E = None   # an empty slot


class ProbeStores:
    """The probe kernel's table and claim-set accesses for a batch of copies.

    A copy's state is (phase, a): "R" reading h_a, "C" CASing h_a, "L" about
    to claim, and the outcomes "F" found, "S" stored by its CAS, "W" won the
    claim, "X" lost the claim."""

    def __init__(self, h, table, batch, rule="first_empty", mistake=None):
        self.h = h
        self.k = len(next(iter(h.values())))
        self.batch = list(batch)
        self.rule = rule
        self.mistake = mistake
        self.before = {x for x in table if x is not E}
        first = ("R", 0) if mistake != "last_empty" else ("R*", 0, -1)
        self.start = (tuple(table), frozenset(), tuple(first for _ in self.batch))

    def step(self, state, i):
        table, claims, copies = state
        x, hs, st = self.batch[i], self.h[self.batch[i]], copies[i]
        ph = st[0]
        if ph in ("F", "S", "W", "X"):
            return None
        table, nxt = list(table), None
        if ph == "R":                       # read h_a; stop at the key or an EMPTY slot
            a = st[1]
            v = table[hs[a]]
            if v == x:
                nxt = ("F",)
            elif v is E:
                may_cas = self.rule == "first_empty" or a == 0
                nxt = ("C", a) if may_cas else ("L",)
            else:
                nxt = ("L",) if a + 1 == self.k else ("R", a + 1)
        elif ph == "R*":                    # planted: read every slot, remember the last EMPTY
            a, last = st[1], st[2]
            v = table[hs[a]]
            if v == x:
                nxt = ("F",)
            else:
                last = a if v is E else last
                if a + 1 < self.k:
                    nxt = ("R*", a + 1, last)
                else:
                    nxt = ("C", last) if last >= 0 else ("L",)
        elif ph == "C":                     # CAS h_a from EMPTY to the key
            a = st[1]
            v = table[hs[a]]
            if v is E:
                table[hs[a]] = x
                nxt = ("S",)
            elif v == x:
                nxt = ("F",)
            elif self.mistake == "claim_on_lost_cas" or self.rule == "h1" or a + 1 == self.k:
                nxt = ("L",)
            else:
                nxt = ("C", a + 1)
        elif ph == "L":                     # one CAS in the dedup set
            if self.mistake == "no_claim":
                nxt = ("W",)
            elif x in claims:
                nxt = ("X",)
            else:
                claims = claims | {x}
                nxt = ("W",)
        c = list(copies)
        c[i] = nxt
        return (tuple(table), claims, tuple(c))

    def check_state(self, state):
        table = state[0]
        stored = [x for x in table if x is not E]
        if len(stored) != len(set(stored)):
            return "a key in two slots: %r" % (table,)
        for s, x in enumerate(table):
            if x is E:
                continue
            hs = self.h[x]
            j = hs.index(s)
            for i in range(j):
                if table[hs[i]] is E:
                    return "key %r at h_%d with h_%d empty: %r" % (x, j + 1, i + 1, table)
        return None

    def check_final(self, state):
        table, _, copies = state
        for x in set(self.batch):
            outs = [copies[i][0] for i in range(len(self.batch)) if self.batch[i] == x]
            new = sum(o in ("S", "W") for o in outs)
            if x in self.before:
                if any(o != "F" for o in outs):
                    return "key %r present before, not found by every copy: %r" % (x, outs)
            elif new != 1:
                return "key %r new for %d copies: %r, table %r" % (x, new, outs, table)
        return None

    def explore(self, limit=2_000_000):
        seen, stack, finals = {self.start}, [self.start], []
        while stack:
            st = stack.pop()
            bad = self.check_state(st)
            if bad:
                return bad, len(seen), finals
            moved = False
            for i in range(len(self.batch)):
                nxt = self.step(st, i)
                if nxt is None:
                    continue
                moved = True
                if nxt not in seen:
                    seen.add(nxt)
                    stack.append(nxt)
                    assert len(seen) < limit
            if not moved:
                bad = self.check_final(st)
                if bad:
                    return bad, len(seen), finals
                finals.append(st)
        return None, len(seen), finals


def _winners(model, final):
    return sorted({model.batch[i] for i, c in enumerate(final[2]) if c[0] == "W"})


def _run_chains_and_check(h, final_table, winners, keys, max_evict=8):
    """The insert kernel after the probe: the claim winners' chains from h_1,
    every interleaving; in each final state every key is in one place and a
    probe with the early exit finds each stored key."""
    c = Chains(h, list(final_table), winners, max_evict=max_evict, start="h1")
    bad, _, finals = c.explore()
    assert bad is None, bad
    for table_f, stash, _ in finals:
        held = [x for x in table_f if x is not E] + list(stash)
        assert sorted(held) == sorted(keys), (held, keys)
        for x in keys:
            if x in stash:
                continue
            found = False
            for s in h[x]:
                if table_f[s] is E:
                    break
                if table_f[s] == x:
                    found = True
                    break
            assert found, (x, table_f)


H = {  # 6 slots, k = 3; 'q' names slot 1 twice (h_1 = h_3)
    "p": [0, 2, 4], "q": [1, 3, 1], "r": [0, 1, 5], "s": [2, 3, 0],
    "t": [0, 4, 2], "u": [1, 0, 3], "v": [4, 5, 0], "w": [3, 0, 5],
}


@pytest.mark.parametrize("rule", ["first_empty", "h1"])
@pytest.mark.parametrize("pre,batch", [
    (["p", "q"], ["r", "r", "s", "t"]),        # collisions on the first EMPTY slot
    (["p", "q"], ["r", "t", "t", "p"]),        # a present key among new ones
    (["p", "q", "s"], ["u", "u", "w", "r"]),   # fuller: some copies see all slots full
    (["p", "q", "r", "s"], ["t", "t", "v"]),   # two slots left: claims and chains
])
def test_probe_stores_are_exact_and_keep_the_early_exit(pre, batch, rule):
    table = _sequential_table(H, pre, 6, max_evict=8, start="first_empty")
    m = ProbeStores(H, table, batch, rule=rule)
    bad, n, finals = m.explore()
    assert bad is None, bad
    assert finals and n > 20
    keys = sorted(set(pre) | set(batch))
    checked = set()
    for f in finals:
        sig = (f[0], tuple(_winners(m, f)))
        if sig in checked:
            continue
        checked.add(sig)
        _run_chains_and_check(H, f[0], list(sig[1]), keys)


@pytest.mark.parametrize("slots,npre,seed", [(8, 4, 1), (8, 5, 2), (9, 5, 3), (7, 4, 5)])
def test_probe_stores_on_random_hashes(slots, npre, seed):
    # k = 3 slots per key drawn at random (repeats allowed), npre keys stored,
    # then a batch of 4 copies of 3 keys (one repeated) at a table load where
    # some copies find every slot full.
    import random
    rng = random.Random(seed)
    names = ["k%d" % i for i in range(npre + 3)]
    h = {x: [rng.randrange(slots) for _ in range(3)] for x in names}
    table = _sequential_table(h, names[:npre], slots, max_evict=10, start="first_empty")
    batch = [names[npre], names[npre], names[npre + 1], names[npre + 2]]
    m = ProbeStores(h, table, batch)
    bad, n, finals = m.explore()
    assert bad is None, bad
    keys = sorted(set(names))
    for sig in {(f[0], tuple(_winners(m, f))) for f in finals}:
        _run_chains_and_check(h, sig[0], list(sig[1]), keys, max_evict=10)


def test_some_copies_claim_and_some_store():
    # The fuller cases reach both paths: in some final state a key is stored
    # by a CAS and another key wins a claim.
    table = _sequential_table(H, ["p", "q", "s"], 6, max_evict=8, start="first_empty")
    m = ProbeStores(H, table, ["u", "u", "w", "r"])
    bad, _, finals = m.explore()
    assert bad is None
    outs = {c[0] for f in finals for c in f[2]}
    assert {"S", "W", "F"} <= outs or {"S", "W", "X"} <= outs


@pytest.mark.parametrize("mistake,pre,batch", [
    # u's h_1 (slot 1) and h_3 (slot 3) are EMPTY: q takes slot 1 between
    # one copy's read and its CAS, that copy claims, and the other copy,
    # probed later, stores u at h_3.
    ("claim_on_lost_cas", ["p"], ["u", "u", "q"]),
    ("no_claim", ["p", "q", "r", "s"], ["t", "t", "v"]),
    ("last_empty", ["p"], ["r", "t", "u"]),
])
def test_checker_catches_planted_mistakes(mistake, pre, batch):
    table = _sequential_table(H, pre, 6, max_evict=8, start="first_empty")
    m = ProbeStores(H, table, batch, mistake=mistake)
    bad, _, _ = m.explore()
    assert bad is not None
