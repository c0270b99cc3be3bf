"""Every interleaving of concurrent Cuckoo eviction chains, on a small model (no GPU).

The insert kernel runs one chain per winner (a key new to the table,
distinct from every other winner): the key is exchanged into its first
slot; an evicted key k' that sat at slot s moves to h_{a+1}(k'), a the
smallest index with h_a(k') = s (after h_k: h_1); after max_evictions
exchanges the held key goes to the stash.  Section 4.1 gives the chain and
starts it at h_1; the smallest-index rule and the wrap are this project's
reading of it.  The kernel's default starts a chain instead at the first
slot h_j that the probe, run on the same table before any insert, saw EMPTY
(h_1 when it saw none): modelled here by choosing each winner's start from
the table as it is before the chains run.

Two facts of the design are checked in every reachable state, with each
exchange one atomic step:
* conservation: every key is in exactly one place -- a slot, the stash, or
  the hand of one chain;
* the probe's early exit: a key stored at h_j (j the smallest index naming
  its slot) has h_1 .. h_{j-1} all occupied, so a probe that finds h_1 EMPTY
  may stop.  Slots never return to EMPTY, which is what makes it hold.
Both start rules are checked.  Two planted mistakes must break the second
fact, so the checker is known to see them: an off-by-one (an evicted key
moves on to h_{a+2} instead of h_{a+1}), and a start at the LAST empty slot
the probe saw instead of the first.
"""
import pytest

E = None   # an empty slot


def start_index(table, hs, rule):
    """The hash index a winner's chain starts at, from the probe's view of the
    table: "h1" (Section 4.1), "first_empty" (the kernel's default: the probe
    stops at an empty h_1, else reads h_2..h_k, and the chain starts at the
    first of them it saw EMPTY, else at h_1) or "last_empty" (a planted
    mistake)."""
    if rule == "h1":
        return 0
    empties = [j for j in range(len(hs)) if table[hs[j]] is E]
    if not empties:
        return 0
    return empties[0] if rule == "first_empty" else empties[-1]


class Chains:
    def __init__(self, h, table, winners, max_evict, skip_one=False, start="h1"):
        self.h = h                          # key -> its slots h_1 .. h_k
        self.k = len(next(iter(h.values())))
        self.max_evict = max_evict
        self.skip_one = skip_one
        self.keys = sorted([x for x in table if x is not E] + list(winners))
        # (held key, target slot, evictions); every start is taken from the
        # table before any chain runs, as the probe kernel sees it.
        threads = tuple((w, h[w][start_index(table, h[w], start)], 0) for w in winners)
        self.start = (tuple(table), (), threads)

    def step(self, state, i):
        table, stash, threads = state
        th = threads[i]
        if th is None:
            return None
        held, slot, ev = th
        table = list(table)
        old = table[slot]
        table[slot] = held                  # one atomic exchange
        t = list(threads)
        if old is E:
            t[i] = None
        elif ev + 1 > self.max_evict:
            t[i] = None
            stash = tuple(sorted(stash + (old,)))
        else:
            hs = self.h[old]
            a = min(j for j in range(self.k) if hs[j] == slot)
            nxt = hs[(a + 2) % self.k] if self.skip_one else hs[(a + 1) % self.k]
            t[i] = (old, nxt, ev + 1)
        return (tuple(table), stash, tuple(t))

    def check_state(self, state):
        table, stash, threads = state
        held = [t[0] for t in threads if t is not None]
        placed = [x for x in table if x is not E] + list(stash) + held
        if sorted(placed) != self.keys:
            return "keys not conserved: %r" % (state,)
        for s, x in enumerate(table):
            if x is E:
                continue
            hs = self.h[x]
            if s not in hs:
                return "key %r at slot %d, not one of its slots" % (x, s)
            j = hs.index(s)
            for i in range(j):
                if table[hs[i]] is E:
                    return "key %r at h_%d with h_%d empty: %r" % (x, j + 1, i + 1, table)
        return None

    def explore(self, limit=1_000_000):
        seen, stack, finals = {self.start}, [self.start], []
        while stack:
            st = stack.pop()
            bad = self.check_state(st)
            if bad:
                return bad, len(seen), finals
            moved = False
            for i in range(len(st[2])):
                nxt = self.step(st, i)
                if nxt is None:
                    continue
                moved = True
                if nxt not in seen:
                    seen.add(nxt)
                    stack.append(nxt)
                    assert len(seen) < limit
            if not moved:
                finals.append(st)
        return None, len(seen), finals


def _sequential_table(h, keys, m, max_evict, start="h1"):
    """A table built by inserting keys one at a time with the same chains."""
    table, stash = [E] * m, []
    for key in keys:
        c = Chains(h, table, [key], max_evict, start=start)
        st = c.start
        while st[2][0] is not None:
            st = c.step(st, 0)
        table, stash = list(st[0]), stash + list(st[1])
    assert not stash
    return table


H = {  # 6 slots, k = 3; 'q' names slot 1 twice (h_1 = h_3)
    "p": [0, 2, 4], "q": [1, 3, 1], "r": [0, 1, 5], "s": [2, 3, 0],
    "t": [0, 4, 2], "u": [1, 0, 3], "v": [4, 5, 0], "w": [3, 0, 5],
}


@pytest.mark.parametrize("start", ["h1", "first_empty"])
@pytest.mark.parametrize("pre,winners", [
    (["p", "q"], ["r", "s", "t"]),
    (["p", "q", "r"], ["s", "t", "u"]),
    (["p", "s", "u"], ["q", "v", "w"]),
])
def test_concurrent_chains_conserve_keys_and_keep_the_early_exit(pre, winners, start):
    table = _sequential_table(H, pre, 6, max_evict=8, start=start)
    c = Chains(H, table, winners, max_evict=8, start=start)
    bad, n, finals = c.explore()
    assert bad is None, bad
    assert finals and n > 5
    for table_f, stash, _ in finals:
        # every key once; a probe with the early exit finds each stored key
        for x in c.keys:
            if x in stash:
                continue
            hs = H[x]
            found = False
            for s in hs:
                if table_f[s] is E:
                    break
                if table_f[s] == x:
                    found = True
                    break
            assert found, (x, table_f)


@pytest.mark.parametrize("slots,npre,seed,start", [
    (9, 5, 1, "h1"), (9, 5, 3, "h1"), (10, 6, 1, "h1"),
    # Seeds where several winners saw the same first empty slot: their chains
    # collide there, one takes it and the others evict it.
    (9, 5, 11, "first_empty"), (9, 5, 16, "first_empty"), (8, 4, 18, "first_empty"), (9, 5, 3, "first_empty"),
])
def test_four_concurrent_chains_on_random_hashes(slots, npre, seed, start):
    # k = 3 slots per key drawn at random (repeats allowed), npre keys stored
    # one at a time, then 4 chains at once into a table of load near 1: long
    # chains, some ending in the stash; thousands of states.
    import random
    rng = random.Random(seed)
    names = ["k%d" % i for i in range(npre + 4)]
    h = {x: [rng.randrange(slots) for _ in range(3)] for x in names}
    table = _sequential_table(h, names[:npre], slots, max_evict=10, start=start)
    c = Chains(h, table, names[npre:], max_evict=10, start=start)
    bad, n, finals = c.explore()
    assert bad is None, bad
    assert n > 1000 and any(f[1] for f in finals)


def test_overfull_table_spills_to_the_stash():
    # 7 keys, 6 slots, short chains: some final states stash keys, and the
    # facts above hold in every state on the way.
    table = _sequential_table(H, ["p", "q", "r", "s"], 6, max_evict=3)
    c = Chains(H, table, ["t", "u", "v"], max_evict=3)
    bad, n, finals = c.explore()
    assert bad is None, bad
    assert any(f[1] for f in finals)


def test_checker_catches_a_skipped_slot():
    # Planted: an evicted key skips h_{a+1} and moves on to h_{a+2}; it can
    # then sit past an EMPTY slot of its own, where a probe that stops at the
    # first EMPTY slot would miss it.
    table = _sequential_table(H, ["p", "q"], 6, max_evict=8)
    c = Chains(H, table, ["r", "s", "t"], max_evict=8, skip_one=True)
    bad, n, finals = c.explore()
    assert bad is not None


def test_first_empty_start_saves_exchanges():
    # The reason for the default: at the same table and winners, starting at
    # the first empty slot the probe saw never takes more exchanges in a
    # sequential run than starting at h_1, and here takes fewer.
    def exchanges(start):
        table, total = _sequential_table(H, ["p", "q", "s"], 6, max_evict=8, start=start), 0
        for w in ["r", "t", "v"]:
            c = Chains(H, table, [w], max_evict=8, start=start)
            st = c.start
            while st[2][0] is not None:
                st = c.step(st, 0)
                total += 1
            table = list(st[0])
        return total
    assert exchanges("first_empty") < exchanges("h1")


def test_checker_catches_a_start_past_an_empty_slot():
    # Planted: the chain starts at the LAST empty slot the probe saw.  The key
    # then sits past an EMPTY slot of its own, which the early exit misses.
    table = _sequential_table(H, ["p", "q"], 6, max_evict=8)
    c = Chains(H, table, ["r", "s", "t"], max_evict=8, start="last_empty")
    bad, n, finals = c.explore()
    assert bad is not None and "empty" in bad
