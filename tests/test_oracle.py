"""Pins of the CPU oracle against things other than itself.

* find-or-put / insert / lookup: brute force on tiny inputs with a plain
  Python list scanned linearly (no hashing at all).
* BFS: the global transition relation of a model written as a sum of
  Kronecker products of per-component adjacency matrices (interleaving =
  Kronecker sum; a synchronising pair = the Kronecker product of the two
  labelled parts), explored with scipy's graph routines.  Packing the state
  vector LSB-first makes the Kronecker index equal the packed vector.
* BFS without synchronisation: closed forms -- the reachable count is the
  product of the per-component windows and the level sizes are the
  convolution of the per-component distance histograms (each interleaving
  step moves exactly one component one local step).
* Hand-built models whose answers are worked out by hand.
"""
import numpy as np
import pytest
import scipy.sparse as sp
from scipy.sparse.csgraph import shortest_path

from workloads import statespace as ss


# ----------------------------------------------------------------- sets/maps
def _brute_find_or_put(stored, keys):
    out = []
    for k in keys:
        hit = False
        for s in stored:          # linear scan, no hashing
            if s == k:
                hit = True
                break
        if hit:
            out.append(0)
        else:
            stored.append(k)
            out.append(1)
    return np.array(out, dtype=np.uint8)


@pytest.mark.parametrize("seed", [0, 1, 2, 3])
@pytest.mark.parametrize("vrange", [4, 64, 100000])
def test_find_or_put_matches_brute_force(oracle_lib, seed, vrange):
    rng = np.random.default_rng(seed)
    t = oracle_lib.OracleTable()
    stored = []
    for _ in range(4):
        n = int(rng.integers(0, 400))
        keys = rng.integers(0, vrange, size=n).astype(np.uint64)
        got = t.find_or_put(keys)
        exp = _brute_find_or_put(stored, keys.tolist())
        np.testing.assert_array_equal(got, exp)
        assert t.size() == len(stored)
    k, _ = t.export()
    np.testing.assert_array_equal(k, np.sort(np.array(stored, dtype=np.uint64)))


def test_find_or_put_first_occurrence_only(oracle_lib):
    # In batch order exactly the first occurrence of each new key is flagged.
    t = oracle_lib.OracleTable()
    got = t.find_or_put(np.array([5, 5, 7, 5, 7, 9], dtype=np.uint64))
    np.testing.assert_array_equal(got, [1, 0, 1, 0, 0, 1])
    got = t.find_or_put(np.array([9, 10, 5, 10], dtype=np.uint64))
    np.testing.assert_array_equal(got, [0, 1, 0, 0])
    assert t.size() == 4


def test_find_or_put_empty_and_large_keys(oracle_lib):
    t = oracle_lib.OracleTable()
    assert len(t.find_or_put(np.array([], dtype=np.uint64))) == 0
    big = np.array([(1 << 63) - 1, 0, (1 << 63) - 1, 0xFFFFFFFE], dtype=np.uint64)
    np.testing.assert_array_equal(t.find_or_put(big), [1, 1, 0, 1])


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_insert_lookup_match_brute_force(oracle_lib, seed):
    rng = np.random.default_rng(100 + seed)
    t = oracle_lib.OracleTable()
    pairs = []                    # (key, value) in insertion order, first wins
    for _ in range(3):
        n = int(rng.integers(1, 300))
        keys = rng.integers(0, 200, size=n).astype(np.uint64)
        vals = rng.integers(0, 2**32 - 1, size=n).astype(np.uint32)
        t.insert(keys, vals)
        for k, v in zip(keys.tolist(), vals.tolist()):
            if not any(pk == k for pk, _ in pairs):
                pairs.append((k, v))
        q = rng.integers(0, 260, size=257).astype(np.uint64)
        found, got = t.lookup(q)
        for i, k in enumerate(q.tolist()):
            match = [pv for pk, pv in pairs if pk == k]
            assert found[i] == (1 if match else 0)
            assert got[i] == (match[0] if match else 0)
    assert t.size() == len(pairs)


# ----------------------------------------------------------------- BFS
def _manual_model(L, trans, pairs=()):
    """trans[c] = list of (u, v, label)."""
    C = len(L)
    bits = np.zeros(ss.CMAX, dtype=np.uint8)
    deg = np.zeros((ss.CMAX, ss.LMAX), dtype=np.uint8)
    tgt = np.zeros((ss.CMAX, ss.LMAX, ss.DMAX), dtype=np.uint8)
    lab = np.zeros((ss.CMAX, ss.LMAX, ss.DMAX), dtype=np.uint8)
    for c in range(C):
        bits[c] = max(1, int(np.ceil(np.log2(L[c]))))
        for (u, v, l) in trans[c]:
            j = deg[c, u]
            tgt[c, u, j] = v
            lab[c, u, j] = l
            deg[c, u] += 1
    return ss.Model(C=C, L=np.array(L), bits=bits, deg=deg, tgt=tgt, lab=lab,
                    pairs=np.array(pairs, dtype=np.uint8).reshape(-1, 2))


def _kron_adjacency(m):
    """Global adjacency (with multiplicities) as a sum of Kronecker products."""
    dims = [1 << int(m.bits[c]) for c in range(m.C)]

    def local(c, label):
        a = sp.lil_matrix((dims[c], dims[c]), dtype=np.int64)
        for u in range(int(m.L[c])):
            for j in range(int(m.deg[c, u])):
                if int(m.lab[c, u, j]) == label:
                    a[u, int(m.tgt[c, u, j])] += 1
        return a.tocsr()

    def chain(factors):
        # factors[c] for component c; the most significant component goes first.
        out = None
        for c in reversed(range(m.C)):
            f = factors.get(c, sp.identity(dims[c], dtype=np.int64, format="csr"))
            out = f if out is None else sp.kron(out, f, format="csr")
        return out

    total = None
    for c in range(m.C):
        term = chain({c: local(c, 0)})
        total = term if total is None else total + term
    for p in range(m.P):
        c1, c2 = int(m.pairs[p, 0]), int(m.pairs[p, 1])
        total = total + chain({c1: local(c1, p + 1), c2: local(c2, p + 1)})
    return total.tocsr()


def _kron_levels(m):
    a = _kron_adjacency(m)
    d = shortest_path(a, method="D", unweighted=True, indices=0, directed=True)
    reach = np.isfinite(d)
    levels = d[reach].astype(np.int64)
    states = np.nonzero(reach)[0].astype(np.uint64)
    return a, states, levels


@pytest.mark.parametrize("seed,C,L,R,P,ps", [
    (1, 3, 8, 5, 0, 0.0),
    (2, 4, [4, 8, 5, 6], [3, 6, 5, 2], 2, 0.5),
    (3, 5, 4, 4, 3, 0.3),
    (4, 2, 32, 20, 1, 0.6),
    (5, 6, [2, 4, 4, 3, 4, 2], [2, 4, 3, 3, 4, 2], 4, 0.4),
])
def test_bfs_matches_kronecker_reachability(oracle_lib, seed, C, L, R, P, ps):
    m = ss.random_model(seed, C=C, L=L, R=R, p_sync=ps, P=P)
    assert m.total_bits <= 16
    a, states, levels = _kron_levels(m)
    res = oracle_lib.bfs(m, max_states=1 << 17)
    assert res.rc == 0
    assert res.total == len(states)
    np.testing.assert_array_equal(res.level_sizes, np.bincount(levels))
    for d in range(len(res.level_sizes)):
        np.testing.assert_array_equal(np.sort(res.level(d)), np.sort(states[levels == d]))
    # successor multiset sizes per level = row sums of the adjacency
    rows = np.asarray(a.sum(axis=1)).ravel()
    for d in range(len(res.level_sizes)):
        assert res.level_succ[d] == rows[states[levels == d].astype(np.int64)].sum()


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_successors_match_kronecker_rows(oracle_lib, seed):
    m = ss.random_model(seed, C=3, L=[8, 4, 8], R=[8, 4, 6], p_sync=0.5, P=2)
    a = _kron_adjacency(m)
    for s in [0, 1, 5, 37, 100, 255]:
        got = np.sort(oracle_lib.successors(m, s))
        row = a.getrow(s)
        exp = np.sort(np.repeat(row.indices, row.data.astype(np.int64)).astype(np.uint64))
        np.testing.assert_array_equal(got, exp)


@pytest.mark.parametrize("seed", [11, 12, 13])
def test_bfs_closed_form_without_sync(oracle_lib, seed):
    from scipy.sparse.csgraph import breadth_first_order
    R = [3, 5, 4, 6, 2]
    m = ss.random_model(seed, C=5, L=[8, 8, 4, 16, 2], R=R, p_sync=0.0, P=0)
    res = oracle_lib.bfs(m, max_states=1 << 20)
    assert res.total == int(np.prod(R))
    poly = np.array([1], dtype=np.int64)
    for c in range(m.C):
        a = sp.lil_matrix((int(m.L[c]), int(m.L[c])))
        for u in range(int(m.L[c])):
            for j in range(int(m.deg[c, u])):
                a[u, int(m.tgt[c, u, j])] = 1
        order, _ = breadth_first_order(a.tocsr(), 0, directed=True)
        assert len(order) == R[c]
        d = shortest_path(a.tocsr(), unweighted=True, indices=0)
        hist = np.bincount(d[np.isfinite(d)].astype(np.int64))
        poly = np.convolve(poly, hist)
    np.testing.assert_array_equal(res.level_sizes, poly)


def test_bfs_hand_models(oracle_lib):
    # One component, an 8-cycle: 8 levels of one state each, in order.
    m = _manual_model([8], [[(u, (u + 1) % 8, 0) for u in range(8)]])
    r = oracle_lib.bfs(m)
    np.testing.assert_array_equal(r.level_sizes, [1] * 8)
    np.testing.assert_array_equal(r.states, np.arange(8, dtype=np.uint64))
    # Two 2-cycles whose every move is synchronised: only 00 and 11 (= 3).
    m = _manual_model([2, 2], [[(0, 1, 1), (1, 0, 1)], [(0, 1, 1), (1, 0, 1)]], pairs=[(0, 1)])
    r = oracle_lib.bfs(m)
    np.testing.assert_array_equal(r.level_sizes, [1, 1])
    np.testing.assert_array_equal(np.sort(r.states), [0, 3])
    # A synchronising pair fires every combination: 2 x 2 joint moves.
    m = _manual_model([4, 4], [[(0, 1, 1), (0, 2, 1)], [(0, 1, 1), (0, 3, 1)]], pairs=[(0, 1)])
    got = np.sort(oracle_lib.successors(m, 0))
    np.testing.assert_array_equal(got, np.sort(np.array([1 | 4, 1 | 12, 2 | 4, 2 | 12], dtype=np.uint64)))
    # A labelled transition without a matching partner never fires alone.
    m = _manual_model([4, 4], [[(0, 1, 1), (0, 2, 0)], [(0, 3, 0)]], pairs=[(0, 1)])
    got = np.sort(oracle_lib.successors(m, 0))
    np.testing.assert_array_equal(got, np.sort(np.array([2, 3 << 2], dtype=np.uint64)))
    # Bit packing: component 1 of a (3-bit, 2-bit) layout sits at bit 3.
    m = _manual_model([5, 3], [[], [(0, 2, 0)]])
    np.testing.assert_array_equal(oracle_lib.successors(m, 0), [2 << 3])


def test_bfs_limits(oracle_lib):
    m = _manual_model([8], [[(u, (u + 1) % 8, 0) for u in range(8)]])
    assert oracle_lib.bfs(m, max_levels=3).rc == 2
    m = ss.random_model(7, C=4, L=8, R=8)
    assert oracle_lib.bfs(m, max_states=100).rc == 1


def test_oracle128_find_or_put_lookup_export_against_brute_force(oracle_lib):
    # Keys that share their low word, keys that share their high word, and
    # repeats: a key is the pair, neither word alone.
    rng = np.random.default_rng(12)
    lo = rng.integers(0, 6, size=3000).astype(np.uint64)
    hi = rng.integers(0, 6, size=3000).astype(np.uint64) << np.uint64(40)
    keys = np.stack([lo, hi], axis=1)
    t = oracle_lib.OracleTable128()
    seen, exp = set(), []
    for a, b in keys.tolist():
        exp.append(int((a, b) not in seen))
        seen.add((a, b))
    got = np.concatenate([t.find_or_put(keys[i:i + 700]) for i in range(0, len(keys), 700)])
    np.testing.assert_array_equal(got, np.array(exp, dtype=np.uint8))
    assert t.size() == len(seen) == 36
    q = np.array([[0, 0], [5, 5 << 40], [6, 0], [0, 6 << 40], [1, 1]], dtype=np.uint64)
    np.testing.assert_array_equal(t.lookup(q), [1, 1, 0, 0, 0])
    assert set(map(tuple, t.export().tolist())) == seen


@pytest.mark.parametrize("words", [1, 3, 8])
def test_oracle_long_find_or_put_lookup_export_against_brute_force(oracle_lib, words):
    # Keys of `words` words drawn from 3 values per word, so that many keys
    # agree on all but one word; a Python set of tuples is the brute force.
    rng = np.random.default_rng(words)
    vals = np.array([0, 7, 2 ** 64 - 1], dtype=np.uint64)
    keys = vals[rng.integers(0, 3, size=(4000, words))]
    t = oracle_lib.OracleTableLong(words)
    seen, exp = set(), []
    for row in map(tuple, keys.tolist()):
        exp.append(int(row not in seen))
        seen.add(row)
    got = np.concatenate([t.find_or_put(keys[i:i + 900]) for i in range(0, len(keys), 900)])
    np.testing.assert_array_equal(got, np.array(exp, dtype=np.uint8))
    assert t.size() == len(seen) == min(3 ** words, len(seen))
    if words <= 3:
        assert len(seen) == 3 ** words             # every combination drawn
    absent = np.full((1, words), 5, dtype=np.uint64)
    q = np.concatenate([keys[:50], absent])
    np.testing.assert_array_equal(t.lookup(q), [1] * 50 + [0])
    assert set(map(tuple, t.export().tolist())) == seen


def test_oracle_long_reduces_to_the_one_and_two_word_sets(oracle_lib):
    # With one word the long-key set is the 64-bit set; with two, the
    # 128-bit set: the same flags, sizes and contents on the same stream.
    rng = np.random.default_rng(9)
    k1 = rng.integers(0, 500, size=5000).astype(np.uint64)
    a, b = oracle_lib.OracleTableLong(1), oracle_lib.OracleTable()
    np.testing.assert_array_equal(a.find_or_put(k1.reshape(-1, 1)), b.find_or_put(k1))
    assert a.size() == b.size()
    k2 = rng.integers(0, 40, size=(5000, 2)).astype(np.uint64)
    c, d = oracle_lib.OracleTableLong(2), oracle_lib.OracleTable128()
    np.testing.assert_array_equal(c.find_or_put(k2), d.find_or_put(k2))
    assert set(map(tuple, c.export().tolist())) == set(map(tuple, d.export().tolist()))


def _component_hist(m, c):
    a = sp.lil_matrix((int(m.L[c]), int(m.L[c])))
    for u in range(int(m.L[c])):
        for j in range(int(m.deg[c, u])):
            a[u, int(m.tgt[c, u, j])] = 1
    d = shortest_path(a.tocsr(), unweighted=True, indices=0)
    return np.bincount(d[np.isfinite(d)].astype(np.int64))


@pytest.mark.parametrize("seed", [21, 22])
def test_wide_bfs_closed_form_without_sync(oracle_lib, seed):
    # 16 components x 5 bits = 80-bit vectors (component 12 straddles the two
    # words): reachable = product of windows, levels = convolution of the
    # per-component distance histograms, and every stored state decodes to
    # local states inside each component's window.
    R = [2, 3, 2, 2, 3, 2, 2, 2, 2, 2, 2, 2, 3, 2, 2, 2]
    m = ss.random_model(seed, C=16, L=32, R=R, p_sync=0.0, P=0)
    assert m.total_bits == 80 and m.key_width == 128
    res = oracle_lib.bfs(m, max_states=1 << 20, wide=True)
    assert res.rc == 0 and res.total == int(np.prod(R))
    poly = np.array([1], dtype=np.int64)
    for c in range(m.C):
        poly = np.convolve(poly, _component_hist(m, c))
    np.testing.assert_array_equal(res.level_sizes, poly)
    full = res.states[:, 0].astype(object) | (res.states[:, 1].astype(object) << 64)
    assert len(set(full.tolist())) == res.total
    off = 0
    for c in range(m.C):
        loc = np.array([(v >> off) & 31 for v in full.tolist()])
        assert loc.max() < R[c] and len(np.unique(loc)) == R[c]
        off += 5


def test_wide_successors_and_bfs_agree_with_the_64_bit_path(oracle_lib):
    # A model that fits 64 bits gives the same successors and levels either way.
    m = ss.random_model(7, C=6, L=[8, 4, 8, 16, 4, 8], R=[5, 4, 6, 7, 3, 5], p_sync=0.4, P=3)
    for s in [0, 3, 100, 4000]:
        a = np.sort(oracle_lib.successors(m, s))
        w = oracle_lib.successors128(m, s)
        assert (w[:, 1] == 0).all()
        np.testing.assert_array_equal(np.sort(w[:, 0]), a)
    r64 = oracle_lib.bfs(m, max_states=1 << 20)
    r128 = oracle_lib.bfs(m, max_states=1 << 20, wide=True)
    np.testing.assert_array_equal(r64.level_sizes, r128.level_sizes)
    np.testing.assert_array_equal(r64.level_succ, r128.level_succ)
    assert set(r64.states.tolist()) == set(r128.states[:, 0].tolist())
