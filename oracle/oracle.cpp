// CPU oracle for the hash-table hot path.  TEST INFRASTRUCTURE ONLY.
//
// Only the test suite, the smoke check and the benchmark's CPU-baseline leg
// load this library.  The CUDA path never links, includes or calls it, and
// it shares no code with the CUDA path.
//
// What it computes is the plain definition of each operation, written
// single-threaded on top of the C++ standard library's hash containers:
//
//  * find-or-put (Section 5 of the paper: every element of the sequence is
//    first looked up; if present nothing happens, otherwise it is inserted;
//    the time to find-or-insert the whole sequence is what is measured).
//    Processed in batch order: is_new[i] = (keys[i] not in S); S += keys[i].
//  * insert-if-absent with a 32-bit value (a duplicate insert keeps the
//    value already stored, Section 5.1.1's duplicate handling), and lookup.
//  * breadth-first state-space exploration (Section 3.2: open and closed
//    sets; successor vectors built from each process's enabled transitions):
//    L_0 = {s0}, L_{d+1} = succ(L_d) minus every state seen so far.
//
// The successor relation follows the model format documented in
// workloads/statespace.py (interleaving of local actions plus binary
// synchronisation on pair labels); that format is the project's own, since
// the paper's models are not available.
//
// Nothing here models hash functions, buckets, slots or eviction: those are
// not observable in the results, so parity is checked on sets, flags and
// values only.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <unordered_map>
#include <unordered_set>
#include <utility>
#include <set>
#include <vector>

namespace {

struct Table {
    std::unordered_map<uint64_t, uint32_t> m;
};

// 128-bit keys (two 64-bit words, low word first): the same set definition.
struct PairHash {
    size_t operator()(const std::pair<uint64_t, uint64_t>& k) const {
        return std::hash<uint64_t>()(k.first) ^ (std::hash<uint64_t>()(k.second) * 0x9E3779B97F4A7C15ull);
    }
};

struct Table128 {
    std::unordered_set<std::pair<uint64_t, uint64_t>, PairHash> s;
};

}  // namespace

extern "C" {

void* orc_new(uint64_t reserve) {
    Table* t = new Table();
    if (reserve) t->m.reserve(reserve);
    return t;
}

void orc_free(void* h) { delete static_cast<Table*>(h); }

uint64_t orc_size(const void* h) { return static_cast<const Table*>(h)->m.size(); }

// Section 5: for each element in sequence order, look it up; insert it if it
// is absent.  is_new[i] records which of the two happened.  A stored value of
// 0 is used for maps (find-or-put carries no value).
void orc_find_or_put(void* h, const uint64_t* keys, uint64_t n, uint8_t* is_new) {
    Table* t = static_cast<Table*>(h);
    for (uint64_t i = 0; i < n; ++i) {
        bool inserted = t->m.emplace(keys[i], 0u).second;
        if (is_new) is_new[i] = inserted ? 1 : 0;
    }
}

// Insert-if-absent: the first value stored for a key is kept.
void orc_insert(void* h, const uint64_t* keys, const uint32_t* vals, uint64_t n) {
    Table* t = static_cast<Table*>(h);
    for (uint64_t i = 0; i < n; ++i) t->m.emplace(keys[i], vals ? vals[i] : 0u);
}

// Lookup: found[i] = keys[i] in S; vals[i] = its stored value (0 if absent).
void orc_lookup(const void* h, const uint64_t* keys, uint64_t n, uint8_t* found, uint32_t* vals) {
    const Table* t = static_cast<const Table*>(h);
    for (uint64_t i = 0; i < n; ++i) {
        auto it = t->m.find(keys[i]);
        bool f = it != t->m.end();
        if (found) found[i] = f ? 1 : 0;
        if (vals) vals[i] = f ? it->second : 0u;
    }
}

// Copy out up to cap (key, value) pairs in unspecified order; returns |S|.
uint64_t orc_export(const void* h, uint64_t* keys, uint32_t* vals, uint64_t cap) {
    const Table* t = static_cast<const Table*>(h);
    uint64_t i = 0;
    for (const auto& kv : t->m) {
        if (i < cap) {
            if (keys) keys[i] = kv.first;
            if (vals) vals[i] = kv.second;
        }
        ++i;
    }
    return i;
}

// ---------------------------------------------------------------------------
// State-space models.  Same field layout as the tables drawn by
// workloads/statespace.py (16 components, 32 local states, 4 transitions per
// local state, 8 sync pairs).
// ---------------------------------------------------------------------------
struct orc_model {
    int32_t C;
    int32_t P;
    uint8_t bits[16];
    uint8_t pc1[8];
    uint8_t pc2[8];
    uint8_t deg[16][32];
    uint8_t tgt[16][32][4];
    uint8_t lab[16][32][4];
};

// 128-bit sets: keys[2i] is key i's low word, keys[2i+1] its high word.
void* orc128_new(uint64_t reserve) {
    Table128* t = new Table128();
    if (reserve) t->s.reserve(reserve);
    return t;
}

void orc128_free(void* h) { delete static_cast<Table128*>(h); }

uint64_t orc128_size(const void* h) { return static_cast<const Table128*>(h)->s.size(); }

// find-or-put in order: is_new[i] = key i not yet in the set; then it is.
void orc128_find_or_put(void* h, const uint64_t* keys, uint64_t n, uint8_t* is_new) {
    auto& s = static_cast<Table128*>(h)->s;
    for (uint64_t i = 0; i < n; ++i) {
        const bool inserted = s.emplace(keys[2 * i], keys[2 * i + 1]).second;
        if (is_new) is_new[i] = inserted ? 1 : 0;
    }
}

void orc128_lookup(const void* h, const uint64_t* keys, uint64_t n, uint8_t* found) {
    const auto& s = static_cast<const Table128*>(h)->s;
    for (uint64_t i = 0; i < n; ++i) found[i] = s.count({keys[2 * i], keys[2 * i + 1]}) ? 1 : 0;
}

uint64_t orc128_export(const void* h, uint64_t* keys, uint64_t cap) {
    const auto& s = static_cast<const Table128*>(h)->s;
    uint64_t i = 0;
    for (const auto& k : s) {
        if (i < cap) {
            keys[2 * i] = k.first;
            keys[2 * i + 1] = k.second;
        }
        ++i;
    }
    return i;
}

// Sets of long keys (W 64-bit words each, W >= 1): keys[W*i .. W*i+W) is
// key i.  The same definition as above -- find, else insert, in order
// (Section 5) -- over an ordered set of word vectors, so two keys are equal
// exactly when all their words are.
struct TableLong {
    uint32_t words;
    std::set<std::vector<uint64_t>> s;
};

void* orclong_new(uint32_t words) {
    if (words == 0) return nullptr;
    TableLong* t = new TableLong();
    t->words = words;
    return t;
}

void orclong_free(void* h) { delete static_cast<TableLong*>(h); }

uint64_t orclong_size(const void* h) { return static_cast<const TableLong*>(h)->s.size(); }

void orclong_find_or_put(void* h, const uint64_t* keys, uint64_t n, uint8_t* is_new) {
    TableLong* t = static_cast<TableLong*>(h);
    const uint32_t w = t->words;
    for (uint64_t i = 0; i < n; ++i) {
        const bool inserted = t->s.insert(std::vector<uint64_t>(keys + w * i, keys + w * i + w)).second;
        if (is_new) is_new[i] = inserted ? 1 : 0;
    }
}

void orclong_lookup(const void* h, const uint64_t* keys, uint64_t n, uint8_t* found) {
    const TableLong* t = static_cast<const TableLong*>(h);
    const uint32_t w = t->words;
    for (uint64_t i = 0; i < n; ++i)
        found[i] = t->s.count(std::vector<uint64_t>(keys + w * i, keys + w * i + w)) ? 1 : 0;
}

// Copies out up to cap keys in the set's (lexicographic) order; returns |S|.
uint64_t orclong_export(const void* h, uint64_t* keys, uint64_t cap) {
    const TableLong* t = static_cast<const TableLong*>(h);
    uint64_t i = 0;
    for (const auto& k : t->s) {
        if (i < cap)
            for (uint32_t j = 0; j < t->words; ++j) keys[t->words * i + j] = k[j];
        ++i;
    }
    return i;
}

}  // extern "C"

namespace {

// Component c's local state is bits [off[c], off[c] + bits[c]) of the state
// vector; S is the vector's type (64 bits, or 128 for wider models).
template <class S>
struct Layout {
    int off[16];
    S mask[16];
};

template <class S>
Layout<S> layout_of(const orc_model* m) {
    Layout<S> l{};
    int o = 0;
    for (int c = 0; c < m->C; ++c) {
        l.off[c] = o;
        l.mask[c] = (S(1) << m->bits[c]) - 1;
        o += m->bits[c];
    }
    return l;
}

template <class S>
inline uint64_t local_of(const Layout<S>& l, S s, int c) { return uint64_t((s >> l.off[c]) & l.mask[c]); }

template <class S>
inline S with_local(const Layout<S>& l, S s, int c, uint64_t v) {
    return (s & ~(l.mask[c] << l.off[c])) | (S(v) << l.off[c]);
}

// Successors of s, in a fixed order (components' local actions, then pairs).
template <class S, class Emit>
void successors(const orc_model* m, const Layout<S>& l, S s, Emit emit) {
    for (int c = 0; c < m->C; ++c) {
        uint64_t u = local_of(l, s, c);
        for (int j = 0; j < m->deg[c][u]; ++j)
            if (m->lab[c][u][j] == 0) emit(with_local(l, s, c, m->tgt[c][u][j]));
    }
    for (int p = 0; p < m->P; ++p) {
        int c1 = m->pc1[p], c2 = m->pc2[p];
        uint64_t u1 = local_of(l, s, c1), u2 = local_of(l, s, c2);
        for (int j1 = 0; j1 < m->deg[c1][u1]; ++j1) {
            if (m->lab[c1][u1][j1] != p + 1) continue;
            for (int j2 = 0; j2 < m->deg[c2][u2]; ++j2) {
                if (m->lab[c2][u2][j2] != p + 1) continue;
                S t = with_local(l, s, c1, m->tgt[c1][u1][j1]);
                emit(with_local(l, t, c2, m->tgt[c2][u2][j2]));
            }
        }
    }
}

using u128 = unsigned __int128;

struct StateHash {
    size_t operator()(uint64_t s) const { return std::hash<uint64_t>()(s); }
    size_t operator()(u128 s) const {
        return std::hash<uint64_t>()(uint64_t(s)) ^ (std::hash<uint64_t>()(uint64_t(s >> 64)) * 0x9E3779B97F4A7C15ull);
    }
};

// Level-synchronous BFS from s0 (see orc_bfs).
template <class S>
int bfs(const orc_model* m, S s0, uint64_t max_states, uint32_t max_levels, uint64_t* level_sizes,
        uint64_t* level_succ, S* states_out, uint64_t states_cap, uint32_t* nlevels, uint64_t* total) {
    const Layout<S> l = layout_of<S>(m);
    std::unordered_map<S, uint32_t, StateHash> seen;  // closed + open sets
    seen.reserve(max_states < (uint64_t(1) << 28) ? max_states + 1 : (uint64_t(1) << 28));
    std::vector<S> cur{s0}, nxt;
    seen.emplace(s0, 0u);
    uint64_t stored = 0;
    auto keep = [&](S s) {
        if (states_out && stored < states_cap) states_out[stored] = s;
        ++stored;
    };
    keep(s0);
    uint32_t d = 0;
    int rc = 0;
    while (!cur.empty()) {
        if (d >= max_levels) { rc = 2; break; }
        level_sizes[d] = cur.size();
        uint64_t gen = 0;
        nxt.clear();
        for (S s : cur) {
            successors(m, l, s, [&](S t) {
                ++gen;
                if (seen.emplace(t, d + 1).second) nxt.push_back(t);
            });
        }
        if (level_succ) level_succ[d] = gen;
        ++d;
        for (S t : nxt) keep(t);
        if (seen.size() > max_states) { rc = 1; break; }
        cur.swap(nxt);
    }
    *nlevels = d;
    *total = stored;
    return rc;
}

}  // namespace

extern "C" {

// All successors of one state; returns how many there are (writes at most cap).
uint64_t orc_successors(const orc_model* m, uint64_t s, uint64_t* out, uint64_t cap) {
    const Layout<uint64_t> l = layout_of<uint64_t>(m);
    uint64_t n = 0;
    successors(m, l, s, [&](uint64_t t) {
        if (n < cap) out[n] = t;
        ++n;
    });
    return n;
}

// Level-synchronous BFS from s0.  level_sizes[d] = |L_d|; level_succ[d] =
// number of successors generated from L_d (with repeats).  states_out (may be
// NULL) receives the states level by level, up to states_cap.  Returns 0 when
// the exploration finished, 1 if more than max_states states were reached,
// 2 if more than max_levels levels were needed.
int orc_bfs(const orc_model* m, uint64_t s0, uint64_t max_states, uint32_t max_levels,
            uint64_t* level_sizes, uint64_t* level_succ, uint64_t* states_out,
            uint64_t states_cap, uint32_t* nlevels, uint64_t* total) {
    return bfs<uint64_t>(m, s0, max_states, max_levels, level_sizes, level_succ, states_out, states_cap, nlevels,
                         total);
}

// The same for models whose state vectors are wider than 64 bits (up to 127):
// a state is two words, low word first (s0, out and states_out likewise).
uint64_t orc_successors128(const orc_model* m, uint64_t s_lo, uint64_t s_hi, uint64_t* out, uint64_t cap) {
    const Layout<u128> l = layout_of<u128>(m);
    const u128 s = (u128(s_hi) << 64) | s_lo;
    uint64_t n = 0;
    successors(m, l, s, [&](u128 t) {
        if (n < cap) {
            out[2 * n] = uint64_t(t);
            out[2 * n + 1] = uint64_t(t >> 64);
        }
        ++n;
    });
    return n;
}

int orc_bfs128(const orc_model* m, uint64_t s0_lo, uint64_t s0_hi, uint64_t max_states, uint32_t max_levels,
               uint64_t* level_sizes, uint64_t* level_succ, uint64_t* states_out, uint64_t states_cap,
               uint32_t* nlevels, uint64_t* total) {
    std::vector<u128> st(states_out ? states_cap : 0);
    const int rc = bfs<u128>(m, (u128(s0_hi) << 64) | s0_lo, max_states, max_levels, level_sizes, level_succ,
                             states_out ? st.data() : nullptr, states_cap, nlevels, total);
    if (states_out)
        for (uint64_t i = 0; i < std::min<uint64_t>(*total, states_cap); ++i) {
            states_out[2 * i] = uint64_t(st[i]);
            states_out[2 * i + 1] = uint64_t(st[i] >> 64);
        }
    return rc;
}

}  // extern "C"
