// Cuckoo hashing after Alcantara et al. (Section 4.1 of the paper).
//
// Slots hold one packed 64-bit word (32-bit key | 32-bit value, or a 64-bit
// key) so a slot moves atomically.  One thread handles one key.
//
// find-or-put of a batch runs as two kernels:
//  1. probe: look each key up in its k slots h_1..h_k (and the stash); a key
//     that is absent claims its key in a per-batch dedup set, and the single
//     claimant per distinct key becomes a "winner" (is_new = 1) appended to
//     a compact list.
//  2. insert: each winner runs the eviction chain: exchange the word into
//     its first slot; if the slot held a word k', find a with h_a(k') = slot
//     and move k' to h_{a+1}(k') (Fig. 2: key 18 evicts 26 from its h_2 slot
//     and 26 moves to h_3), until an empty slot takes the word or
//     max_evictions is reached; then the stash takes it (Section 4.1: a small
//     stash, and a rebuild with new hash constants when it overflows).
//     Section 4.1 starts every chain at h_1.  Here a chain starts by default
//     at the first of h_1..h_k that the probe saw EMPTY (h_1 if none): the
//     probe has read those slots anyway, and most new keys then need one
//     exchange instead of an eviction at h_1 (t.chain_h1 = 1 keeps h_1).
//
// The probe stops at an empty h_1 (a key is never stored past an empty
// slot of its own).  Why that holds with either start: slots never return
// to EMPTY (an exchange always leaves a word), a chain's key is placed at
// h_j only when h_1..h_(j-1) were seen occupied, and an evicted key moves
// from h_a to h_(a+1) with h_a now occupied by its evictor.
//
// Why the dedup set: the paper's duplicate handling (Section 5.1.1: a thread
// that evicts its own key stops) does not stop a duplicate whose first copy
// was just evicted by a third key's chain, so the same key could be stored
// twice with two is_new flags.  The table is not written between the probe
// and the insert kernel, so every winner is truly absent and all winners are
// distinct -- the precondition of Alcantara's insertion.
#include "ht_internal.cuh"

namespace ht {
namespace {

#ifndef HT_CUCKOO_KEYS_PER_THREAD
#define HT_CUCKOO_KEYS_PER_THREAD 4
#endif
constexpr int kU = HT_CUCKOO_KEYS_PER_THREAD;   // keys in flight per thread
#ifndef HT_CUCKOO_PROBE_MIN_BLOCKS
#define HT_CUCKOO_PROBE_MIN_BLOCKS 3
#endif
#ifndef HT_CUCKOO_INSERT_MIN_BLOCKS
#define HT_CUCKOO_INSERT_MIN_BLOCKS 3
#endif

// Probe (and, for find-or-put, dedup).  Each thread holds U keys of a round,
// strided by the grid so every load of keys stays coalesced; all U first
// probes are issued together, then all remaining probes of the misses, then
// every miss's first dedup claim, so U memory latencies overlap.  KH bounds
// the table's k at compile time (4 for the usual k <= 4, else 8): the probe
// words in flight are held in registers, and sizing them for k <= 4 keeps
// enough warps resident per SM.
#ifndef HT_CUCKOO_INSERT_PREFETCH
#define HT_CUCKOO_INSERT_PREFETCH 1
#endif
#ifndef HT_CUCKOO_PROBE_SPLIT
#define HT_CUCKOO_PROBE_SPLIT 2
#endif
#ifndef HT_CUCKOO_STAGE
#define HT_CUCKOO_STAGE 128                    // staged winners per warp
#endif

// A winner waiting in a warp's shared-memory stage: its record and its
// position in the batch (to clear its flag if the list turns out full).
struct StagedWinner {
    uint64_t word;
    uint64_t i;
    uint32_t spos;
    uint32_t start;
};

template <int KW, bool VALUES, bool LOOKUP, int KH>
__global__ void __launch_bounds__(kBlock, KH <= 4 ? HT_CUCKOO_PROBE_MIN_BLOCKS : 1)
cuckoo_probe_kernel(const DevTable t, const DevScratch sc, uint32_t parity,
                    const void* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t n,
                    const unsigned long long* __restrict__ d_n, uint64_t off,
                    uint8_t* __restrict__ out_flag, uint32_t* __restrict__ out_val) {
    using K = Keys<KW>;
    if (d_n) {                                   // batch size produced on the device
        const uint64_t total = __ldcg(d_n);
        n = total > off ? min(n, total - off) : 0;
    }
    const uint32_t stash_used = __ldcg(&t.ctr->stash_used);
    const uint32_t ovf_used = __ldcg(&t.ctr->ovf_used);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t rounds = (n + stride * kU - 1) / (stride * kU);     // warp-uniform trip count
    const uint64_t dseed = t.aux_seed * 3 + 1;
    const int lane = threadIdx.x & 31;
    unsigned long long probes = 0;            // slots read (h_1, then h_2..h_k if h_1 is occupied)
    unsigned long long misses = 0, miss_reads = 0;   // keys found nowhere, and the slots they read
    constexpr int kStage = LOOKUP ? 1 : HT_CUCKOO_STAGE;
    __shared__ StagedWinner s_win[kBlock / 32][kStage];
    StagedWinner* stage = s_win[threadIdx.x >> 5];
    uint32_t pend = 0;
    // Lists the staged winners: one atomic on the winner count per flush.
    // Entries past the list's capacity (more winners than the table holds)
    // give their claim back, are reported dropped and lose their flag.
    auto flush = [&]() {
        __syncwarp();
        if (pend) {
            unsigned int b = 0;
            if (lane == 0) b = atomicAdd(&t.ctr->winners[parity], pend);
            b = __shfl_sync(0xFFFFFFFFu, b, 0);
            for (uint32_t j = lane; j < pend; j += 32) {
                const StagedWinner e = stage[j];
                const uint64_t at = uint64_t(b) + j;
                if (at < sc.win_cap) {
                    Winner wn;
                    wn.word = e.word;
                    wn.spos = e.spos;
                    wn.start = e.start;
                    sc.win[at] = wn;
                } else {
                    sc.set[e.spos] = kEmpty;       // no insert will clear its claim
                    set_flag(t.ctr, kFlagDropped);
                    atomicAdd(&t.ctr->dropped, 1ull);
                    if (out_flag) out_flag[e.i] = 0;
                }
            }
        }
        __syncwarp();
        pend = 0;
    };
    // The next round's keys are loaded while this round waits on the table.
    uint64_t next_key[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        const uint64_t i = uint64_t(u) * stride + tid;
        next_key[u] = i < n ? K::load(keys, i) : 0;
    }
    for (uint64_t r = 0; r < rounds; ++r) {
        uint64_t key[kU], w[kU];
        bool act[kU], found[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            const uint64_t i = (r * kU + u) * stride + tid;
            act[u] = i < n;
            key[u] = next_key[u];
            const uint64_t j = ((r + 1) * kU + u) * stride + tid;
            if (j < n) next_key[u] = K::load(keys, j);
            if (act[u] && K::reserved(key[u])) {
                set_flag(t.ctr, kFlagInvalidKey);
                act[u] = false;
            }
        }
        // Section 4.1: a key is found in at most k probes; h_1 first.
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (act[u]) w[u] = __ldcg(reinterpret_cast<const unsigned long long*>(t.slots + hidx(key[u], t.seed[0], t.nslots)));
        // An empty h_1 slot ends the table probe: a key stored at h_j has
        // h_1 .. h_{j-1} all occupied (see the top of this file).  A miss at
        // table load a then costs 1 + a (k - 1) probes, not k.
        bool more[kU], occ1[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            found[u] = act[u] && K::keyof(w[u]) == key[u];
            more[u] = act[u] && !found[u] && !K::empty(w[u]);
            occ1[u] = more[u];
            probes += act[u] ? 1u : 0u;
        }
        // The chain start of a miss: the first of h_2..h_k seen EMPTY (0 =
        // h_1: empty, or every slot occupied).
        uint32_t start[kU];
        uint64_t ws[kU][KH];
#pragma unroll
        for (int u = 0; u < kU; ++u) start[u] = 0;
        // h_2..h_k in groups [a0, a1): the slots of a group are read together,
        // and a key goes on to the next group only while it is neither found
        // nor past an EMPTY slot (a key never sits past an empty slot of its
        // own).  HT_CUCKOO_PROBE_SPLIT: 0 one group; 1 h_2, then the rest;
        // 2 (default) one slot at a time.  The probe is bound by the random
        // lines it reads, not by its round trips: one slot at a time reads
        // 1.63 slots per key over a fill to load 0.8 instead of 2.06, and a
        // launch takes 0.141 instead of 0.157 ms.
        auto probe_group = [&](int a0, int a1) {
#pragma unroll
            for (int u = 0; u < kU; ++u)
#pragma unroll
                for (int a = 1; a < KH; ++a)
                    if (a >= a0 && a < a1 && a < int(t.k) && more[u]) {
                        ws[u][a] = __ldcg(reinterpret_cast<const unsigned long long*>(t.slots + hidx(key[u], t.seed[a], t.nslots)));
                        ++probes;
                    }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                if (!more[u]) continue;
#pragma unroll
                for (int a = KH - 1; a >= 1; --a)
                    if (a >= a0 && a < a1 && a < int(t.k)) {
                        if (K::keyof(ws[u][a]) == key[u]) {
                            found[u] = true;
                            w[u] = ws[u][a];
                        }
                        if (K::empty(ws[u][a])) start[u] = uint32_t(a);
                    }
                more[u] = !found[u] && start[u] == 0;
            }
        };
        if (HT_CUCKOO_PROBE_SPLIT == 0) {
            probe_group(1, KH);
        } else if (HT_CUCKOO_PROBE_SPLIT == 1) {
            probe_group(1, 2);
            bool any = false;
#pragma unroll
            for (int u = 0; u < kU; ++u) any |= more[u];
            if (__any_sync(0xFFFFFFFFu, any)) probe_group(2, KH);
        } else {
#pragma unroll
            for (int a = 1; a < KH; ++a) {
                bool any = false;
#pragma unroll
                for (int u = 0; u < kU; ++u) any |= more[u];
                if (a < int(t.k) && __any_sync(0xFFFFFFFFu, any)) probe_group(a, a + 1);
            }
        }
        if (stash_used | ovf_used) {
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (act[u] && !found[u]) found[u] = find_spill<KW>(t, key[u], stash_used, ovf_used, &w[u]);
        }
        // The slots read by the keys found nowhere (the table counters keep
        // them apart from the hits' reads).
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (act[u] && !found[u]) {
                ++misses;
                const uint32_t k = t.k;
                miss_reads += !occ1[u] ? 1u
                              : HT_CUCKOO_PROBE_SPLIT == 0 ? k
                              : HT_CUCKOO_PROBE_SPLIT == 1 ? (start[u] == 1 ? 2u : k)
                                                           : (start[u] ? 1u + start[u] : k);
            }
        if constexpr (LOOKUP) {
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint64_t i = (r * kU + u) * stride + tid;
                if (i < n) {
                    if (out_flag) out_flag[i] = uint8_t(found[u]);
                    if (out_val) out_val[i] = found[u] ? K::value(w[u]) : 0u;
                }
            }
        } else {
            // In-batch dedup: the one claimant of each absent key wins.  Every
            // miss first CASes its key into its slot of the claim set (kept in
            // L2); a slot holding another key sends it on by linear probing.
            uint32_t spos[kU];
            uint64_t sw[kU];
            bool need[kU], winner[kU];
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                need[u] = act[u] && !found[u];
                spos[u] = uint32_t(mix64(key[u] ^ dseed) & sc.mask);
                sw[u] = kEmpty;
                if (need[u]) sw[u] = atomicCAS(reinterpret_cast<unsigned long long*>(sc.set + spos[u]), kEmpty, key[u]);
            }
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                winner[u] = false;
                if (!need[u]) continue;
                if (sw[u] == kEmpty) {
                    winner[u] = true;                          // our CAS filled the empty slot
                } else if (K::keyof(sw[u]) != key[u]) {        // another key sits there: probe on
                    uint32_t at = 0;
                    const uint32_t next = spos[u] + 1 == uint32_t(sc.mask + 1) ? 0u : spos[u] + 1;
                    const int rc = lp_insert<KW>(sc.set, uint32_t(sc.mask + 1), next, key[u], key[u], &at);
                    winner[u] = rc == 1;
                    spos[u] = at;
                    if (rc < 0) {                              // more distinct misses than the table holds
                        set_flag(t.ctr, kFlagDropped);
                        atomicAdd(&t.ctr->dropped, 1ull);
                    }
                }
            }
            // The round's winners go to the warp's stage in shared memory,
            // listed with one atomic per flush rather than one per round, so
            // the next round does not wait on a shared counter.
#pragma unroll
            for (int u = 0; u < kU; ++u) {
                const uint64_t i = (r * kU + u) * stride + tid;
                const unsigned wm = __ballot_sync(0xFFFFFFFFu, winner[u]);
                if (wm) {
                    if (pend + __popc(wm) > uint32_t(kStage)) flush();
                    if (winner[u]) {
                        StagedWinner& e = stage[pend + __popc(wm & ((1u << lane) - 1))];
                        e.word = K::word(key[u], VALUES ? vals[i] : 0u);
                        e.i = i;
                        e.spos = spos[u];
                        e.start = t.chain_h1 ? 0u : start[u];
                    }
                    pend += __popc(wm);
                }
                if (i < n && out_flag) out_flag[i] = uint8_t(winner[u]);
            }
        }
    }
    if constexpr (!LOOKUP) flush();
    for (int o = 16; o; o >>= 1) {
        probes += __shfl_down_sync(0xFFFFFFFFu, probes, o);
        misses += __shfl_down_sync(0xFFFFFFFFu, misses, o);
        miss_reads += __shfl_down_sync(0xFFFFFFFFu, miss_reads, o);
    }
    if (lane == 0 && probes) atomicAdd(&t.ctr->probes, probes);
    if (lane == 0 && misses) {
        atomicAdd(&t.ctr->probe_misses, misses);
        atomicAdd(&t.ctr->probe_miss_reads, miss_reads);
    }
}

// Eviction-chain insert of the winners.  Each thread keeps U chains in
// flight so their exchanges overlap, and a chain that ends (an empty slot,
// or the stash) is replaced at once by the thread's next winner: chain
// lengths vary widely at high load, and refilling keeps every slot of the
// thread busy instead of waiting for the longest chain of a round.
template <int KW, bool APPEND>
__global__ void __launch_bounds__(kBlock, HT_CUCKOO_INSERT_MIN_BLOCKS)
cuckoo_insert_kernel(const DevTable t, const DevScratch sc, uint32_t parity, uint64_t max_winners,
                     typename Keys<KW>::T* __restrict__ new_out, unsigned long long* __restrict__ new_count,
                     uint64_t new_cap) {
    using K = Keys<KW>;
    const uint64_t count = min(uint64_t(__ldcg(&t.ctr->winners[parity])), max_winners);
    // The other parity's list was consumed by the previous insert kernel on
    // this stream; reset its counter for the next probe kernel.
    if (blockIdx.x == 0 && threadIdx.x == 0) t.ctr->winners[parity ^ 1u] = 0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    if (APPEND) {
        // Every winner is a new key: append them all, warp-aggregated.
        const uint64_t rounds = (count + stride - 1) / stride;
        for (uint64_t r = 0; r < rounds; ++r) {
            const uint64_t i = r * stride + tid;
            const uint64_t key = i < count ? K::keyof(sc.win[i].word) : 0;
            warp_append<typename K::T>(i < count, typename K::T(key), new_out, new_count, new_cap);
        }
    }
    unsigned long long placed = 0, exchanges = 0;
    uint64_t next = tid;                  // this thread's next winner: tid, tid + stride, ...
    uint64_t word[kU], pos[kU];
    uint32_t evictions[kU];
    bool live[kU];
    // Each chain slot's next winner record is loaded one winner ahead, so a
    // slot that frees up starts its next chain without waiting for the read.
    Winner pre[kU];
    bool pre_ok[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        live[u] = false;
        word[u] = 0;
        pos[u] = 0;
        evictions[u] = 0;
        pre_ok[u] = HT_CUCKOO_INSERT_PREFETCH && next < count;
        if (pre_ok[u]) pre[u] = sc.win[next];
        if (HT_CUCKOO_INSERT_PREFETCH) next += stride;
    }
    // Bounded: each winner is taken once and its chain ends after at most
    // max_evictions + 1 exchanges.
    for (;;) {
        bool any = false;
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (!live[u] && (HT_CUCKOO_INSERT_PREFETCH ? pre_ok[u] : next < count)) {
                Winner wn;
                if (HT_CUCKOO_INSERT_PREFETCH) {
                    wn = pre[u];
                    pre_ok[u] = next < count;
                    if (pre_ok[u]) pre[u] = sc.win[next];
                } else {
                    wn = sc.win[next];
                }
                next += stride;
                sc.set[wn.spos] = kEmpty;      // leave the dedup set empty for the next batch
                word[u] = wn.word;
                pos[u] = hidx(K::keyof(wn.word), t.seed[wn.start < t.k ? wn.start : 0u], t.nslots);
                evictions[u] = 0;
                live[u] = true;
            }
            any |= live[u];
        }
        if (!any) break;
        uint64_t old[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (live[u]) old[u] = atomicExch(reinterpret_cast<unsigned long long*>(t.slots + pos[u]), word[u]);
#pragma unroll
        for (int u = 0; u < kU; ++u) {
            if (!live[u]) continue;
            ++exchanges;
            if (K::empty(old[u])) {
                live[u] = false;
                ++placed;
                continue;
            }
            // Section 4.1: the evicted key k' sat at h_a(k') = pos; it moves
            // on to h_{a+1}(k') (cyclically after h_k).
            word[u] = old[u];
            if (++evictions[u] > t.max_evict) {
                // The chain hit the eviction bound: the held word goes to the stash.
                if (place_spill<KW>(t, K::keyof(word[u]), word[u]) == 1) ++placed;
                live[u] = false;
                continue;
            }
            const uint64_t key = K::keyof(old[u]);
            uint32_t a = 0;
            for (; a + 1 < t.k; ++a)
                if (hidx(key, t.seed[a], t.nslots) == pos[u]) break;
            const uint32_t nxt = (a + 1 == t.k) ? 0u : a + 1;
            pos[u] = hidx(key, t.seed[nxt], t.nslots);
        }
    }
    for (int o = 16; o; o >>= 1) {
        placed += __shfl_down_sync(0xFFFFFFFFu, placed, o);
        exchanges += __shfl_down_sync(0xFFFFFFFFu, exchanges, o);
    }
    if ((threadIdx.x & 31) == 0 && placed) atomicAdd(&t.ctr->size, placed);
    if ((threadIdx.x & 31) == 0 && exchanges) atomicAdd(&t.ctr->exchanges, exchanges);
}

}  // namespace

cudaError_t cuckoo_probe(int kw, const DevTable& t, const DevScratch& sc, uint32_t parity,
                         const void* keys, const uint32_t* vals, uint64_t n,
                         const unsigned long long* d_n, uint64_t off, uint8_t* is_new, cudaStream_t s,
                         const L2Window& w) {
    ProfScope ps(kKCuckooProbe, s);
#define L(KW, V)                                                                                        \
    {                                                                                                   \
        auto k = t.k <= 4 ? cuckoo_probe_kernel<KW, V, false, 4> : cuckoo_probe_kernel<KW, V, false, kMaxCuckooHashes>; \
        return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, sc, parity, keys, vals, n, \
                          d_n, off, is_new, (uint32_t*)nullptr);                                        \
    }
    if (kw == 32) {
        if (vals) L(32, true) else L(32, false)
    }
    L(64, false)
#undef L
}

cudaError_t cuckoo_insert(int kw, const DevTable& t, const DevScratch& sc, uint32_t parity,
                          void* new_out, unsigned long long* new_count, uint64_t new_cap,
                          uint64_t max_winners, cudaStream_t s, const L2Window& w) {
    ProfScope ps(kKCuckooInsert, s);
#define L(KW, A)                                                                                        \
    {                                                                                                   \
        auto k = cuckoo_insert_kernel<KW, A>;                                                           \
        return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, sc, parity, max_winners, \
                          static_cast<typename Keys<KW>::T*>(new_out), new_count, new_cap);             \
    }
    if (kw == 32) {
        if (new_out) L(32, true) else L(32, false)
    }
    if (new_out) L(64, true)
    L(64, false)
#undef L
}

cudaError_t cuckoo_lookup(int kw, const DevTable& t, const void* keys, uint64_t n, uint32_t* vals,
                          uint8_t* found, cudaStream_t s, const L2Window& w) {
    ProfScope ps(kKCuckooLookup, s);
    DevScratch none{};
    if (kw == 32) {
        auto k = t.k <= 4 ? cuckoo_probe_kernel<32, false, true, 4> : cuckoo_probe_kernel<32, false, true, kMaxCuckooHashes>;
        return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, none, 0u, keys,
                          (const uint32_t*)nullptr, n, (const unsigned long long*)nullptr, uint64_t(0), found, vals);
    }
    auto k = t.k <= 4 ? cuckoo_probe_kernel<64, false, true, 4> : cuckoo_probe_kernel<64, false, true, kMaxCuckooHashes>;
    return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, none, 0u, keys,
                      (const uint32_t*)nullptr, n, (const unsigned long long*)nullptr, uint64_t(0), found, vals);
}

}  // namespace ht
