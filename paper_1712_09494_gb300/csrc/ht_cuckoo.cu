// Cuckoo hashing after Alcantara et al. (Section 4.1 of the paper).
//
// Slots hold one packed 64-bit word (32-bit key | 32-bit value, or a 64-bit
// key) so a slot moves atomically.  One thread handles one key.
//
// find-or-put of a batch runs as two kernels:
//  1. probe: look each key up in its k slots h_1..h_k (and the stash).  An
//     absent key that saw an EMPTY slot stores itself at the first one with
//     a CAS from EMPTY, going on in slot order if another key took it first
//     (is_new = 1 for the copy whose CAS succeeded).  An absent key whose k
//     slots are all full claims its key in a per-batch dedup set, and the
//     single claimant per such key becomes a "winner" (is_new = 1).  Every
//     new key is appended to a compact list.
//  2. insert: each winner runs the eviction chain: exchange the word into
//     h_1; if the slot held a word k', find a with h_a(k') = slot and move
//     k' to h_{a+1}(k') (Fig. 2: key 18 evicts 26 from its h_2 slot and 26
//     moves to h_3), until an empty slot takes the word or max_evictions is
//     reached; then the stash takes it (Section 4.1: a small stash, and a
//     rebuild with new hash constants when it overflows).  Keys stored by
//     the probe are only counted here (and appended, for a frontier).
//     Section 4.1 starts every insertion at h_1 with an exchange.  Here an
//     insertion starts by default at the first of h_1..h_k that the probe
//     saw EMPTY, where it needs no eviction, and only keys with all k slots
//     full start a chain at h_1; t.chain_h1 = 1 keeps the paper's rule (a
//     CAS only at an EMPTY h_1, every other insertion a chain from h_1).
//     A Cuckoo insertion's cost is its atomics (random CASes and exchanges
//     run at the same rate whether their line is in L2 or not), so storing
//     in the probe with the one CAS that also settles duplicates takes the
//     dedup claim off most new keys.
//
// The probe stops at an empty h_1 (a key is never stored past an empty
// slot of its own).  Why that holds: slots never return to EMPTY (a CAS or
// an exchange always leaves a word), a key is stored at h_j only when
// h_1..h_(j-1) were seen occupied, and an evicted key moves from h_a to
// h_(a+1) with h_a now occupied by its evictor.
//
// Why duplicates need care: the paper's duplicate handling (Section 5.1.1:
// a thread that evicts its own key stops) does not stop a duplicate whose
// first copy was just evicted by a third key's chain, so the same key could
// be stored twice with two is_new flags.  Nothing moves a stored key during
// the probe kernel: its only table writes are CASes from EMPTY.  Copies of
// a key that store in the probe claim in slot order, so at most one CAS
// succeeds and a copy probed later finds the key; a copy that saw all k
// slots full read each after it was filled, so no copy stores the key in
// the table during the probe and the dedup set elects one winner.  Every
// winner is thus truly absent and all winners are distinct -- the
// precondition of Alcantara's insertion.
#include "ht_internal.cuh"

namespace ht {
namespace {

#ifndef HT_CUCKOO_KEYS_PER_THREAD
#define HT_CUCKOO_KEYS_PER_THREAD 4
#endif
constexpr int kU = HT_CUCKOO_KEYS_PER_THREAD;   // keys in flight per thread
// Blocks per SM the probe is compiled for: find-or-put holds the CAS
// results of its U keys besides their probe words (2 blocks, no spills: the
// fill is 17% faster than at 3 blocks with spills); lookup keeps 3.
#ifndef HT_CUCKOO_PROBE_MIN_BLOCKS
#define HT_CUCKOO_PROBE_MIN_BLOCKS 2
#endif
#ifndef HT_CUCKOO_LOOKUP_MIN_BLOCKS
#define HT_CUCKOO_LOOKUP_MIN_BLOCKS 3
#endif
// Tables that fit in L2 get a find-or-put probe of kUL2 keys per thread at
// 3 blocks per SM: their keys are mostly hits served by L2, where more warps
// hide more latency (a replay of 10^8 keys of multiplicity 1000: 2.04 ms
// instead of 2.33).  Larger tables keep kU keys at 2 blocks (the 2^27-key
// fill: 18.7 ms instead of 19.2).
#ifndef HT_CUCKOO_KEYS_PER_THREAD_L2
#define HT_CUCKOO_KEYS_PER_THREAD_L2 3
#endif
#ifndef HT_CUCKOO_PROBE_L2_MIN_BLOCKS
#define HT_CUCKOO_PROBE_L2_MIN_BLOCKS 3
#endif
constexpr int kUL2 = HT_CUCKOO_KEYS_PER_THREAD_L2;
#ifndef HT_CUCKOO_INSERT_MIN_BLOCKS
#define HT_CUCKOO_INSERT_MIN_BLOCKS 3
#endif

// Probe (and, for find-or-put, the stores and the dedup).  Each thread
// holds U keys of a round, strided by the grid so every load of keys stays
// coalesced; all U first probes are issued together, then the remaining
// probes of the misses, then the misses' CASes, then the dedup claims of
// the keys that found every slot full, so U memory latencies overlap.  KH bounds
// the table's k at compile time (4 for the usual k <= 4, else 8): the probe
// words in flight are held in registers, and sizing them for k <= 4 keeps
// enough warps resident per SM.
#ifndef HT_CUCKOO_PROBE_SPLIT
#define HT_CUCKOO_PROBE_SPLIT 2
#endif
#ifndef HT_CUCKOO_DIRECT
#define HT_CUCKOO_DIRECT 1                     // absent keys CAS themselves into the EMPTY slot they saw
#endif
#ifndef HT_CUCKOO_STAGE
#define HT_CUCKOO_STAGE 128                    // staged winners per warp
#endif

// Adds the block's per-warp sums (held by each warp's lane 0) to N table
// counters with one atomic per counter and block, not per warp: the last
// step of a kernel, reached by every thread of the block.  At one atomic per
// warp, thousands of warps ending together queued on each counter's L2
// slice, a fixed cost per launch that small launches (a BFS level's chunks)
// paid in full.
template <int N>
__device__ __forceinline__ void block_add_counters(unsigned long long* const (&dst)[N],
                                                   const unsigned long long (&v)[N]) {
    __shared__ unsigned long long s_sum[N][kBlock / 32];
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) s_sum[c][w] = v[c];
    }
    __syncthreads();
    if (threadIdx.x == 0) {
#pragma unroll
        for (int c = 0; c < N; ++c) {
            unsigned long long total = 0;
#pragma unroll
            for (int j = 0; j < kBlock / 32; ++j) total += s_sum[c][j];
            if (total) atomicAdd(dst[c], total);       // no return value: the adds do not wait on each other
        }
    }
}

// The start field of a winner record whose key the probe already stored.
constexpr uint32_t kStartPlaced = 0xFFFFFFFFu;

// A winner waiting in a warp's shared-memory stage: its record and its
// position in the batch (to clear its flag if the list turns out full).
struct StagedWinner {
    uint64_t word;
    uint64_t i;
    uint32_t spos;
    uint32_t start;
};

template <int KW, bool VALUES, bool LOOKUP, int KH, int U = kU>
__global__ void __launch_bounds__(kBlock, KH > 4 ? 1 : LOOKUP ? HT_CUCKOO_LOOKUP_MIN_BLOCKS
                                          : U == kU ? HT_CUCKOO_PROBE_MIN_BLOCKS : HT_CUCKOO_PROBE_L2_MIN_BLOCKS)
cuckoo_probe_kernel(const DevTable t, const DevScratch sc, uint32_t parity,
                    const void* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t n,
                    const unsigned long long* __restrict__ d_n, uint64_t off,
                    uint8_t* __restrict__ out_flag, uint32_t* __restrict__ out_val, bool list_stored) {
    using K = Keys<KW>;
    if (d_n) {                                   // batch size produced on the device
        const uint64_t total = __ldcg(d_n);
        n = total > off ? min(n, total - off) : 0;
    }
    const uint32_t stash_used = __ldcg(&t.ctr->stash_used);
    const uint32_t ovf_used = __ldcg(&t.ctr->ovf_used);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t rounds = (n + stride * U - 1) / (stride * U);     // warp-uniform trip count
    const uint64_t dseed = t.aux_seed * 3 + 1;
    const int lane = threadIdx.x & 31;
    unsigned long long probes = 0;            // slots read (h_1, then h_2..h_k if h_1 is occupied)
    unsigned long long misses = 0, miss_reads = 0;   // keys found nowhere, and the slots they read
    unsigned long long direct = 0;            // CASes of absent keys into table slots
    unsigned long long stored = 0;            // keys stored here and not listed
    constexpr int kStage = LOOKUP ? 1 : HT_CUCKOO_STAGE;
    __shared__ StagedWinner s_win[kBlock / 32][kStage];
    StagedWinner* stage = s_win[threadIdx.x >> 5];
    uint32_t pend = 0;
    // Lists the staged winners: one atomic on the winner count per flush.
    // Entries past the list's capacity (more winners than the table holds)
    // give their claim back, are reported dropped and lose their flag --
    // unless the probe stored them already.
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
                } else if (e.start == kStartPlaced) {
                    atomicAdd(&t.ctr->size, 1ull);     // stored already (it holds no claim)
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
    uint64_t next_key[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        const uint64_t i = uint64_t(u) * stride + tid;
        next_key[u] = i < n ? K::load(keys, i) : 0;
    }
    for (uint64_t r = 0; r < rounds; ++r) {
        uint64_t key[U], w[U];
        bool act[U], found[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t i = (r * U + u) * stride + tid;
            act[u] = i < n;
            key[u] = next_key[u];
            const uint64_t j = ((r + 1) * U + u) * stride + tid;
            if (j < n) next_key[u] = K::load(keys, j);
            if (act[u] && K::reserved(key[u])) {
                set_flag(t.ctr, kFlagInvalidKey);
                act[u] = false;
            }
        }
        // Section 4.1: a key is found in at most k probes; h_1 first.
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (act[u]) w[u] = __ldcg(reinterpret_cast<const unsigned long long*>(t.slots + hidx(key[u], t.seed[0], t.nslots)));
        // An empty h_1 slot ends the table probe: a key stored at h_j has
        // h_1 .. h_{j-1} all occupied (see the top of this file).  A miss at
        // table load a then costs 1 + a (k - 1) probes, not k.
        bool more[U], occ1[U];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            found[u] = act[u] && K::keyof(w[u]) == key[u];
            more[u] = act[u] && !found[u] && !K::empty(w[u]);
            occ1[u] = more[u];
            probes += act[u] ? 1u : 0u;
        }
        // The chain start of a miss: the first of h_2..h_k seen EMPTY (0 =
        // h_1: empty, or every slot occupied).
        uint32_t start[U];
        uint64_t ws[U][KH];
#pragma unroll
        for (int u = 0; u < U; ++u) start[u] = 0;
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
            for (int u = 0; u < U; ++u)
#pragma unroll
                for (int a = 1; a < KH; ++a)
                    if (a >= a0 && a < a1 && a < int(t.k) && more[u]) {
                        ws[u][a] = __ldcg(reinterpret_cast<const unsigned long long*>(t.slots + hidx(key[u], t.seed[a], t.nslots)));
                        ++probes;
                    }
#pragma unroll
            for (int u = 0; u < U; ++u) {
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
            for (int u = 0; u < U; ++u) any |= more[u];
            if (__any_sync(0xFFFFFFFFu, any)) probe_group(2, KH);
        } else {
#pragma unroll
            for (int a = 1; a < KH; ++a) {
                bool any = false;
#pragma unroll
                for (int u = 0; u < U; ++u) any |= more[u];
                if (a < int(t.k) && __any_sync(0xFFFFFFFFu, any)) probe_group(a, a + 1);
            }
        }
        if (stash_used | ovf_used) {
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (act[u] && !found[u]) found[u] = find_spill<KW>(t, key[u], stash_used, ovf_used, &w[u]);
        }
        // The slots read by the keys found nowhere (the table counters keep
        // them apart from the hits' reads; find-or-put only -- counting them
        // costs a lookup registers it spills).
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (!LOOKUP && act[u] && !found[u]) {
                ++misses;
                const uint32_t k = t.k;
                miss_reads += !occ1[u] ? 1u
                              : HT_CUCKOO_PROBE_SPLIT == 0 ? k
                              : HT_CUCKOO_PROBE_SPLIT == 1 ? (start[u] == 1 ? 2u : k)
                                                           : (start[u] ? 1u + start[u] : k);
            }
        if constexpr (LOOKUP) {
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t i = (r * U + u) * stride + tid;
                if (i < n) {
                    if (out_flag) out_flag[i] = uint8_t(found[u]);
                    if (out_val) out_val[i] = found[u] ? K::value(w[u]) : 0u;
                }
            }
        } else {
            // A miss that saw an EMPTY slot stores itself there with a CAS
            // from EMPTY, trying its slots in order from that one: a CAS that
            // returns the key means another copy stored it first (not new);
            // one that returns another key moves on to the next slot, which
            // the CAS reads as well.  This is the bucket scheme's claim in
            // slot order (Section 4.2), over h_a..h_k.  Nothing leaves a slot
            // during the probe kernel, so a key is stored in at most one slot
            // and every copy probed later finds it; a copy that saw all k
            // slots full read them after they were full, so no copy stores
            // it in the table here.  With t.chain_h1 only an EMPTY h_1 is
            // tried (Section 4.1 starts every insertion at h_1).
            bool placed[U], claim[U], pend_cas[U];
            uint32_t at[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const bool miss = act[u] && !found[u];
                at[u] = occ1[u] ? start[u] : 0u;
                pend_cas[u] = HT_CUCKOO_DIRECT && miss && (!occ1[u] || (start[u] != 0 && !t.chain_h1));
                claim[u] = miss && !pend_cas[u];
                placed[u] = false;
            }
#pragma unroll
            for (int pass = 0; pass < KH; ++pass) {
                bool any = false;
#pragma unroll
                for (int u = 0; u < U; ++u) any |= pend_cas[u];
                if (!__any_sync(0xFFFFFFFFu, any)) break;
                uint64_t cw[U];
#pragma unroll
                for (int u = 0; u < U; ++u)
                    if (pend_cas[u]) {
                        const uint64_t i = (r * U + u) * stride + tid;
                        cw[u] = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + hidx(key[u], t.seed[at[u]], t.nslots)),
                                          kEmpty, K::word(key[u], VALUES ? vals[i] : 0u));
                        ++direct;
                    }
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    if (!pend_cas[u]) continue;
                    if (cw[u] == kEmpty) {
                        placed[u] = true;
                        pend_cas[u] = false;
                    } else if (K::keyof(cw[u]) == key[u]) {
                        pend_cas[u] = false;                   // another copy stored it
                    } else if (t.chain_h1 || at[u] + 1 >= t.k) {
                        claim[u] = true;                       // every slot is full now
                        pend_cas[u] = false;
                    } else {
                        ++at[u];
                    }
                }
            }
            // The misses that found all k slots full go through the claim
            // set: the one claimant of each such key wins and runs an
            // eviction chain from h_1 in the insert kernel.  Each CASes its
            // key into its slot of the claim set (kept in L2); a slot holding
            // another key sends it on by linear probing.
            uint32_t spos[U];
            uint64_t sw[U];
            bool winner[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                spos[u] = uint32_t(mix64(key[u] ^ dseed) & sc.mask);
                sw[u] = kEmpty;
                if (claim[u]) sw[u] = atomicCAS(reinterpret_cast<unsigned long long*>(sc.set + spos[u]), kEmpty, key[u]);
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                winner[u] = placed[u];
                if (!claim[u]) continue;
                if (sw[u] == kEmpty) {
                    winner[u] = true;                          // our CAS filled the empty slot
                } else if (K::keyof(sw[u]) != key[u]) {        // another key sits there: probe on
                    uint32_t sat = 0;
                    const uint32_t next = spos[u] + 1 == uint32_t(sc.mask + 1) ? 0u : spos[u] + 1;
                    const int rc = lp_insert<KW>(sc.set, uint32_t(sc.mask + 1), next, key[u], key[u], &sat);
                    winner[u] = rc == 1;
                    spos[u] = sat;
                    if (rc < 0) {                              // more distinct misses than the table holds
                        set_flag(t.ctr, kFlagDropped);
                        atomicAdd(&t.ctr->dropped, 1ull);
                    }
                }
            }
            // The round's winners go to the warp's stage in shared memory,
            // listed with one atomic per flush rather than one per round, so
            // the next round does not wait on a shared counter.  Keys this
            // kernel stored are listed only for a caller that appends the new
            // keys (list_stored); otherwise they are just counted.
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint64_t i = (r * U + u) * stride + tid;
                const bool listed = winner[u] && (list_stored || !placed[u]);
                stored += (placed[u] && !list_stored) ? 1u : 0u;
                const unsigned wm = __ballot_sync(0xFFFFFFFFu, listed);
                if (wm) {
                    if (pend + __popc(wm) > uint32_t(kStage)) flush();
                    if (listed) {
                        StagedWinner& e = stage[pend + __popc(wm & ((1u << lane) - 1))];
                        e.word = K::word(key[u], VALUES ? vals[i] : 0u);
                        e.i = i;
                        e.spos = spos[u];
                        e.start = placed[u] ? kStartPlaced : (HT_CUCKOO_DIRECT || t.chain_h1) ? 0u : start[u];
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
        direct += __shfl_down_sync(0xFFFFFFFFu, direct, o);
        stored += __shfl_down_sync(0xFFFFFFFFu, stored, o);
    }
    unsigned long long* const dst[5] = {&t.ctr->size, &t.ctr->probes, &t.ctr->probe_cas, &t.ctr->probe_misses,
                                        &t.ctr->probe_miss_reads};
    const unsigned long long sums[5] = {stored, probes, direct, misses, miss_reads};
    block_add_counters<5>(dst, sums);
}

// Eviction-chain insert of the winners.  Each thread keeps U chains in
// flight so their exchanges overlap, and a chain that ends (an empty slot,
// or the stash) is replaced at once by the thread's next winner: chain
// lengths vary widely at high load, and refilling keeps every slot of the
// thread busy instead of waiting for the longest chain of a round.  Each
// step reads the next records for all free chain slots together with the
// live chains' exchanges.  A record of a key the probe stored (listed only
// for a caller that collects the new keys) holds no claim and is counted.
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
#pragma unroll
    for (int u = 0; u < kU; ++u) {
        live[u] = false;
        word[u] = 0;
        pos[u] = 0;
        evictions[u] = 0;
    }
    // Bounded: each step takes at least one record or runs at least one
    // exchange; each winner is taken once and its chain ends after at most
    // max_evictions + 1 exchanges.
    for (;;) {
        uint32_t nfree = 0;
#pragma unroll
        for (int u = 0; u < kU; ++u) nfree += live[u] ? 0u : 1u;
        Winner rec[kU];
        bool got[kU];
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            got[j] = uint32_t(j) < nfree && next < count;
            if (got[j]) {
                rec[j] = sc.win[next];
                next += stride;
            }
        }
        uint64_t old[kU];
#pragma unroll
        for (int u = 0; u < kU; ++u)
            if (live[u]) old[u] = atomicExch(reinterpret_cast<unsigned long long*>(t.slots + pos[u]), word[u]);
        bool any = false;
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
            any = true;
        }
        // The records read this step: a key the probe stored is counted; a
        // claimant gives its claim back (the dedup set is left empty for the
        // next batch) and takes a free chain slot (there are at least as
        // many as records read).
#pragma unroll
        for (int j = 0; j < kU; ++j) {
            if (!got[j]) continue;
            if (rec[j].start == kStartPlaced) {
                ++placed;
                continue;
            }
            sc.set[rec[j].spos] = kEmpty;
            bool taken = false;
#pragma unroll
            for (int u = 0; u < kU; ++u)
                if (!live[u] && !taken) {
                    word[u] = rec[j].word;
                    pos[u] = hidx(K::keyof(rec[j].word), t.seed[rec[j].start < t.k ? rec[j].start : 0u], t.nslots);
                    evictions[u] = 0;
                    live[u] = true;
                    taken = true;
                }
            any = true;
        }
        if (!any && next >= count) break;
    }
    for (int o = 16; o; o >>= 1) {
        placed += __shfl_down_sync(0xFFFFFFFFu, placed, o);
        exchanges += __shfl_down_sync(0xFFFFFFFFu, exchanges, o);
    }
    unsigned long long* const dst[2] = {&t.ctr->size, &t.ctr->exchanges};
    const unsigned long long sums[2] = {placed, exchanges};
    block_add_counters<2>(dst, sums);
}

}  // namespace

namespace {
// The current device's L2 size in bytes (queried once per device).
uint64_t l2_bytes() {
    static int cached[64] = {};
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 0;
    if (!cached[dev]) {
        int v = 0;
        cudaDeviceGetAttribute(&v, cudaDevAttrL2CacheSize, dev);
        cached[dev] = v > 0 ? v : -1;
    }
    return cached[dev] > 0 ? uint64_t(cached[dev]) : 0;
}
}  // namespace

cudaError_t cuckoo_probe(int kw, const DevTable& t, const DevScratch& sc, uint32_t parity,
                         const void* keys, const uint32_t* vals, uint64_t n,
                         const unsigned long long* d_n, uint64_t off, uint8_t* is_new, cudaStream_t s,
                         const L2Window& w, bool list_stored) {
    ProfScope ps(kKCuckooProbe, s);
    const bool in_l2 = t.nslots * 8 <= l2_bytes();
#define L(KW, V)                                                                                        \
    {                                                                                                   \
        auto k = t.k > 4 ? cuckoo_probe_kernel<KW, V, false, kMaxCuckooHashes>                          \
                 : in_l2 ? cuckoo_probe_kernel<KW, V, false, 4, kUL2> : cuckoo_probe_kernel<KW, V, false, 4>; \
        return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, sc, parity, keys, vals, n, \
                          d_n, off, is_new, (uint32_t*)nullptr, list_stored);                           \
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
                          (const uint32_t*)nullptr, n, (const unsigned long long*)nullptr, uint64_t(0), found, vals,
                          false);
    }
    auto k = t.k <= 4 ? cuckoo_probe_kernel<64, false, true, 4> : cuckoo_probe_kernel<64, false, true, kMaxCuckooHashes>;
    return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, none, 0u, keys,
                      (const uint32_t*)nullptr, n, (const unsigned long long*)nullptr, uint64_t(0), found, vals,
                      false);
}

}  // namespace ht
