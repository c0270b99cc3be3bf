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
//     slot h_1(k); if the slot held a word k', find a with h_a(k') = slot and
//     move k' to h_{a+1}(k') (Fig. 2: key 18 evicts 26 from its h_2 slot and
//     26 moves to h_3), until an empty slot takes the word or max_evictions
//     is reached; then the stash takes it (Section 4.1: a small stash, and a
//     rebuild with new hash constants when it overflows).
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

template <int KW, bool VALUES, bool LOOKUP>
__global__ void __launch_bounds__(kBlock)
cuckoo_probe_kernel(const DevTable t, const DevScratch sc, uint32_t parity,
                    const void* __restrict__ keys, const uint32_t* __restrict__ vals, uint64_t n,
                    uint8_t* __restrict__ out_flag, uint32_t* __restrict__ out_val) {
    using K = Keys<KW>;
    const uint32_t stash_used = __ldcg(&t.ctr->stash_used);
    const uint32_t ovf_used = __ldcg(&t.ctr->ovf_used);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t rounds = (n + stride - 1) / stride;     // warp-uniform trip count
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x + r * stride;
        const bool active = i < n;
        const uint64_t key = active ? K::load(keys, i) : 0;
        uint32_t flag = 0, value = 0;
        bool winner = false;
        uint64_t word = 0;
        uint32_t spos = 0;
        if (!active) {
        } else if (K::reserved(key)) {
            set_flag(t.ctr, kFlagInvalidKey);
        } else {
            // Section 4.1: a key is found in at most k probes.
            uint64_t w = __ldcg(reinterpret_cast<const unsigned long long*>(
                t.slots + hidx(key, t.seed[0], t.nslots)));
            bool found = K::keyof(w) == key;
            if (!found) {
                uint64_t ws[kMaxCuckooHashes];
#pragma unroll
                for (int a = 1; a < kMaxCuckooHashes; ++a)
                    if (a < int(t.k))
                        ws[a] = __ldcg(reinterpret_cast<const unsigned long long*>(
                            t.slots + hidx(key, t.seed[a], t.nslots)));
#pragma unroll
                for (int a = 1; a < kMaxCuckooHashes; ++a)
                    if (a < int(t.k) && !found && K::keyof(ws[a]) == key) {
                        found = true;
                        w = ws[a];
                    }
            }
            if (!found && (stash_used | ovf_used)) found = find_spill<KW>(t, key, stash_used, ovf_used, &w);
            if (LOOKUP) {
                flag = found;
                value = found ? K::value(w) : 0u;
            } else if (!found) {
                word = K::word(key, VALUES ? vals[i] : 0u);
                const int claim = lp_insert<KW>(sc.set, uint32_t(sc.mask + 1),
                                            mix64(key ^ (t.aux_seed * 3 + 1)) & sc.mask, key, key, &spos);
                winner = claim == 1;
                flag = winner;
            }
        }
        if (active && out_flag) out_flag[i] = uint8_t(flag);
        if (LOOKUP && active && out_val) out_val[i] = value;
        if (!LOOKUP) {
            // Warp-aggregated append of the winners to the insert list.
            const unsigned wm = __ballot_sync(0xFFFFFFFFu, winner);
            if (wm) {
                const int lane = threadIdx.x & 31;
                const int leader = __ffs(wm) - 1;
                unsigned int b = 0;
                if (lane == leader) b = atomicAdd(&t.ctr->winners[parity], unsigned(__popc(wm)));
                b = __shfl_sync(0xFFFFFFFFu, b, leader);
                if (winner) {
                    Winner wn;
                    wn.word = word;
                    wn.spos = spos;
                    wn.pad_ = 0;
                    sc.win[b + __popc(wm & ((1u << lane) - 1))] = wn;
                }
            }
        }
    }
}

template <int KW, bool APPEND>
__global__ void __launch_bounds__(kBlock)
cuckoo_insert_kernel(const DevTable t, const DevScratch sc, uint32_t parity, uint64_t max_winners,
                     typename Keys<KW>::T* __restrict__ new_out, unsigned long long* __restrict__ new_count) {
    using K = Keys<KW>;
    const uint64_t count = min(uint64_t(__ldcg(&t.ctr->winners[parity])), max_winners);
    // The other parity's list was consumed by the previous insert kernel on
    // this stream; reset its counter for the next probe kernel.
    if (blockIdx.x == 0 && threadIdx.x == 0) t.ctr->winners[parity ^ 1u] = 0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    unsigned long long placed = 0;
    const uint64_t i0 = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t rounds = (count + stride - 1) / stride;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = i0 + r * stride;
        const bool active = i < count;
        uint64_t first_key = 0;
        if (active) {
            const Winner wn = sc.win[i];
            sc.set[wn.spos] = kEmpty;          // leave the dedup set empty for the next batch
            uint64_t word = wn.word;
            first_key = K::keyof(word);
            uint64_t key = first_key;
            uint64_t pos = hidx(key, t.seed[0], t.nslots);
            bool done = false;
            for (uint32_t e = 0; e <= t.max_evict; ++e) {
                const uint64_t old = atomicExch(reinterpret_cast<unsigned long long*>(t.slots + pos), word);
                if (K::empty(old)) {
                    done = true;
                    break;
                }
                // Section 4.1: the evicted key k' sat at h_a(k') = pos; it
                // moves on to h_{a+1}(k') (cyclically after h_k).
                word = old;
                key = K::keyof(old);
                uint32_t a = 0;
                for (; a + 1 < t.k; ++a)
                    if (hidx(key, t.seed[a], t.nslots) == pos) break;
                const uint32_t nxt = (a + 1 == t.k) ? 0u : a + 1;
                pos = hidx(key, t.seed[nxt], t.nslots);
            }
            if (done || place_spill<KW>(t, key, word) == 1) ++placed;
        }
        if (APPEND) warp_append<typename K::T>(active, typename K::T(first_key), new_out, new_count);
    }
    for (int o = 16; o; o >>= 1) placed += __shfl_down_sync(0xFFFFFFFFu, placed, o);
    if ((threadIdx.x & 31) == 0 && placed) atomicAdd(&t.ctr->size, placed);
}

}  // namespace

cudaError_t cuckoo_probe(int kw, const DevTable& t, const DevScratch& sc, uint32_t parity,
                         const void* keys, const uint32_t* vals, uint64_t n, uint8_t* is_new,
                         cudaStream_t s) {
    ProfScope ps(kKCuckooProbe, s);
#define L(KW, V)                                                                    \
    {                                                                               \
        auto k = cuckoo_probe_kernel<KW, V, false>;                                 \
        const int grid = launch_blocks((const void*)k, kBlock);                     \
        k<<<grid, kBlock, 0, s>>>(t, sc, parity, keys, vals, n, is_new, nullptr);   \
    }
    if (kw == 32) {
        if (vals) L(32, true) else L(32, false)
    } else {
        L(64, false)
    }
#undef L
    return cudaGetLastError();
}

cudaError_t cuckoo_insert(int kw, const DevTable& t, const DevScratch& sc, uint32_t parity,
                          void* new_out, unsigned long long* new_count, uint64_t max_winners,
                          cudaStream_t s) {
    ProfScope ps(kKCuckooInsert, s);
#define L(KW, A)                                                                               \
    {                                                                                          \
        auto k = cuckoo_insert_kernel<KW, A>;                                                  \
        const int grid = launch_blocks((const void*)k, kBlock);                                \
        k<<<grid, kBlock, 0, s>>>(t, sc, parity, max_winners,                                  \
                                  static_cast<typename Keys<KW>::T*>(new_out), new_count);     \
    }
    if (kw == 32) {
        if (new_out) L(32, true) else L(32, false)
    } else {
        if (new_out) L(64, true) else L(64, false)
    }
#undef L
    return cudaGetLastError();
}

cudaError_t cuckoo_lookup(int kw, const DevTable& t, const void* keys, uint64_t n, uint32_t* vals,
                          uint8_t* found, cudaStream_t s) {
    ProfScope ps(kKCuckooLookup, s);
    DevScratch none{};
    if (kw == 32) {
        auto k = cuckoo_probe_kernel<32, false, true>;
        const int grid = launch_blocks((const void*)k, kBlock);
        k<<<grid, kBlock, 0, s>>>(t, none, 0, keys, nullptr, n, found, vals);
    } else {
        auto k = cuckoo_probe_kernel<64, false, true>;
        const int grid = launch_blocks((const void*)k, kBlock);
        k<<<grid, kBlock, 0, s>>>(t, none, 0, keys, nullptr, n, found, vals);
    }
    return cudaGetLastError();
}

}  // namespace ht
