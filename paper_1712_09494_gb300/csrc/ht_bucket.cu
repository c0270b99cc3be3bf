// GPUexplore-style bucket table (Section 4.2 of the paper).
//
// A key hashes to a bucket of BS 8-byte slots (BS*8 = 64/128/256 bytes,
// aligned so one group's read is a single coalesced request).  A group of G
// lanes reads the bucket, each lane BS/G consecutive slots; ballots give
// every lane the bucket-wide "matches" and "free" masks (Fig. 4, steps 1-2).
// If the key is present the group stops.  Otherwise the group CASes the free
// slots in a fixed order until one CAS succeeds or returns the key itself
// (step 3: another group may take a slot between the read and the CAS).
// When the bucket has no free slot left, the next hash function picks the
// next bucket; after the last one the key goes to the stash.
//
// Exactly-once: a slot never returns to empty and never changes its key, and
// every group claims in the same slot order.  A group that claims slot s saw
// every earlier slot (by load or by a failed CAS) holding another key, so a
// concurrent group with the same key either meets the claimed word first or
// finds the bucket full only after the word was written there.  A key goes
// to bucket f+1 only after bucket f was observed full without it, and
// fullness is permanent, so lookups may stop at the first non-full bucket.
#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

template <int SPL>
__device__ __forceinline__ void load_lane(const uint64_t* p, uint64_t (&w)[SPL]) {
    if constexpr (SPL == 1) {
        w[0] = __ldcg(reinterpret_cast<const unsigned long long*>(p));
    } else {
#pragma unroll
        for (int j = 0; j < SPL; j += 2) {
            ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(p + j));
            w[j] = v.x;
            w[j + 1] = v.y;
        }
    }
}

// Group masks in "claim position" order: position q = j*G + sub names slot
// sub*SPL + j of the bucket, so each ballot contributes one contiguous run
// of G bits and no bit interleaving is needed.
template <int G, int SPL>
__device__ __forceinline__ uint32_t group_mask(const bool (&pred)[SPL], int gbase) {
    constexpr uint32_t kGMask = (G == 32) ? 0xFFFFFFFFu : ((1u << G) - 1u);
    uint32_t m = 0;
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
        const uint32_t b = __ballot_sync(kFull, pred[j]);
        m |= ((b >> gbase) & kGMask) << (j * G);
    }
    return m;
}

enum : int { kDone = 0, kRead = 1, kClaim = 2, kSpill = 3 };

template <int KW, int BS, int G, bool VALUES, bool APPEND>
__global__ void __launch_bounds__(kBlock)
bucket_fop_kernel(const DevTable t, const void* __restrict__ keys, const uint32_t* __restrict__ vals,
                  uint64_t n, uint8_t* __restrict__ is_new, typename Keys<KW>::T* __restrict__ new_out,
                  unsigned long long* __restrict__ new_count) {
    using K = Keys<KW>;
    constexpr int SPL = BS / G;
    constexpr int GPW = 32 / G;
    static_assert(SPL >= 1 && SPL <= 4 && BS % G == 0, "bucket/lane split");
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G, gbase = grp * G;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    unsigned long long stored = 0;

    for (uint64_t base = ((uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += nwarps * 32) {
        uint64_t mykey = 0;
        uint32_t myval = 0;
        const bool mine = base + lane < n;
        if (mine) {
            mykey = K::load(keys, base + lane);
            if (VALUES) myval = vals[base + lane];
        }
        uint32_t my_new = 0;
#pragma unroll 1
        for (int r = 0; r < G; ++r) {
            const int kidx = r * GPW + grp;
            const uint64_t key = __shfl_sync(kFull, mykey, kidx);
            const uint32_t val = VALUES ? __shfl_sync(kFull, myval, kidx) : 0u;
            int state = kDone;
            if (base + kidx < n) {
                if (K::reserved(key)) {
                    if (sub == 0) set_flag(t.ctr, kFlagInvalidKey);
                } else {
                    state = kRead;
                }
            }
            const uint64_t word = K::word(key, val);
            uint32_t f = 0;
            uint64_t b = hidx(key, t.seed[0], t.nbuckets);
            uint32_t free_mask = 0;
            uint32_t res = 0;
            // Bounded: each pass either ends the key, consumes a free slot of
            // the current bucket (<= BS per bucket) or moves to the next hash
            // function (<= k buckets), then the spill path ends it.
            while (__any_sync(kFull, state != kDone)) {
                bool m[SPL], e[SPL];
                if (state == kRead) {
                    uint64_t w[SPL];
                    load_lane<SPL>(t.slots + b * BS + sub * SPL, w);
#pragma unroll
                    for (int j = 0; j < SPL; ++j) {
                        m[j] = K::keyof(w[j]) == key;
                        e[j] = K::empty(w[j]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < SPL; ++j) m[j] = e[j] = false;
                }
                const uint32_t M = group_mask<G, SPL>(m, gbase);
                const uint32_t E = group_mask<G, SPL>(e, gbase);
                if (state == kRead) {
                    if (M) {
                        state = kDone;
                    } else if (E) {
                        state = kClaim;
                        free_mask = E;
                    } else if (++f < t.k) {
                        b = hidx(key, t.seed[f], t.nbuckets);
                    } else {
                        state = kSpill;
                    }
                }
                int owner = lane;
                uint64_t old = 0;
                uint64_t* target = nullptr;
                if (state == kClaim) {
                    const int q = __ffs(free_mask) - 1;
                    owner = gbase + (q % G);
                    target = t.slots + b * BS + (q % G) * SPL + q / G;
                }
                if (lane == owner && target)
                    old = atomicCAS(reinterpret_cast<unsigned long long*>(target), kEmpty, word);
                old = __shfl_sync(kFull, old, owner);
                if (state == kClaim) {
                    if (old == kEmpty) {
                        state = kDone;
                        res = 1;
                    } else if (K::keyof(old) == key) {
                        state = kDone;
                    } else {
                        free_mask &= free_mask - 1;
                        if (!free_mask) {
                            if (++f < t.k) {
                                b = hidx(key, t.seed[f], t.nbuckets);
                                state = kRead;
                            } else {
                                state = kSpill;
                            }
                        }
                    }
                }
                if (state == kSpill) {
                    if (sub == 0) res = place_spill<KW>(t, key, word) == 1 ? 1u : 0u;
                    state = kDone;
                }
            }
            // Key r*GPW+grp's result lives on its group's first lane.
            const uint32_t got = __shfl_sync(kFull, res, (lane % GPW) * G);
            if (lane / GPW == r) my_new = got;
        }
        if (mine && is_new) is_new[base + lane] = uint8_t(my_new);
        if (APPEND) warp_append<typename K::T>(mine && my_new, typename K::T(mykey), new_out, new_count);
        stored += __popc(__ballot_sync(kFull, my_new != 0));
    }
    if ((threadIdx.x & 31) == 0 && stored) atomicAdd(&t.ctr->size, stored);
}

template <int KW, int BS, int G>
__global__ void __launch_bounds__(kBlock)
bucket_lookup_kernel(const DevTable t, const void* __restrict__ keys, uint64_t n,
                     uint32_t* __restrict__ vals, uint8_t* __restrict__ found) {
    using K = Keys<KW>;
    constexpr int SPL = BS / G;
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G, gbase = grp * G;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    const uint32_t stash_used = __ldcg(&t.ctr->stash_used);
    const uint32_t ovf_used = __ldcg(&t.ctr->ovf_used);

    for (uint64_t base = ((uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += nwarps * 32) {
        const bool mine = base + lane < n;
        const uint64_t mykey = mine ? K::load(keys, base + lane) : 0;
        uint32_t my_found = 0, my_val = 0;
#pragma unroll 1
        for (int r = 0; r < G; ++r) {
            const int kidx = r * GPW + grp;
            const uint64_t key = __shfl_sync(kFull, mykey, kidx);
            int state = (base + kidx < n && !K::reserved(key)) ? kRead : kDone;
            if (base + kidx < n && K::reserved(key) && sub == 0) set_flag(t.ctr, kFlagInvalidKey);
            uint32_t f = 0;
            uint64_t b = hidx(key, t.seed[0], t.nbuckets);
            uint32_t res_found = 0, res_val = 0;
            while (__any_sync(kFull, state != kDone)) {
                bool m[SPL], e[SPL];
                uint64_t w[SPL];
                if (state == kRead) {
                    load_lane<SPL>(t.slots + b * BS + sub * SPL, w);
#pragma unroll
                    for (int j = 0; j < SPL; ++j) {
                        m[j] = K::keyof(w[j]) == key;
                        e[j] = K::empty(w[j]);
                    }
                } else {
#pragma unroll
                    for (int j = 0; j < SPL; ++j) {
                        m[j] = e[j] = false;
                        w[j] = 0;
                    }
                }
                const uint32_t M = group_mask<G, SPL>(m, gbase);
                const uint32_t E = group_mask<G, SPL>(e, gbase);
                int owner = lane;
                int q = 0;
                if (state == kRead && M) {
                    q = __ffs(M) - 1;
                    owner = gbase + (q % G);
                }
                uint64_t mw = 0;
#pragma unroll
                for (int j = 0; j < SPL; ++j)
                    if (j == q / G) mw = w[j];
                mw = __shfl_sync(kFull, mw, owner);
                if (state == kRead) {
                    if (M) {
                        res_found = 1;
                        res_val = K::value(mw);
                        state = kDone;
                    } else if (E) {
                        state = kDone;              // a non-full bucket ends the search
                    } else if (++f < t.k) {
                        b = hidx(key, t.seed[f], t.nbuckets);
                    } else {
                        state = kSpill;
                    }
                }
                if (state == kSpill) {
                    if (sub == 0) {
                        uint64_t sw;
                        if (find_spill<KW>(t, key, stash_used, ovf_used, &sw)) {
                            res_found = 1;
                            res_val = K::value(sw);
                        }
                    }
                    state = kDone;
                }
            }
            const int src = (lane % GPW) * G;
            const uint32_t gf = __shfl_sync(kFull, res_found, src);
            const uint32_t gv = __shfl_sync(kFull, res_val, src);
            if (lane / GPW == r) {
                my_found = gf;
                my_val = gv;
            }
        }
        if (mine) {
            if (found) found[base + lane] = uint8_t(my_found);
            if (vals) vals[base + lane] = my_val;
        }
    }
}

template <int KW, int BS, int G>
cudaError_t launch_fop(const DevTable& t, const void* keys, const uint32_t* vals, uint64_t n,
                       uint8_t* is_new, void* new_out, unsigned long long* new_count,
                       cudaStream_t s) {
    using T = typename Keys<KW>::T;
    ProfScope ps(kKBucketFop, s);
    if (vals) {
        auto k = bucket_fop_kernel<KW, BS, G, true, false>;
        const int grid = launch_blocks((const void*)k, kBlock);
        k<<<grid, kBlock, 0, s>>>(t, keys, vals, n, is_new, nullptr, nullptr);
    } else if (new_out) {
        auto k = bucket_fop_kernel<KW, BS, G, false, true>;
        const int grid = launch_blocks((const void*)k, kBlock);
        k<<<grid, kBlock, 0, s>>>(t, keys, nullptr, n, is_new, static_cast<T*>(new_out), new_count);
    } else {
        auto k = bucket_fop_kernel<KW, BS, G, false, false>;
        const int grid = launch_blocks((const void*)k, kBlock);
        k<<<grid, kBlock, 0, s>>>(t, keys, nullptr, n, is_new, nullptr, nullptr);
    }
    return cudaGetLastError();
}

template <int KW, int BS, int G>
cudaError_t launch_lookup(const DevTable& t, const void* keys, uint64_t n, uint32_t* vals,
                          uint8_t* found, cudaStream_t s) {
    ProfScope ps(kKBucketLookup, s);
    auto k = bucket_lookup_kernel<KW, BS, G>;
    const int grid = launch_blocks((const void*)k, kBlock);
    k<<<grid, kBlock, 0, s>>>(t, keys, n, vals, found);
    return cudaGetLastError();
}

// (bucket_slots, lanes) pairs that are instantiated.
#define HT_BUCKET_CONFIGS(X) \
    X(8, 4) X(8, 8) X(16, 4) X(16, 8) X(16, 16) X(32, 8) X(32, 16) X(32, 32)

}  // namespace

cudaError_t bucket_find_or_put(const BucketCfg& c, const DevTable& t, const void* keys,
                               const uint32_t* vals, uint64_t n, uint8_t* is_new, void* new_out,
                               unsigned long long* new_count, cudaStream_t s) {
#define X(BS, G)                                                                          \
    if (c.bucket_slots == BS && c.lanes == G)                                             \
        return c.kw == 32 ? launch_fop<32, BS, G>(t, keys, vals, n, is_new, new_out, new_count, s) \
                          : launch_fop<64, BS, G>(t, keys, vals, n, is_new, new_out, new_count, s);
    HT_BUCKET_CONFIGS(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t bucket_lookup(const BucketCfg& c, const DevTable& t, const void* keys, uint64_t n,
                          uint32_t* vals, uint8_t* found, cudaStream_t s) {
#define X(BS, G)                                                                    \
    if (c.bucket_slots == BS && c.lanes == G)                                       \
        return c.kw == 32 ? launch_lookup<32, BS, G>(t, keys, n, vals, found, s)   \
                          : launch_lookup<64, BS, G>(t, keys, n, vals, found, s);
    HT_BUCKET_CONFIGS(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace ht
