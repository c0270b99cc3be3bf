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
#include <algorithm>

#include "ht_bucket_tile.cuh"

namespace ht {
namespace {

using namespace bucket;

#ifndef HT_BUCKET_MIN_BLOCKS
#define HT_BUCKET_MIN_BLOCKS 3
#endif

// Plain find-or-put over one table.  The next tile's keys are loaded while
// the current tile waits on the table.  (Pipelining tile i's claims with tile
// i+1's bucket reads was measured slower on GB300: the extra live state costs
// occupancy, and occupancy is what hides the table's latency here.)
template <int KW, int BS, int G, bool VALUES, bool APPEND>
__global__ void __launch_bounds__(kBlock, HT_BUCKET_MIN_BLOCKS)
bucket_fop_kernel(const DevTable t, const void* __restrict__ keys, const uint32_t* __restrict__ vals,
                  uint64_t n, const unsigned long long* __restrict__ d_n, uint8_t* __restrict__ is_new,
                  typename Keys<KW>::T* __restrict__ new_out, unsigned long long* __restrict__ new_count,
                  uint64_t new_cap) {
    if (d_n) n = min(n, uint64_t(__ldcg(d_n)));        // batch size produced on the device
    using K = Keys<KW>;
    using T = typename K::T;
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    const uint64_t step = nwarps * 32;
    unsigned long long stored = 0;
    __shared__ T s_new[APPEND ? kBlock / 32 : 1][APPEND ? kStageCap : 1];   // new keys awaiting the append
    WarpStage<T, kStageCap> stage(s_new[APPEND ? (threadIdx.x >> 5) : 0]);
    uint64_t base = ((uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32;
    uint64_t next_key = 0;
    uint32_t next_val = 0;
    if (base + lane < n) {
        next_key = K::load(keys, base + lane);
        if (VALUES) next_val = vals[base + lane];
    }
    for (; base < n; base += step) {
        const bool mine = base + lane < n;
        const uint64_t mykey = next_key;
        const uint32_t myval = next_val;
        if (base + step + lane < n) {
            next_key = K::load(keys, base + step + lane);
            if (VALUES) next_val = vals[base + step + lane];
        }
        const bool myok = mine && !K::reserved(mykey);
        if (mine && !myok) set_flag(t.ctr, kFlagInvalidKey);
        const uint32_t my_new = bucket_tile<KW, BS, G>(t, mykey, myval, myok);
        if (mine && is_new) is_new[base + lane] = uint8_t(my_new);
        if (APPEND) stage.push(mine && my_new, T(mykey), new_out, new_count, new_cap);
        stored += __popc(__ballot_sync(kFull, my_new != 0));
    }
    if (APPEND) stage.flush(new_out, new_count, new_cap);
    if ((threadIdx.x & 31) == 0 && stored) atomicAdd(&t.ctr->size, stored);
}

// Lookup: like find-or-put without claims; a bucket with a free slot ends the
// search (a key only moves on from a full bucket), all k full -> the spill.
// One round at a time: a read-only probe gains more from the occupancy of a
// small register footprint than from reading all rounds up front (measured:
// 24.7 vs 20.1 G lookups/s on 2^27 keys at load 0.8).
template <int KW, int BS, int G>
__global__ void __launch_bounds__(kBlock)
bucket_lookup_kernel(const DevTable t, const void* __restrict__ keys, uint64_t n,
                     uint32_t* __restrict__ vals, uint8_t* __restrict__ found) {
    using K = Keys<KW>;
    constexpr int SPL = BS / G;
    constexpr int GPW = 32 / G;
    constexpr int PF = Prefetch<G, SPL>::kRounds;
    constexpr uint32_t kGMask = (G == 32) ? 0xFFFFFFFFu : ((1u << G) - 1u);
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G, gbase = grp * G;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    const uint32_t stash_used = __ldcg(&t.ctr->stash_used);
    const uint32_t ovf_used = __ldcg(&t.ctr->ovf_used);

    for (uint64_t base = ((uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += nwarps * 32) {
        const bool mine = base + lane < n;
        const uint64_t mykey = mine ? K::load(keys, base + lane) : 0;
        const bool myok = mine && !K::reserved(mykey);
        if (mine && !myok) set_flag(t.ctr, kFlagInvalidKey);
        const uint64_t mybkt = hidx(mykey, t.seed[0], t.nbuckets);
        uint32_t my_found = 0, my_val = 0;
#pragma unroll 1
        for (int r0 = 0; r0 < G; r0 += PF) {
            uint64_t w[PF][SPL];
#pragma unroll
            for (int q = 0; q < PF; ++q) {
                const int kidx = (r0 + q) * GPW + grp;
                const uint64_t b = __shfl_sync(kFull, mybkt, kidx);
                const bool ok = __shfl_sync(kFull, myok, kidx);
                if (ok) {
                    load_lane<SPL>(t.slots + b * BS + sub * SPL, w[q]);
                } else {
#pragma unroll
                    for (int j = 0; j < SPL; ++j) w[q][j] = kEmpty;
                }
            }
#pragma unroll
            for (int q = 0; q < PF; ++q) {
                const int kidx = (r0 + q) * GPW + grp;
                const uint64_t key = __shfl_sync(kFull, mykey, kidx);
                int state = __shfl_sync(kFull, myok, kidx) ? kRead : kDone;
                uint64_t cur[SPL];
#pragma unroll
                for (int j = 0; j < SPL; ++j) cur[j] = w[q][j];
                uint32_t lm, le;
                scan_lane<KW, SPL>(cur, key, lm, le);
                uint32_t f = 0, res_found = 0, res_val = 0;
                while (__any_sync(kFull, state != kDone)) {
                    const uint32_t Mb = __ballot_sync(kFull, state == kRead && lm != 0);
                    const uint32_t M = (Mb >> gbase) & kGMask;
                    const uint32_t E = (__ballot_sync(kFull, state == kRead && le != 0) >> gbase) & kGMask;
                    uint32_t v = 0;
                    if (lm) {
                        const int j = __ffs(lm) - 1;
#pragma unroll
                        for (int jj = 0; jj < SPL; ++jj)
                            if (jj == j) v = K::value(cur[jj]);
                    }
                    const int owner = M ? gbase + __ffs(M) - 1 : lane;
                    v = __shfl_sync(kFull, v, owner);
                    if (state == kRead) {
                        if (M) {
                            res_found = 1;
                            res_val = v;
                            state = kDone;
                        } else if (E) {
                            state = kDone;
                        } else if (++f < t.k) {
                            const uint64_t b = hidx(key, t.seed[f], t.nbuckets);
                            load_lane<SPL>(t.slots + b * BS + sub * SPL, cur);
                            scan_lane<KW, SPL>(cur, key, lm, le);
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
                const int src = ((lane - (r0 + q) * GPW) & (GPW - 1)) * G;
                const uint32_t gf = __shfl_sync(kFull, res_found, src);
                const uint32_t gv = __shfl_sync(kFull, res_val, src);
                if (lane / GPW == r0 + q) {
                    my_found = gf;
                    my_val = gv;
                }
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
                       const unsigned long long* d_n, uint8_t* is_new, void* new_out,
                       unsigned long long* new_count, uint64_t new_cap, cudaStream_t s, const L2Window& w) {
    using T = typename Keys<KW>::T;
    ProfScope ps(kKBucketFop, s);
    if (vals) {
        auto k = bucket_fop_kernel<KW, BS, G, true, false>;
        return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, keys, vals, n, d_n, is_new,
                          (T*)nullptr, (unsigned long long*)nullptr, uint64_t(0));
    } else if (new_out) {
        auto k = bucket_fop_kernel<KW, BS, G, false, true>;
        return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, keys, (const uint32_t*)nullptr, n,
                          d_n, is_new, static_cast<T*>(new_out), new_count, new_cap);
    }
    auto k = bucket_fop_kernel<KW, BS, G, false, false>;
    return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, keys, (const uint32_t*)nullptr, n, d_n,
                      is_new, (T*)nullptr, (unsigned long long*)nullptr, uint64_t(0));
}

template <int KW, int BS, int G>
cudaError_t launch_lookup(const DevTable& t, const void* keys, uint64_t n, uint32_t* vals,
                          uint8_t* found, cudaStream_t s, const L2Window& w) {
    ProfScope ps(kKBucketLookup, s);
    auto k = bucket_lookup_kernel<KW, BS, G>;
    return launch_win(k, launch_blocks((const void*)k, kBlock), kBlock, s, w, t, keys, n, vals, found);
}

// Multi-table find-or-put of one step (the body is shared with the
// persistent kernel, bucket::multi_find_or_put).
template <int BS, int G>
__global__ void __launch_bounds__(kBlock, HT_BUCKET_MIN_BLOCKS)
multi_bucket_fop_kernel(const MultiDev m, uint64_t) {
    __shared__ uint64_t s_new[kBlock / 32][kStageCap];
    __shared__ unsigned int s_first[multi::kExactTileExpl + 1];
    __shared__ unsigned long long s_scan[multi::kAdvShared];
    const multi::TileMap tm = multi::tile_map<kBlock>(m, s_first, s_scan);
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    multi_find_or_put<BS, G>(m, tm, gw, nwarps, s_new[threadIdx.x >> 5]);
}

// One warp per exploration: level 0 is the initial state.
template <int BS, int G>
__global__ void __launch_bounds__(kBlock) multi_bucket_init_kernel(const MultiDev m) {
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    for (uint64_t e = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; e < m.count; e += nwarps) {
        const uint64_t key = m.s0[e];
        const bool ok = lane == 0 && !Keys<64>::reserved(key);
        const DevTable& t = m.tables[e];
        const uint32_t my_new = bucket_tile<64, BS, G>(t, key, 0, ok);
        __syncwarp();
        if (lane == 0) {
            if (ok && my_new) {
                if (m.narrow[e]) static_cast<unsigned int*>(m.states[e])[0] = static_cast<unsigned int>(key);
                else static_cast<unsigned long long*>(m.states[e])[0] = key;
                atomicAdd(&t.ctr->size, 1ull);
            }
            const unsigned long long n0 = (ok && my_new) ? 1 : 0;
            m.total[e] = n0;
            m.lo[e] = 0;
            m.hi[e] = n0;
            m.cur[e] = 0;
            m.take[e] = 0;
            m.gen[e] = 0;
            m.level[e] = 0;
            m.done[e] = n0 ? 0u : 1u;
            if (n0) m.level_sizes[e * m.max_levels] = n0;
        }
    }
}

template <int BS, int G>
cudaError_t launch_multi(const MultiDev& m, uint64_t max_tiles, bool init, cudaStream_t s) {
    if (init) {
        auto k = multi_bucket_init_kernel<BS, G>;
        const int grid = int(std::min<uint64_t>(launch_blocks((const void*)k, kBlock), (m.count + 7) / 8));
        k<<<grid, kBlock, 0, s>>>(m);
    } else {
        ProfScope ps(kKBucketFop, s);
        auto k = multi_bucket_fop_kernel<BS, G>;
        k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(m, max_tiles);
    }
    return cudaGetLastError();
}

// Packed multi-table find-or-put (the serving loop's batches and
// ht_multi_find_or_put): the items' 32-key tiles are numbered across the
// items and each warp takes a contiguous range of them, finds its first
// tile's item once and walks the items in order, keeping the item's
// descriptor in registers and its table's size count until it moves on.
template <int KW, int BS, int G>
__global__ void __launch_bounds__(kBlock, HT_BUCKET_MIN_BLOCKS)
packed_bucket_kernel(const DevTable* __restrict__ tables, const WorkDesc* __restrict__ items, uint32_t nitems,
                     uint64_t ntiles) {
    using K = Keys<KW>;
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    const uint64_t gw = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5;
    const uint64_t per = (ntiles + nwarps - 1) / nwarps;
    const uint64_t t_begin = min(ntiles, gw * per), t_end = min(ntiles, t_begin + per);
    if (t_begin >= t_end) return;
    uint32_t r = 0, b = nitems;                        // largest r with tile_off[r] <= t_begin
    while (b - r > 1) {
        const uint32_t mid = (r + b) / 2;
        if (items[mid].tile_off <= t_begin) r = mid; else b = mid;
    }
    WorkDesc d = items[r];
    uint64_t next_off = r + 1 < nitems ? items[r + 1].tile_off : ~0ull;
    unsigned long long stored = 0;
    for (uint64_t tile = t_begin; tile < t_end; ++tile) {
        if (tile >= next_off) {                        // into a later item
            if (lane == 0 && stored) atomicAdd(&tables[d.table].ctr->size, stored);
            stored = 0;
            do {
                ++r;
                next_off = r + 1 < nitems ? items[r + 1].tile_off : ~0ull;
            } while (tile >= next_off);
            d = items[r];
        }
        const uint64_t i = (tile - d.tile_off) * 32 + lane;
        const bool mine = i < d.n;
        const uint64_t key = mine ? K::load(d.keys, i) : 0;
        const bool ok = mine && !K::reserved(key);
        const DevTable& t = tables[d.table];
        if (mine && !ok) set_flag(t.ctr, kFlagInvalidKey);
        const uint32_t my_new = bucket_tile<KW, BS, G>(t, key, 0, ok);
        if (mine && d.flags) d.flags[i] = uint8_t(my_new);
        stored += __popc(__ballot_sync(kFull, my_new != 0));
    }
    if (lane == 0 && stored) atomicAdd(&tables[d.table].ctr->size, stored);
}

// One BFS level with successor generation and find-or-put fused (the
// GPUexplore way of exploring on the fly, Section 3.2): lane l of a warp
// expands frontier state l of the warp's 32; the warp lays their successors
// out in shared memory (in chunks of kFusedStage) and runs them through the
// bucket claim tile by tile; new states are appended to `out` through the
// warp's stage.  No successor buffer goes through HBM.
constexpr int kFusedBlock = 128;
constexpr int kFusedStage = 512;

template <int KW, int BS, int G>
__global__ void __launch_bounds__(kFusedBlock, HT_BUCKET_MIN_BLOCKS * 2)
bfs_fused_kernel(const PreparedModel* __restrict__ model, const typename Keys<KW>::T* __restrict__ frontier,
                 uint64_t n, const DevTable t, typename Keys<KW>::T* __restrict__ out,
                 unsigned long long* __restrict__ count, uint64_t cap, unsigned long long* __restrict__ gen) {
    using K = Keys<KW>;
    using T = typename K::T;
    __shared__ PreparedModel sm;
    __shared__ uint64_t s_succ[kFusedBlock / 32][kFusedStage];
    __shared__ T s_new[kFusedBlock / 32][kStageCap];
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(model);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sm);
        for (int i = threadIdx.x; i < int(sizeof(PreparedModel) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int warp = threadIdx.x >> 5;
    uint64_t* buf = s_succ[warp];
    WarpStage<T, kStageCap> stage(s_new[warp]);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t rounds = (n + stride - 1) / stride;       // warp-uniform trip count
    unsigned long long made = 0, stored = 0;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = r * stride + uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
        const bool act = i < n;
        const uint64_t st = act ? uint64_t(frontier[i]) : 0;
        const uint32_t cnt = act ? count_successors(sm, st) : 0;
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t tot = __shfl_sync(kFull, incl, 31);
        const uint32_t excl = incl - cnt;
        for (uint32_t chunk = 0; chunk < tot; chunk += kFusedStage) {
            if (act && excl < chunk + kFusedStage && incl > chunk) {
                uint32_t k = excl;
                for_each_successor(sm, st, [&](uint64_t v) {
                    if (k >= chunk && k < chunk + kFusedStage) buf[k - chunk] = v;
                    ++k;
                });
            }
            __syncwarp();
            const uint32_t m = min(uint32_t(kFusedStage), tot - chunk);
            for (uint32_t j0 = 0; j0 < m; j0 += 32) {
                const bool mine = j0 + lane < m;
                const uint64_t key = mine ? buf[j0 + lane] : 0;
                const bool ok = mine && !K::reserved(key);
                if (mine && !ok) set_flag(t.ctr, kFlagInvalidKey);
                const uint32_t my_new = bucket_tile<KW, BS, G>(t, key, 0, ok);
                stage.push(mine && my_new, T(key), out, count, cap);
                stored += __popc(__ballot_sync(kFull, my_new != 0));
            }
            __syncwarp();
        }
        made += cnt;
    }
    stage.flush(out, count, cap);
    for (int o = 16; o; o >>= 1) made += __shfl_down_sync(kFull, made, o);
    if (lane == 0 && stored) atomicAdd(&t.ctr->size, stored);
    if (lane == 0 && made) atomicAdd(gen, made);
}

// (bucket_slots, lanes) pairs that are instantiated.
#define HT_BUCKET_CONFIGS(X) \
    X(8, 2) X(8, 4) X(8, 8) X(16, 2) X(16, 4) X(16, 8) X(16, 16) X(32, 4) X(32, 8) X(32, 16) X(32, 32)

}  // namespace

cudaError_t bucket_find_or_put(const BucketCfg& c, const DevTable& t, const void* keys,
                               const uint32_t* vals, uint64_t n, const unsigned long long* d_n,
                               uint8_t* is_new, void* new_out, unsigned long long* new_count,
                               uint64_t new_cap, cudaStream_t s, const L2Window& w) {
#define X(BS, G)                                                                                  \
    if (c.bucket_slots == BS && c.lanes == G)                                                     \
        return c.kw == 32 ? launch_fop<32, BS, G>(t, keys, vals, n, d_n, is_new, new_out, new_count, new_cap, s, w) \
                          : launch_fop<64, BS, G>(t, keys, vals, n, d_n, is_new, new_out, new_count, new_cap, s, w);
    HT_BUCKET_CONFIGS(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t multi_bucket_find_or_put(const BucketCfg& c, const MultiDev& m, uint64_t max_tiles, cudaStream_t s) {
#define X(BS, G)                                                                       \
    if (c.bucket_slots == BS && c.lanes == G)                                          \
        return launch_multi<BS, G>(m, max_tiles, false, s);
    HT_BUCKET_CONFIGS(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t multi_bucket_init(const BucketCfg& c, const MultiDev& m, cudaStream_t s) {
#define X(BS, G)                                                                       \
    if (c.bucket_slots == BS && c.lanes == G)                                          \
        return launch_multi<BS, G>(m, 0, true, s);
    HT_BUCKET_CONFIGS(X)
#undef X
    return cudaErrorInvalidValue;
}

cudaError_t packed_bucket_find_or_put(const BucketCfg& c, const DevTable* tables, const WorkDesc* items,
                                      uint32_t nitems, uint64_t ntiles, cudaStream_t s) {
    if (!nitems || !ntiles) return cudaSuccess;
    ProfScope ps(kKBucketFop, s);
#define L(KW, BS, G)                                                                                      \
    {                                                                                                     \
        auto k = packed_bucket_kernel<KW, BS, G>;                                                         \
        const int grid = int(std::min<uint64_t>(launch_blocks((const void*)k, kBlock), (ntiles + 7) / 8)); \
        k<<<grid, kBlock, 0, s>>>(tables, items, nitems, ntiles);                                         \
        return cudaGetLastError();                                                                        \
    }
#define X(BS, G)                                                                                          \
    if (c.bucket_slots == BS && c.lanes == G) {                                                           \
        if (c.kw == 32) L(32, BS, G)                                                                      \
        L(64, BS, G)                                                                                      \
    }
    HT_BUCKET_CONFIGS(X)
#undef X
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t bfs_fused_level(const BucketCfg& c, const PreparedModel* model, const void* frontier, uint64_t n,
                            const DevTable& t, void* out, unsigned long long* count, uint64_t cap,
                            unsigned long long* gen, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ProfScope ps(kKBucketFop, s);
#define L(KW, BS, G)                                                                                     \
    {                                                                                                    \
        using T = typename Keys<KW>::T;                                                                  \
        auto k = bfs_fused_kernel<KW, BS, G>;                                                            \
        k<<<launch_blocks((const void*)k, kFusedBlock), kFusedBlock, 0, s>>>(                            \
            model, static_cast<const T*>(frontier), n, t, static_cast<T*>(out), count, cap, gen);        \
        return cudaGetLastError();                                                                       \
    }
#define X(BS, G)                                                                                         \
    if (c.bucket_slots == BS && c.lanes == G) {                                                          \
        if (c.kw == 32) L(32, BS, G)                                                                     \
        L(64, BS, G)                                                                                     \
    }
    HT_BUCKET_CONFIGS(X)
#undef X
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t bucket_lookup(const BucketCfg& c, const DevTable& t, const void* keys, uint64_t n,
                          uint32_t* vals, uint8_t* found, cudaStream_t s, const L2Window& w) {
#define X(BS, G)                                                                    \
    if (c.bucket_slots == BS && c.lanes == G)                                       \
        return c.kw == 32 ? launch_lookup<32, BS, G>(t, keys, n, vals, found, s, w)   \
                          : launch_lookup<64, BS, G>(t, keys, n, vals, found, s, w);
    HT_BUCKET_CONFIGS(X)
#undef X
    return cudaErrorInvalidValue;
}

}  // namespace ht
