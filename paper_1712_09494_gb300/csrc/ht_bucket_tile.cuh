// Warp-cooperative bucket probe and claim of the GPUexplore-style table
// (Section 4.2 of the paper), shared by the kernels that find-or-put tiles
// of 32 keys: the single-table, multi-table, packed and persistent kernels.
// The protocol and its exactly-once argument are described at the top of
// ht_bucket.cu.
#pragma once

#include "ht_multi_dev.cuh"

namespace ht {
namespace bucket {

constexpr unsigned kFull = 0xFFFFFFFFu;

// One lane's share of a bucket: SPL consecutive slots, read through L2
// (the table is written by atomics, so L1 copies would be stale).  Shares of
// 32 bytes or more use 256-bit loads.
template <int SPL>
__device__ __forceinline__ void load_lane(const uint64_t* p, uint64_t (&w)[SPL]) {
    if constexpr (SPL == 1) {
        w[0] = __ldcg(reinterpret_cast<const unsigned long long*>(p));
    } else if constexpr (SPL == 2) {
        const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(p));
        w[0] = v.x;
        w[1] = v.y;
    } else {
#pragma unroll
        for (int j = 0; j < SPL; j += 4) {
            unsigned long long a, b, c, d;
            asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];"
                         : "=l"(a), "=l"(b), "=l"(c), "=l"(d)
                         : "l"(p + j));
            w[j] = a;
            w[j + 1] = b;
            w[j + 2] = c;
            w[j + 3] = d;
        }
    }
}

enum : int { kDone = 0, kRead = 1, kSpill = 3 };

// Per-lane view of its SPL slots: which hold the key, which are free.
template <int KW, int SPL>
__device__ __forceinline__ void scan_lane(const uint64_t (&w)[SPL], uint64_t key, uint32_t& m, uint32_t& e) {
    using K = Keys<KW>;
    m = 0;
    e = 0;
#pragma unroll
    for (int j = 0; j < SPL; ++j) {
        m |= uint32_t(K::keyof(w[j]) == key) << j;
        e |= uint32_t(K::empty(w[j])) << j;
    }
}

// Rounds whose first bucket reads are issued together: up to 128 bytes of
// slot words per lane in flight.
template <int G, int SPL>
struct Prefetch {
    static constexpr int kCap = (16 / SPL) < 8 ? (16 / SPL) : 8;   // <= 128 B of words per lane
    static constexpr int kRounds = kCap < G ? kCap : G;
};

// The general claim loop of one round, for the rare keys whose first claim
// lost or whose first bucket was full.  `le` is this lane's view of its free
// slots in bucket b (no match was seen there).  Returns the group's result
// (1 = stored) on every lane of the group.
template <int KW, int BS, int G>
__device__ __noinline__ uint32_t claim_slow(const DevTable t, bool active, uint64_t key, uint64_t word,
                                            uint64_t b, uint32_t le, int sub, int gbase, int lane) {
    using K = Keys<KW>;
    constexpr int SPL = BS / G;
    constexpr uint32_t kGMask = (G == 32) ? 0xFFFFFFFFu : ((1u << G) - 1u);
    int state = active ? kRead : kDone;
    uint32_t lm = 0, f = 0, res = 0;
    // Bounded: every pass ends the key, takes one free slot out of the
    // group's view (<= BS per bucket) or moves to the next of k buckets;
    // after the last one the spill path ends it.
    while (__any_sync(kFull, state != kDone)) {
        const uint32_t M = (__ballot_sync(kFull, state == kRead && lm != 0) >> gbase) & kGMask;
        const uint32_t E = (__ballot_sync(kFull, state == kRead && le != 0) >> gbase) & kGMask;
        int owner = -1;
        if (state == kRead) {
            if (M) {
                state = kDone;
            } else if (E) {
                owner = gbase + __ffs(E) - 1;
            } else if (++f < t.k) {
                b = hidx(key, t.seed[f], t.nbuckets);
                uint64_t nw[SPL];
                load_lane<SPL>(t.slots + b * BS + sub * SPL, nw);
                scan_lane<KW, SPL>(nw, key, lm, le);
            } else {
                state = kSpill;
            }
        }
        uint32_t code = 0;
        if (lane == owner) {
            const int j = __ffs(le) - 1;
            const uint64_t old =
                atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + b * BS + sub * SPL + j), kEmpty, word);
            code = old == kEmpty ? 0u : (K::keyof(old) == key ? 1u : 2u);
            le &= ~(1u << j);
        }
        code = __shfl_sync(kFull, code, owner >= 0 ? owner : lane);
        if (owner >= 0 && code != 2u) {
            state = kDone;
            res = code == 0u;
        }
        if (state == kSpill) {
            if (sub == 0) res = place_spill<KW>(t, key, word) == 1 ? 1u : 0u;
            state = kDone;
        }
    }
    return __shfl_sync(kFull, res, gbase);
}

// find-or-put / insert.  A warp takes 32 keys; lane l hashes key l once.  In
// round r, group g (G lanes) serves key r*(32/G)+g.  The first bucket of
// every round is read up front (chunk_read); the rounds' first claims are
// then decided from those reads and all their CASes issued together
// (chunk_claim); the CAS results are read and the rare leftovers finished
// (chunk_resolve).  Claims go in slot-index order: the lowest lane of the
// group holding a free slot (in the group's view) CASes its lowest free
// slot; a failed CAS marks that slot taken and claim_slow tries the next one.

// State of rounds [r0, r0 + R) of one tile between its phases: the claim
// bookkeeping (TileClaims) and, when read into registers, the first bucket
// of each round (TileWords).
template <int KW, int BS, int G, int R>
struct TileClaims {
    static constexpr int SPL = BS / G;
    uint64_t old[R];          // first CAS result (owner lanes)
    uint64_t owner_pack;      // 5 bits per round: claiming lane within the group
    uint32_t le_pack;         // SPL bits per round: free slots in this lane's share
    uint32_t claim, slow;     // per round: first claim issued / needs claim_slow
};

template <int KW, int BS, int G>
struct TileWords {
    static constexpr int SPL = BS / G;
    static constexpr int PF = Prefetch<G, SPL>::kRounds;
    uint64_t w[PF][SPL];      // first bucket of each round, this lane's share
};

// The key of lane l (`mykey`, `myok`) is served in round l / GPW by group l % GPW.
template <int KW, int BS, int G>
__device__ __forceinline__ void chunk_read(const DevTable& t, TileWords<KW, BS, G>& c, int r0, uint64_t mybkt,
                                           bool myok) {
    using C = TileWords<KW, BS, G>;
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G;
#pragma unroll
    for (int q = 0; q < C::PF; ++q) {
        const int kidx = (r0 + q) * GPW + grp;
        const uint64_t b = __shfl_sync(kFull, mybkt, kidx);
        if (__shfl_sync(kFull, myok, kidx)) {
            load_lane<C::SPL>(t.slots + b * BS + sub * C::SPL, c.w[q]);
        } else {
#pragma unroll
            for (int j = 0; j < C::SPL; ++j) c.w[q][j] = kEmpty;
        }
    }
}

// Decides rounds r0..r0+R-1 from their first buckets (fetch(q, w) supplies
// this lane's share of round r0+q's bucket) and issues their first CASes.
template <int KW, int BS, int G, int R, class Fetch>
__device__ __forceinline__ void chunk_claim(const DevTable& t, TileClaims<KW, BS, G, R>& c, int r0, uint64_t mykey,
                                            uint64_t mybkt, uint64_t myword, bool myok, Fetch&& fetch) {
    using C = TileClaims<KW, BS, G, R>;
    constexpr int GPW = 32 / G;
    constexpr uint32_t kGMask = (G == 32) ? 0xFFFFFFFFu : ((1u << G) - 1u);
    constexpr uint32_t kLMask = (1u << C::SPL) - 1u;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G, gbase = grp * G;
    c.le_pack = c.claim = c.slow = 0;
    c.owner_pack = 0;
    // Decide each round from its read: found, claim, or slow path.
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int kidx = (r0 + q) * GPW + grp;
        const uint64_t key = __shfl_sync(kFull, mykey, kidx);
        const bool ok = __shfl_sync(kFull, myok, kidx);
        uint64_t w[C::SPL];
        fetch(q, w);
        uint32_t lm, le;
        scan_lane<KW, C::SPL>(w, key, lm, le);
        const uint32_t M = (__ballot_sync(kFull, ok && lm != 0) >> gbase) & kGMask;
        const uint32_t E = (__ballot_sync(kFull, ok && le != 0) >> gbase) & kGMask;
        c.le_pack |= le << (q * C::SPL);
        if (ok && !M) {
            if (E) {
                c.claim |= 1u << q;
                c.owner_pack |= uint64_t(__ffs(E) - 1) << (5 * q);
            } else {
                c.slow |= 1u << q;
            }
        }
    }
    // Issue every round's first CAS; the results are read in chunk_resolve.
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int kidx = (r0 + q) * GPW + grp;
        const uint64_t b = __shfl_sync(kFull, mybkt, kidx);
        const uint64_t word = __shfl_sync(kFull, myword, kidx);
        c.old[q] = kEmpty;
        if (((c.claim >> q) & 1u) && sub == int((c.owner_pack >> (5 * q)) & 31u)) {
            const int j = __ffs((c.le_pack >> (q * C::SPL)) & kLMask) - 1;
            c.old[q] = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + b * BS + sub * C::SPL + j),
                                 kEmpty, word);
            c.le_pack &= ~(1u << (q * C::SPL + j));
        }
    }
}

// Returns bit q set (group-uniform) when the group's key of round r0 + q was stored.
template <int KW, int BS, int G, int R>
__device__ __forceinline__ uint32_t chunk_resolve(const DevTable& t, TileClaims<KW, BS, G, R>& c, int r0,
                                                  uint64_t mykey, uint64_t mybkt, uint64_t myword) {
    using K = Keys<KW>;
    using C = TileClaims<KW, BS, G, R>;
    constexpr int GPW = 32 / G;
    constexpr uint32_t kLMask = (1u << C::SPL) - 1u;
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G, gbase = grp * G;
    uint32_t res = 0;
#pragma unroll
    for (int q = 0; q < R; ++q) {
        const int kidx = (r0 + q) * GPW + grp;
        const uint64_t key = __shfl_sync(kFull, mykey, kidx);
        const uint32_t code = c.old[q] == kEmpty ? 0u : (K::keyof(c.old[q]) == key ? 1u : 2u);
        const int src = gbase + int((c.owner_pack >> (5 * q)) & 31u);
        const uint32_t v = __shfl_sync(kFull, code, src);
        if ((c.claim >> q) & 1u) {
            if (v == 0u) res |= 1u << q;
            else if (v == 2u) c.slow |= 1u << q;
        }
    }
    // Rare: claims that lost to another key, and full first buckets.
    if (__any_sync(kFull, c.slow != 0)) {
#pragma unroll 1
        for (int q = 0; q < R; ++q) {
            if (!__any_sync(kFull, (c.slow >> q) & 1u)) continue;
            const int kidx = (r0 + q) * GPW + grp;
            const uint64_t key = __shfl_sync(kFull, mykey, kidx);
            const uint64_t word = __shfl_sync(kFull, myword, kidx);
            const uint64_t b = __shfl_sync(kFull, mybkt, kidx);
            const uint32_t r = claim_slow<KW, BS, G>(t, (c.slow >> q) & 1u, key, word, b,
                                                     (c.le_pack >> (q * C::SPL)) & kLMask, sub, gbase, lane);
            if (r) res |= 1u << q;
        }
    }
    return res;
}

// Lane l's key was served by group l % GPW in round l / GPW.
template <int G>
__device__ __forceinline__ uint32_t my_result(uint32_t res_all) {
    constexpr int GPW = 32 / G;
    const int lane = threadIdx.x & 31;
    return (__shfl_sync(kFull, res_all, (lane % GPW) * G) >> (lane / GPW)) & 1u;
}

// One warp serves one tile of up to 32 keys: lane l holds key l (myok false
// on lanes without a valid key).  Returns 1 on the lanes whose key this call
// stored.  Used by the multi-table BFS step and the serving kernel, which
// pass a different table per tile.
template <int KW, int BS, int G>
__device__ __forceinline__ uint32_t bucket_tile(const DevTable& t, uint64_t mykey, uint32_t myval, bool myok) {
    using K = Keys<KW>;
    using W = TileWords<KW, BS, G>;
    constexpr int PF = W::PF;
    static_assert(W::SPL >= 1 && W::SPL <= 8 && BS % G == 0 && G % PF == 0 && PF * W::SPL <= 32,
                  "bucket/lane split");
    const uint64_t mybkt = hidx(mykey, t.seed[0], t.nbuckets);
    const uint64_t myword = K::word(mykey, myval);
    uint32_t res_all = 0;            // bit r: the group's key of round r was stored
#pragma unroll 1
    for (int r0 = 0; r0 < G; r0 += PF) {
        W words;
        TileClaims<KW, BS, G, PF> c;
        chunk_read<KW, BS, G>(t, words, r0, mybkt, myok);
        chunk_claim<KW, BS, G, PF>(t, c, r0, mykey, mybkt, myword, myok, [&](int q, uint64_t (&w)[W::SPL]) {
#pragma unroll
            for (int j = 0; j < W::SPL; ++j) w[j] = words.w[q][j];
        });
        res_all |= chunk_resolve<KW, BS, G, PF>(t, c, r0, mykey, mybkt, myword) << r0;
    }
    return my_result<G>(res_all);
}

// Multi-table find-or-put of warps [gw] of [nwarps]: the step's tiles (the
// TileMap numbering of each exploration's successors) are cut into equal
// contiguous ranges, one per warp, so a warp finds its first tile's
// exploration once and then walks on in order with that exploration's
// descriptor in registers; each tile runs against exploration e's table
// (addressed as a 64-bit key table, which a 32-bit set table's words also
// are) and its new states are appended to e's states.
template <int BS, int G>
__device__ void multi_find_or_put(const MultiDev& m, const multi::TileMap& tm, uint64_t gw, uint64_t nwarps,
                                  uint64_t* stage_buf) {
    using K = Keys<64>;
    const uint64_t tiles = tm.total(m);
    const int lane = threadIdx.x & 31;
    const uint64_t per = (tiles + nwarps - 1) / nwarps;
    const uint64_t t_begin = min(tiles, gw * per), t_end = min(tiles, t_begin + per);
    if (t_begin >= t_end) return;
    // New states are staged per warp and appended, with the table's size, in
    // one atomic each when the warp moves to another exploration or the stage
    // is full: the large explorations' counters are shared by many warps.
    multi::StateStage<kStageCap> stage(stage_buf);
    multi::TileCursor cur;
    cur.start(m, tm, t_begin);
    uint32_t e = cur.e;
    uint64_t cnt = multi::step_count(m, e);
    unsigned long long stored = 0;
    auto settle = [&]() {
        stage.flush(m, e);
        if (lane == 0 && stored) atomicAdd(&m.tables[e].ctr->size, stored);
        stored = 0;
    };
    // The next tile's keys are loaded while this one is claimed.  Lanes past
    // an exploration's count read unused words of its segment.
    uint64_t next_key = __ldcg(reinterpret_cast<const unsigned long long*>(m.succ + cur.key_index(m, t_begin, lane)));
    for (uint64_t tile = t_begin; tile < t_end; ++tile) {
        const uint64_t cur_key = next_key;
        if (tile >= cur.b1) {                          // into a later exploration's tiles
            settle();
            cur.seek(m, tm, tile);
            e = cur.e;
            cnt = multi::step_count(m, e);
        }
        const uint64_t i = 32 * (tile - cur.b0) + lane;
        if (tile + 1 < t_end) {
            multi::TileCursor nx = cur;
            nx.seek(m, tm, tile + 1);
            next_key = __ldcg(reinterpret_cast<const unsigned long long*>(m.succ + nx.key_index(m, tile + 1, lane)));
        }
        const bool mine = i < cnt;
        if (!__any_sync(kFull, mine)) continue;
        const uint64_t key = mine ? cur_key : 0;
        const bool ok = mine && !K::reserved(key);
        const uint32_t my_new = bucket_tile<64, BS, G>(m.tables[e], key, 0, ok);
        stage.push(mine && my_new, key, m, e);
        stored += __popc(__ballot_sync(kFull, my_new != 0));
    }
    settle();
}

}  // namespace bucket
}  // namespace ht
