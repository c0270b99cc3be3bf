// Device bodies of one step of the batched exploration (many independent BFS
// runs advanced together), shared by the per-step kernels (ht_multi.cu,
// ht_bfs.cu) and the persistent kernel (ht_persist.cu).
//
// Each exploration e owns a table, a states array (all its states in level
// order; level d is [lo, hi) while it is expanded) and a cursor `cur` into
// the current level.  A step is: advance (move every cursor past the states
// expanded last step, open the next level when one is done, and share the
// successor buffer among the explorations with work), successors (each
// expanded state's successors into its exploration's segment of the
// buffer), and find-or-put of every segment against its own table, new
// states appended to the exploration's states (Section 3.2: the open set).
#pragma once

#include "ht_internal.cuh"

namespace ht {
namespace multi {

// Block-wide sum of one value per thread (NT threads, a multiple of 32).
template <int NT>
__device__ __forceinline__ unsigned long long block_sum(unsigned long long v, unsigned long long* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    if (warp == 0) {
        unsigned long long t = lane < (NT / 32) ? sh[lane] : 0;
        for (int o = 16; o; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// Block-wide exclusive scan of one value per thread.
template <int NT>
__device__ __forceinline__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    unsigned long long incl = v;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned long long x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o) incl += x;
    }
    __syncthreads();
    if (lane == 31) sh[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        const unsigned long long w = lane < (NT / 32) ? sh[lane] : 0;
        unsigned long long wi = w;
        for (int o = 1; o < 32; o <<= 1) {
            const unsigned long long x = __shfl_up_sync(0xFFFFFFFFu, wi, o);
            if (lane >= o) wi += x;
        }
        sh[lane] = wi - w;
    }
    __syncthreads();
    return sh[warp] + incl - v;
}

constexpr int kAdvShared = 40;   // words of shared scratch advance() needs

// The advance of one step, run by one block of NT threads.  Shares `budget`
// successors among the explorations in proportion to their remaining work
// (each gets at least one state), capped per exploration by take_cap when
// given; lays the segments out at multiples of 32 so every 32-key tile
// belongs to one exploration.
template <int NT>
__device__ inline void advance(const MultiDev& m, uint64_t budget, unsigned long long* sh) {
    const uint32_t per = (m.count + NT - 1) / NT;
    const uint32_t e0 = min(m.count, threadIdx.x * per), e1 = min(m.count, e0 + per);
    unsigned long long want = 0, act = 0;
    // The per-exploration state may have been written by other blocks (the
    // persistent kernel's initial placement), so it is read through L2.
    for (uint32_t e = e0; e < e1; ++e) {
        if (__ldcg(m.done + e)) {
            m.take[e] = 0;
            continue;
        }
        const unsigned long long cur = __ldcg(m.cur + e) + __ldcg(m.take + e);
        unsigned long long hi = __ldcg(m.hi + e);
        m.cur[e] = cur;
        m.take[e] = 0;
        if (cur >= hi) {                               // the level is fully expanded
            const unsigned long long nh = __ldcg(m.total + e);
            if (nh > m.states_cap[e]) {
                m.done[e] = 2;                         // states array full
            } else if (nh == hi) {
                m.done[e] = 1;                         // no new states: finished
            } else if (__ldcg(m.level + e) + 1 >= m.max_levels) {
                m.done[e] = 2;
            } else {
                const unsigned int lvl = __ldcg(m.level + e) + 1;
                m.level[e] = lvl;
                m.level_sizes[uint64_t(e) * m.max_levels + lvl] = nh - hi;
                m.lo[e] = hi;
                m.hi[e] = nh;
                hi = nh;
            }
        }
        if (!m.done[e]) {
            want += (hi - cur) * m.msucc[e];
            ++act;
        }
    }
    const unsigned long long total_want = block_sum<NT>(want, sh);
    const unsigned long long total_act = block_sum<NT>(act, sh);
    const double scale = total_want <= budget ? 1.0 : double(budget) / double(total_want);
    unsigned long long my_take = 0, my_seg = 0;
    for (uint32_t e = e0; e < e1; ++e) {
        if (__ldcg(m.done + e)) continue;
        const unsigned long long rem = __ldcg(m.hi + e) - __ldcg(m.cur + e);
        unsigned long long tk = scale >= 1.0 ? rem : (unsigned long long)(double(rem) * scale);
        if (m.take_cap && m.take_cap[e]) tk = min(tk, (unsigned long long)m.take_cap[e]);
        tk = max(1ull, min(tk, rem));
        m.take[e] = tk;
        my_take += tk;
        my_seg += (tk * m.msucc[e] + 31) / 32 * 32;
    }
    unsigned long long w_off = block_excl_scan<NT>(my_take, sh);
    unsigned long long s_off = block_excl_scan<NT>(my_seg, sh);
    for (uint32_t e = e0; e < e1; ++e) {
        m.work_off[e] = w_off;
        m.seg_off[e] = s_off;
        m.seg_cnt[e] = 0;
        w_off += m.take[e];
        s_off += (m.take[e] * m.msucc[e] + 31) / 32 * 32;
    }
    if (threadIdx.x == NT - 1) {
        *m.work_total = w_off;
        *m.tiles_total = s_off / 32;
        *m.active = unsigned(total_act);
        if (m.win_count) *m.win_count = 0;
    }
}

// State idx of exploration e, whatever its width (read through L2: the
// states may have been appended by other blocks of the same launch).
__device__ __forceinline__ uint64_t state_at(const MultiDev& m, uint32_t e, uint64_t idx) {
    return m.narrow[e] ? uint64_t(__ldcg(static_cast<const unsigned int*>(m.states[e]) + idx))
                       : uint64_t(__ldcg(static_cast<const unsigned long long*>(m.states[e]) + idx));
}

// New states of one warp staged in shared memory (CAP per warp) and appended
// to their exploration's states array with one atomic on its count per
// flush (the large explorations' counters are shared by many warps).  Every
// lane calls push / flush together; entries past states_cap[e] are not
// written (the count still counts them, which ends the exploration).
template <int CAP>
struct StateStage {
    uint64_t* buf;
    uint32_t pend;
    __device__ __forceinline__ explicit StateStage(uint64_t* b) : buf(b), pend(0) {}
    __device__ __forceinline__ void flush(const MultiDev& m, uint32_t e) {
        __syncwarp();
        if (pend) {
            const int lane = threadIdx.x & 31;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(m.total + e, (unsigned long long)pend);
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            const uint64_t cap = m.states_cap[e];
            if (m.narrow[e]) {
                unsigned int* out = static_cast<unsigned int*>(m.states[e]);
                for (uint32_t j = lane; j < pend; j += 32)
                    if (base + j < cap) out[base + j] = static_cast<unsigned int>(buf[j]);
            } else {
                unsigned long long* out = static_cast<unsigned long long*>(m.states[e]);
                for (uint32_t j = lane; j < pend; j += 32)
                    if (base + j < cap) out[base + j] = buf[j];
            }
        }
        __syncwarp();
        pend = 0;
    }
    __device__ __forceinline__ void push(bool pred, uint64_t v, const MultiDev& m, uint32_t e) {
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
        const uint32_t c = __popc(mask);
        if (pend + c > uint32_t(CAP)) flush(m, e);
        const int lane = threadIdx.x & 31;
        if (pred) buf[pend + __popc(mask & ((1u << lane) - 1))] = v;
        pend += c;
    }
};

// Successors of the step's expanded states: they form one index space
// [0, work_total); index v belongs to the largest e with work_off[e] <= v
// (binary search) and its successors go to e's segment of the buffer.
// Threads [gtid] of [nthreads] stride the space in warp-uniform rounds.
__device__ inline void successors(const MultiDev& m, uint64_t max_work, uint64_t gtid, uint64_t nthreads) {
    const uint64_t work = min(uint64_t(__ldcg(m.work_total)), max_work);
    const uint64_t rounds = (work + nthreads - 1) / nthreads;       // warp-uniform trip count
    const int lane = threadIdx.x & 31;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t v = r * nthreads + gtid;
        const bool act = v < work;
        uint32_t e = 0;
        uint32_t cnt = 0;
        uint64_t s = 0;
        if (act) {
            uint32_t a = 0, b = m.count;               // largest e with work_off[e] <= v
            while (b - a > 1) {
                const uint32_t mid = (a + b) / 2;
                if (__ldcg(m.work_off + mid) <= v) a = mid; else b = mid;
            }
            e = a;
            const uint64_t idx = __ldcg(m.cur + e) + (v - __ldcg(m.work_off + e));
            s = state_at(m, e, idx);
            cnt = count_successors(m.models[e], s);
        }
        // Consecutive lanes hold consecutive v, so lanes of one exploration
        // form a contiguous run; the run's first lane reserves for the run.
        const unsigned peers = __match_any_sync(0xFFFFFFFFu, act ? e : 0xFFFFFFFFu);
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t x = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += x;
        }
        const int first = __ffs(peers) - 1;
        const int last = 31 - __clz(peers);
        const uint32_t before = __shfl_sync(0xFFFFFFFFu, incl - cnt, first);
        const uint32_t run = __shfl_sync(0xFFFFFFFFu, incl, last) - before;
        unsigned long long base = 0;
        if (act && lane == first && run) {
            base = atomicAdd(m.seg_cnt + e, (unsigned long long)run);
            atomicAdd(m.gen + e, (unsigned long long)run);
        }
        base = __shfl_sync(0xFFFFFFFFu, base, first);
        if (!act || !cnt) continue;
        uint64_t pos = __ldcg(m.seg_off + e) + base + (incl - cnt - before);
        const uint64_t end = __ldcg(m.seg_off + e) + __ldcg(m.take + e) * __ldcg(m.msucc + e);
        for_each_successor(m.models[e], s, [&](uint64_t x) {
            if (pos < end && pos < m.succ_cap) m.succ[pos] = x;
            ++pos;
        });
    }
}

// The step's find-or-put work as 32-key tiles.  Exploration e's successors
// of this step are succ[seg_off[e] .. seg_off[e] + cnt(e)), cnt(e) =
// min(seg_cnt[e], take[e] * msucc[e]).  Its segment was laid out for the
// upper bound take[e] * msucc[e] (about twice the successors a state has on
// average), so the tiles are numbered over the successors actually made:
// e owns tiles [first[e], first[e + 1]) with first[e] the prefix of
// ceil(cnt / 32) -- computed by every block into shared memory when the
// group has at most kExactTileExpl explorations (each warp then gets an
// equal share of real tiles), else taken from the upper-bound layout
// (first[e] = seg_off[e] / 32, empty tiles skipped).
constexpr uint32_t kExactTileExpl = 4096;

struct TileMap {
    const unsigned int* first;        // [count + 1] prefix in shared memory, or nullptr
    __device__ __forceinline__ uint64_t begin(const MultiDev& m, uint32_t e) const {
        if (first) return first[e];
        return e < m.count ? __ldcg(m.seg_off + e) / 32 : ~0ull / 64;
    }
    __device__ __forceinline__ uint64_t total(const MultiDev& m) const {
        return first ? first[m.count] : uint64_t(__ldcg(m.tiles_total));
    }
    // The exploration owning tile t: the largest e with begin(e) <= t.
    __device__ __forceinline__ uint32_t owner(const MultiDev& m, uint64_t t) const {
        uint32_t e = 0, b = m.count;
        while (b - e > 1) {
            const uint32_t mid = (e + b) / 2;
            if (begin(m, mid) <= t) e = mid; else b = mid;
        }
        return e;
    }
};

// A warp's position in the tile space: exploration e owns [b0, b1).
struct TileCursor {
    uint32_t e;
    uint64_t b0, b1;
    __device__ __forceinline__ void start(const MultiDev& m, const TileMap& tm, uint64_t t) {
        e = tm.owner(m, t);
        b0 = tm.begin(m, e);
        b1 = tm.begin(m, e + 1);
    }
    // Moves forward to the exploration owning tile t (t >= b0).
    __device__ __forceinline__ void seek(const MultiDev& m, const TileMap& tm, uint64_t t) {
        while (t >= b1) {
            ++e;
            b0 = b1;
            b1 = tm.begin(m, e + 1);
        }
    }
    // Index in the successor buffer of lane `lane`'s key of tile t (may lie
    // past the exploration's count, but inside its 32-rounded segment).
    __device__ __forceinline__ uint64_t key_index(const MultiDev& m, uint64_t t, int lane) const {
        return __ldcg(m.seg_off + e) + 32 * (t - b0) + uint64_t(lane);
    }
};

__device__ __forceinline__ uint64_t step_count(const MultiDev& m, uint32_t e) {
    return min(uint64_t(__ldcg(m.seg_cnt + e)), uint64_t(__ldcg(m.take + e)) * uint64_t(__ldcg(m.msucc + e)));
}

// Block-wide (NT threads): the exact tile prefix into first[0..count]
// (kExactTileExpl + 1 entries; a step has at most 2^26 successors, so
// 32-bit entries suffice) with `scratch` (kAdvShared words) for the scans.
// Returns the map: the upper-bound layout when the group is too large.
template <int NT>
__device__ __forceinline__ TileMap tile_map(const MultiDev& m, unsigned int* first, unsigned long long* scratch) {
    TileMap tm;
    tm.first = nullptr;
    if (m.count > kExactTileExpl) return tm;
    unsigned long long carry = 0;
    for (uint32_t base = 0; base < m.count; base += NT) {
        const uint32_t e = base + threadIdx.x;
        const unsigned long long v = e < m.count ? (step_count(m, e) + 31) / 32 : 0;
        const unsigned long long x = block_excl_scan<NT>(v, scratch);
        if (e < m.count) first[e] = unsigned(carry + x);
        carry += block_sum<NT>(v, scratch);
    }
    if (threadIdx.x == 0) first[m.count] = unsigned(carry);
    __syncthreads();
    tm.first = first;
    return tm;
}



}  // namespace multi
}  // namespace ht
