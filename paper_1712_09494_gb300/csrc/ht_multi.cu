// Batched exploration: many independent state-space BFS runs of uneven
// sizes advanced together, one step of every run per graph launch.
//
// Each exploration e owns a table, a states array (all its states in level
// order: level d is [lo, hi) when it is being expanded) and a cursor `cur`
// into the current level.  One step is three kernels over all explorations
// of a group (tables of the same key width and bucket shape):
//   advance     one block: moves every cursor past the states expanded in the
//               previous step, opens the next level when a level is done,
//               and shares the successor buffer among the explorations that
//               still have work (`take` states each), with prefix sums;
//   successors  one thread per expanded state, found by binary search;
//   find-or-put one warp per 32 successors of one exploration (bucket_tile),
//               new states appended to that exploration's states array.
// The step is captured once as a CUDA graph and replayed until no
// exploration is active; the host reads one flag per step.
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ht_internal.cuh"

using namespace ht;

namespace ht {
namespace {

// Status bits of every table of a group (a key that found no place sets
// kFlagDropped), gathered after a run in one launch.
__global__ void multi_flags_kernel(const DevTable* __restrict__ tables, uint32_t n, unsigned int* __restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __ldcg(&tables[i].ctr->flags);
}

constexpr int kAdvThreads = 1024;

// Block-wide sum of one value per thread (blockDim.x == kAdvThreads).
__device__ unsigned long long block_sum(unsigned long long v, unsigned long long* sh) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int o = 16; o; o >>= 1) v += __shfl_down_sync(0xFFFFFFFFu, v, o);
    __syncthreads();
    if (lane == 0) sh[warp] = v;
    __syncthreads();
    unsigned long long t = 0;
    if (warp == 0) {
        t = lane < (kAdvThreads / 32) ? sh[lane] : 0;
        for (int o = 16; o; o >>= 1) t += __shfl_down_sync(0xFFFFFFFFu, t, o);
        if (lane == 0) sh[32] = t;
    }
    __syncthreads();
    return sh[32];
}

// Block-wide exclusive scan of one value per thread.
__device__ unsigned long long block_excl_scan(unsigned long long v, unsigned long long* sh) {
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
        unsigned long long w = lane < (kAdvThreads / 32) ? sh[lane] : 0;
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

__global__ void __launch_bounds__(kAdvThreads) multi_advance_kernel(const MultiDev m, uint64_t budget) {
    __shared__ unsigned long long sh[40];
    const uint32_t per = (m.count + kAdvThreads - 1) / kAdvThreads;
    const uint32_t e0 = min(m.count, threadIdx.x * per), e1 = min(m.count, e0 + per);
    unsigned long long want = 0, act = 0;
    for (uint32_t e = e0; e < e1; ++e) {
        if (m.done[e]) {
            m.take[e] = 0;
            continue;
        }
        const unsigned long long cur = m.cur[e] + m.take[e];
        unsigned long long hi = m.hi[e];
        m.cur[e] = cur;
        m.take[e] = 0;
        if (cur >= hi) {                               // the level is fully expanded
            const unsigned long long nh = __ldcg(m.total + e);
            if (nh > m.states_cap[e]) {
                m.done[e] = 2;                         // states array full
            } else if (nh == hi) {
                m.done[e] = 1;                         // no new states: finished
            } else if (m.level[e] + 1 >= m.max_levels) {
                m.done[e] = 2;
            } else {
                const unsigned int lvl = m.level[e] + 1;
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
    const unsigned long long total_want = block_sum(want, sh);
    const unsigned long long total_act = block_sum(act, sh);
    // Fair share of the successor buffer, in proportion to remaining work.
    const double scale = total_want <= budget ? 1.0 : double(budget) / double(total_want);
    unsigned long long my_take = 0, my_seg = 0;
    for (uint32_t e = e0; e < e1; ++e) {
        if (m.done[e]) continue;
        const unsigned long long rem = m.hi[e] - m.cur[e];
        unsigned long long tk = scale >= 1.0 ? rem : (unsigned long long)(double(rem) * scale);
        tk = max(1ull, min(tk, rem));
        m.take[e] = tk;
        my_take += tk;
        my_seg += (tk * m.msucc[e] + 31) / 32 * 32;
    }
    unsigned long long w_off = block_excl_scan(my_take, sh);
    unsigned long long s_off = block_excl_scan(my_seg, sh);
    for (uint32_t e = e0; e < e1; ++e) {
        m.work_off[e] = w_off;
        m.seg_off[e] = s_off;
        m.seg_cnt[e] = 0;
        w_off += m.take[e];
        s_off += (m.take[e] * m.msucc[e] + 31) / 32 * 32;
    }
    if (threadIdx.x == kAdvThreads - 1) {
        *m.work_total = w_off;
        *m.tiles_total = s_off / 32;
        *m.active = unsigned(total_act);
    }
}

}  // namespace

cudaError_t multi_advance(const MultiDev& m, uint64_t budget, cudaStream_t s) {
    multi_advance_kernel<<<1, kAdvThreads, 0, s>>>(m, budget);
    return cudaGetLastError();
}

}  // namespace ht

namespace {

struct Group {
    BucketCfg cfg;
    std::vector<uint32_t> members;   // exploration ids
    MultiDev dev;
    void* arena = nullptr;           // counters and tables
    uint64_t budget = 0;             // successors per step
    uint64_t max_work = 0, max_tiles = 0;
    unsigned int* h_active = nullptr;  // pinned
    unsigned int* d_flags = nullptr;   // [count] tables' device status bits after a run
    cudaStream_t s = nullptr;          // the group's stream in a step (groups after the first)
    cudaEvent_t joined = nullptr;      // the group's step is done
};


}  // namespace

struct ht_multi {
    int device = 0;
    cudaStream_t stream = nullptr;
    uint32_t count = 0;
    uint32_t max_levels = 0;
    std::vector<ht_table*> tables;
    std::vector<void*> states;
    std::vector<uint64_t> states_cap;
    std::vector<ht_model> models;
    std::vector<uint64_t> s0;
    std::vector<Group> groups;
    cudaEvent_t fork = nullptr;        // a step starts (the other groups' streams wait for it)
    cudaGraphExec_t graph = nullptr;
    // results (host)
    std::vector<uint64_t> res_states, res_levels, res_gen;
    std::vector<int> res_complete;
    std::vector<uint64_t> res_sizes;   // count * max_levels
    uint64_t steps = 0;
};

namespace {

void destroy_multi(ht_multi* m) {
    if (!m) return;
    if (m->graph) cudaGraphExecDestroy(m->graph);
    for (auto& g : m->groups) {
        cudaFree(g.arena);
        cudaFree(g.dev.succ);
        cudaFree(g.d_flags);
        cudaFreeHost(g.h_active);
        if (g.s) cudaStreamDestroy(g.s);
        if (g.joined) cudaEventDestroy(g.joined);
    }
    if (m->fork) cudaEventDestroy(m->fork);
    for (void* p : m->states) cudaFree(p);
    for (ht_table* t : m->tables) ht_destroy(t);
    if (m->stream) cudaStreamDestroy(m->stream);
    delete m;
}

template <typename T>
T* carve(char*& p, uint64_t n) {
    T* r = reinterpret_cast<T*>(p);
    p += (n * sizeof(T) + 255) / 256 * 256;
    return r;
}

// One step: each group (explorations of one key width and bucket shape)
// advances, generates successors and finds-or-puts them.  Groups are
// independent, so groups after the first run on their own streams, forked
// from and joined back into the main stream (parallel branches when the step
// is captured as a graph).
ht_status step_launches(ht_multi* m) {
    if (cudaEventRecord(m->fork, m->stream) != cudaSuccess) return HT_ERR_CUDA;
    for (size_t i = 0; i < m->groups.size(); ++i) {
        Group& g = m->groups[i];
        const cudaStream_t s = i == 0 ? m->stream : g.s;
        if (i > 0 && cudaStreamWaitEvent(s, m->fork, 0) != cudaSuccess) return HT_ERR_CUDA;
        if (multi_advance(g.dev, g.budget, s) != cudaSuccess ||
            multi_successors(g.cfg.kw, g.dev, g.max_work, s) != cudaSuccess ||
            multi_bucket_find_or_put(g.cfg, g.dev, g.max_tiles, s) != cudaSuccess ||
            cudaMemcpyAsync(g.h_active, g.dev.active, sizeof(unsigned int), cudaMemcpyDeviceToHost, s) != cudaSuccess)
            return HT_ERR_CUDA;
        if (i > 0 && (cudaEventRecord(g.joined, s) != cudaSuccess || cudaStreamWaitEvent(m->stream, g.joined, 0) != cudaSuccess))
            return HT_ERR_CUDA;
    }
    return HT_OK;
}

ht_status reset_multi(ht_multi* m) {
    for (ht_table* t : m->tables) {
        ht_status st = ht_clear(t, m->stream);
        if (st != HT_OK) return st;
    }
    for (auto& g : m->groups) {
        const uint64_t n = g.members.size();
        // Zero every counter array (they sit contiguously at the arena's start).
        const char* first = reinterpret_cast<const char*>(g.dev.total);
        const char* last = reinterpret_cast<const char*>(g.dev.active) + 256;
        if (cudaMemsetAsync(const_cast<char*>(first), 0, size_t(last - first), m->stream) != cudaSuccess)
            return HT_ERR_CUDA;
        if (cudaMemsetAsync(g.dev.level_sizes, 0, n * m->max_levels * sizeof(unsigned long long), m->stream) !=
            cudaSuccess)
            return HT_ERR_CUDA;
    }
    return HT_OK;
}

}  // namespace

extern "C" {

ht_status ht_multi_create(uint32_t count, const ht_model* h_models, const uint64_t* h_s0, const uint64_t* h_capacity,
                          const ht_params* h_params, uint32_t max_levels, void* stream, ht_multi** out) {
    if (!out || count == 0 || count > (1u << 16) || !h_models || !h_s0 || !h_capacity || max_levels == 0 ||
        max_levels > 65536)
        return HT_ERR_INVALID;
    *out = nullptr;
    ht_multi* m = new (std::nothrow) ht_multi();
    if (!m) return HT_ERR_OOM;
    cudaGetDevice(&m->device);
    m->count = count;
    m->max_levels = max_levels;
    m->models.assign(h_models, h_models + count);
    m->s0.assign(h_s0, h_s0 + count);
    if (cudaStreamCreateWithFlags(&m->stream, cudaStreamNonBlocking) != cudaSuccess) {
        delete m;
        return HT_ERR_CUDA;
    }
    // One table per exploration (bucket scheme), key width from the model.
    std::vector<uint64_t> msucc(count);
    std::vector<uint32_t> kws(count);
    for (uint32_t e = 0; e < count; ++e) {
        uint32_t bits = 0;
        for (int c = 0; c < h_models[e].num_components && c < 16; ++c) bits += h_models[e].bits[c];
        kws[e] = bits <= 31 ? 32 : 64;
        msucc[e] = model_max_successors(&h_models[e], kws[e]);
        const ht_params* p = h_params ? &h_params[e] : nullptr;
        ht_table* t = nullptr;
        ht_status st = msucc[e] && (kws[e] == 64 || h_s0[e] < 0xFFFFFFFFull) && (kws[e] == 32 || !(h_s0[e] >> 63))
                           ? ht_create(h_capacity[e], HT_BUCKET, kws[e], p, m->stream, &t)
                           : HT_ERR_INVALID;
        if (st != HT_OK) {
            destroy_multi(m);
            return st;
        }
        m->tables.push_back(t);
        uint64_t slots = 0;
        ht_info(t, &slots, nullptr, nullptr);
        const DevTable& dt = table_dev(t);
        m->states_cap.push_back(slots + dt.stash_slots + dt.ovf_slots);
        void* sp = nullptr;
        if (cudaMalloc(&sp, m->states_cap.back() * (kws[e] / 8)) != cudaSuccess) {
            destroy_multi(m);
            return HT_ERR_OOM;
        }
        m->states.push_back(sp);
    }
    // Group explorations by (key width, bucket shape).
    for (uint32_t e = 0; e < count; ++e) {
        const BucketCfg c = table_bucket_cfg(m->tables[e]);
        Group* g = nullptr;
        for (auto& x : m->groups)
            if (x.cfg.kw == c.kw && x.cfg.bucket_slots == c.bucket_slots && x.cfg.lanes == c.lanes) g = &x;
        if (!g) {
            m->groups.emplace_back();
            g = &m->groups.back();
            g->cfg = c;
        }
        g->members.push_back(e);
    }
    if (cudaEventCreateWithFlags(&m->fork, cudaEventDisableTiming) != cudaSuccess) {
        destroy_multi(m);
        return HT_ERR_CUDA;
    }
    for (size_t i = 1; i < m->groups.size(); ++i) {
        Group& g = m->groups[i];
        if (cudaStreamCreateWithFlags(&g.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&g.joined, cudaEventDisableTiming) != cudaSuccess) {
            destroy_multi(m);
            return HT_ERR_CUDA;
        }
    }
    for (auto& g : m->groups) {
        const uint64_t n = g.members.size();
        uint64_t most = 1;
        for (uint32_t e : g.members) most = std::max(most, msucc[e]);
        g.budget = uint64_t(1) << 24;
        const uint64_t succ_cap = g.budget + n * (32 + most) + 32;
        const uint64_t bytes = 16 * ((n * 8 + 255) / 256 * 256) + ((n * max_levels * 8 + 255) / 256 * 256) +
                               3 * 256 + n * sizeof(DevTable) + 256 + n * sizeof(PreparedModel) + 256 +
                               n * sizeof(void*) + 256;
        if (cudaMalloc(&g.arena, bytes) != cudaSuccess || cudaMalloc(&g.dev.succ, succ_cap * 8) != cudaSuccess ||
            cudaMalloc(&g.d_flags, n * sizeof(unsigned int)) != cudaSuccess ||
            cudaMallocHost(&g.h_active, sizeof(unsigned int)) != cudaSuccess) {
            destroy_multi(m);
            return HT_ERR_OOM;
        }
        char* p = static_cast<char*>(g.arena);
        MultiDev& d = g.dev;
        d.count = uint32_t(n);
        d.max_levels = max_levels;
        d.succ_cap = succ_cap;
        // Counters first (reset_multi zeroes [total, active]).
        d.total = carve<unsigned long long>(p, n);
        d.lo = carve<unsigned long long>(p, n);
        d.hi = carve<unsigned long long>(p, n);
        d.cur = carve<unsigned long long>(p, n);
        d.take = carve<unsigned long long>(p, n);
        d.work_off = carve<unsigned long long>(p, n);
        d.seg_off = carve<unsigned long long>(p, n);
        d.seg_cnt = carve<unsigned long long>(p, n);
        d.gen = carve<unsigned long long>(p, n);
        d.level = carve<unsigned int>(p, n);
        d.done = carve<unsigned int>(p, n);
        d.work_total = carve<unsigned long long>(p, 1);
        d.tiles_total = carve<unsigned long long>(p, 1);
        d.active = carve<unsigned int>(p, 1);
        // Constant per-exploration data.
        unsigned long long* caps = carve<unsigned long long>(p, n);
        unsigned long long* ms = carve<unsigned long long>(p, n);
        unsigned long long* s0 = carve<unsigned long long>(p, n);
        d.level_sizes = carve<unsigned long long>(p, n * max_levels);
        DevTable* tabs = carve<DevTable>(p, n);
        PreparedModel* mods = carve<PreparedModel>(p, n);
        void** sts = carve<void*>(p, n);
        d.states_cap = caps;
        d.msucc = ms;
        d.s0 = s0;
        d.tables = tabs;
        d.models = mods;
        d.states = sts;
        std::vector<unsigned long long> hc(n), hm(n), hs(n);
        std::vector<DevTable> ht(n);
        std::vector<PreparedModel> hp(n);
        std::vector<void*> hst(n);
        for (uint64_t i = 0; i < n; ++i) {
            const uint32_t e = g.members[i];
            hc[i] = m->states_cap[e];
            hm[i] = msucc[e];
            hs[i] = h_s0[e];
            ht[i] = table_dev(m->tables[e]);
            hp[i] = prepare_model(h_models[e]);
            hst[i] = m->states[e];
        }
        cudaStream_t s = m->stream;
        if (cudaMemcpyAsync(caps, hc.data(), n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(ms, hm.data(), n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(s0, hs.data(), n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(tabs, ht.data(), n * sizeof(DevTable), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(mods, hp.data(), n * sizeof(PreparedModel), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(sts, hst.data(), n * sizeof(void*), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            destroy_multi(m);
            return HT_ERR_CUDA;
        }
        g.max_work = g.budget + n;
        g.max_tiles = succ_cap / 32;
    }
    m->res_states.assign(count, 0);
    m->res_levels.assign(count, 0);
    m->res_gen.assign(count, 0);
    m->res_complete.assign(count, 0);
    m->res_sizes.assign(uint64_t(count) * max_levels, 0);
    ht_status st = reset_multi(m);
    if (st == HT_OK && cudaStreamSynchronize(m->stream) != cudaSuccess) st = HT_ERR_CUDA;
    if (st != HT_OK) {
        destroy_multi(m);
        return st;
    }
    (void)stream;
    *out = m;
    return HT_OK;
}

ht_status ht_multi_reset(ht_multi* m, void* stream) {
    if (!m) return HT_ERR_INVALID;
    cudaSetDevice(m->device);
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return HT_ERR_CUDA;
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    cudaEventRecord(ev, caller);
    cudaStreamWaitEvent(m->stream, ev, 0);
    ht_status st = reset_multi(m);
    cudaEventRecord(ev, m->stream);
    cudaStreamWaitEvent(caller, ev, 0);
    cudaEventDestroy(ev);
    return st;
}

ht_status ht_multi_destroy(ht_multi* m) {
    if (!m) return HT_OK;
    cudaSetDevice(m->device);
    cudaStreamSynchronize(m->stream);
    destroy_multi(m);
    return HT_OK;
}

ht_status ht_multi_run(ht_multi* m, int mode, uint64_t max_steps, void* stream) {
    if (!m || mode < 0 || mode > 2) return HT_ERR_INVALID;
    cudaSetDevice(m->device);
    cudaStream_t caller = static_cast<cudaStream_t>(stream);
    cudaEvent_t ev;
    if (cudaEventCreateWithFlags(&ev, cudaEventDisableTiming) != cudaSuccess) return HT_ERR_CUDA;
    cudaEventRecord(ev, caller);
    cudaStreamWaitEvent(m->stream, ev, 0);
    ht_status st = HT_OK;
    m->steps = 0;
    if (st == HT_OK && mode == 2) {
        // Baseline: one exploration after another, each with its own per-level
        // launches and synchronisation (ht_bfs).
        std::vector<uint64_t> sizes(m->max_levels);
        for (uint32_t e = 0; e < m->count && st == HT_OK; ++e) {
            ht_bfs_result r;
            st = ht_bfs(m->tables[e], &m->models[e], m->s0[e], m->max_levels, sizes.data(), m->states[e],
                        m->states_cap[e], &r, m->stream);
            if (st != HT_OK) break;
            m->res_states[e] = r.states;
            m->res_levels[e] = r.levels;
            m->res_gen[e] = r.successors;
            m->res_complete[e] = r.complete;
            std::copy(sizes.begin(), sizes.begin() + std::min<uint64_t>(r.levels, m->max_levels),
                      m->res_sizes.begin() + uint64_t(e) * m->max_levels);
            m->steps += r.levels;
        }
    } else if (st == HT_OK) {
        for (auto& g : m->groups)
            if (multi_bucket_init(g.cfg, g.dev, m->stream) != cudaSuccess) st = HT_ERR_CUDA;
        if (st == HT_OK && mode == 0 && !m->graph) {
            // Capture one step (all groups) as a graph, once.
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(m->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) st = HT_ERR_CUDA;
            ht_status ls = st == HT_OK ? step_launches(m) : st;
            if (cudaStreamEndCapture(m->stream, &graph) != cudaSuccess || ls != HT_OK) st = HT_ERR_CUDA;
            if (st == HT_OK && cudaGraphInstantiate(&m->graph, graph, 0) != cudaSuccess) st = HT_ERR_CUDA;
            if (graph) cudaGraphDestroy(graph);
        }
        const uint64_t limit = max_steps ? max_steps : (uint64_t(1) << 22);
        while (st == HT_OK && m->steps < limit) {
            if (mode == 0) {
                if (cudaGraphLaunch(m->graph, m->stream) != cudaSuccess) st = HT_ERR_CUDA;
            } else {
                st = step_launches(m);
            }
            if (st != HT_OK || cudaStreamSynchronize(m->stream) != cudaSuccess) {
                st = st == HT_OK ? HT_ERR_CUDA : st;
                break;
            }
            ++m->steps;
            unsigned int active = 0;
            for (auto& g : m->groups) active += *g.h_active;
            if (!active) break;
        }
        // Collect per-exploration results.
        for (auto& g : m->groups) {
            if (st != HT_OK) break;
            const uint64_t n = g.members.size();
            std::vector<unsigned long long> tot(n), gen(n), sz(n * m->max_levels);
            std::vector<unsigned int> lvl(n), done(n), flags(n);
            multi_flags_kernel<<<uint32_t((n + 255) / 256), 256, 0, m->stream>>>(g.dev.tables, uint32_t(n), g.d_flags);
            if (cudaGetLastError() != cudaSuccess ||
                cudaMemcpyAsync(flags.data(), g.d_flags, n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
                cudaMemcpyAsync(tot.data(), g.dev.total, n * 8, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
                cudaMemcpyAsync(gen.data(), g.dev.gen, n * 8, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
                cudaMemcpyAsync(lvl.data(), g.dev.level, n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
                cudaMemcpyAsync(done.data(), g.dev.done, n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
                cudaMemcpyAsync(sz.data(), g.dev.level_sizes, n * m->max_levels * 8, cudaMemcpyDeviceToHost,
                                m->stream) != cudaSuccess ||
                cudaStreamSynchronize(m->stream) != cudaSuccess) {
                st = HT_ERR_CUDA;
                break;
            }
            for (uint64_t i = 0; i < n; ++i) {
                const uint32_t e = g.members[i];
                // A table that dropped a key makes the exploration inexact.
                if (flags[i] & kFlagDropped) st = HT_ERR_FULL;
                m->res_complete[e] = done[i] == 1;
                m->res_states[e] = std::min<uint64_t>(tot[i], m->states_cap[e]);
                m->res_levels[e] = tot[i] ? uint64_t(lvl[i]) + 1 : 0;
                m->res_gen[e] = gen[i];
                std::copy(sz.begin() + i * m->max_levels, sz.begin() + (i + 1) * m->max_levels,
                          m->res_sizes.begin() + uint64_t(e) * m->max_levels);
            }
        }
    }
    cudaEventRecord(ev, m->stream);
    cudaStreamWaitEvent(caller, ev, 0);
    cudaEventDestroy(ev);
    return st;
}

ht_status ht_multi_result(const ht_multi* m, uint32_t i, uint64_t* levels, uint64_t* states, uint64_t* successors,
                          int32_t* complete, uint64_t* h_level_sizes, const void** d_states, void* h_states,
                          uint64_t h_states_cap) {
    if (!m || i >= m->count) return HT_ERR_INVALID;
    if (h_states && h_states_cap) {
        cudaSetDevice(m->device);
        const uint32_t kw = table_key_width(m->tables[i]);
        const uint64_t n = std::min<uint64_t>(m->res_states[i], h_states_cap);
        if (cudaMemcpyAsync(h_states, m->states[i], n * (kw / 8), cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaStreamSynchronize(m->stream) != cudaSuccess)
            return HT_ERR_CUDA;
    }
    if (levels) *levels = m->res_levels[i];
    if (states) *states = m->res_states[i];
    if (successors) *successors = m->res_gen[i];
    if (complete) *complete = m->res_complete[i];
    if (h_level_sizes)
        std::copy(m->res_sizes.begin() + uint64_t(i) * m->max_levels,
                  m->res_sizes.begin() + uint64_t(i) * m->max_levels + std::min<uint64_t>(m->res_levels[i], m->max_levels),
                  h_level_sizes);
    if (d_states) *d_states = m->states[i];
    return HT_OK;
}

uint64_t ht_multi_steps(const ht_multi* m) { return m ? m->steps : 0; }

}  // extern "C"
