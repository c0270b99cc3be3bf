// Batched exploration: many independent state-space BFS runs of uneven
// sizes advanced together (ht_multi_*).
//
// Each exploration e owns a table, a states array (all its states in level
// order: level d is [lo, hi) when it is being expanded) and a cursor `cur`
// into the current level.  Explorations are grouped by table kind (key
// width, scheme, bucket shape); a step of a group is advance / successors /
// find-or-put over all its explorations (ht_multi_dev.cuh).  Four ways to
// run them (ht_multi_run's mode):
//   0  persistent: one cooperative launch per group runs every step, with
//      bounded grid barriers between phases (ht_persist.cu); the host waits
//      once, for the results.  Bucket and Cuckoo groups.
//   1  one launch per phase and step, the host reading an `active` flag
//      after every step (bucket groups).
//   2  one exploration after another with ht_bfs (the baseline: per-level
//      launches for one table at a time).  Bucket and Cuckoo.
//   3  mode 1's step captured once as a CUDA graph and replayed per step
//      (bucket groups).
#include <algorithm>
#include <cstring>
#include <new>
#include <vector>

#include "ht_multi_dev.cuh"

// Successors a step may generate (the upper bound take * msucc summed over
// the explorations); the successor buffer holds that plus per-exploration
// rounding slack.
#ifndef HT_MULTI_BUDGET_LOG2
#define HT_MULTI_BUDGET_LOG2 26
#endif

namespace {
constexpr uint64_t kDefaultBarrierNs = 2000000000ull;   // a persistent run's bound on one barrier wait
}

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

__global__ void __launch_bounds__(kAdvThreads) multi_advance_kernel(const MultiDev m, uint64_t budget) {
    __shared__ unsigned long long sh[multi::kAdvShared];
    multi::advance<kAdvThreads>(m, budget, sh);
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
    ht_scheme scheme = HT_BUCKET;
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
        cudaFree(g.dev.win);
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

// One step: each group (explorations of one scheme and bucket shape)
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
        const char* last = reinterpret_cast<const char*>(g.dev.steps) + 256;
        if (cudaMemsetAsync(const_cast<char*>(first), 0, size_t(last - first), m->stream) != cudaSuccess)
            return HT_ERR_CUDA;
        if (cudaMemsetAsync(g.dev.level_sizes, 0, n * m->max_levels * sizeof(unsigned long long), m->stream) !=
            cudaSuccess)
            return HT_ERR_CUDA;
    }
    return HT_OK;
}

// Reads every exploration's counters, level sizes and table status after a
// batched run (modes 0, 1, 3): all groups' copies, then one synchronisation.
// The persistent mode also reports its steps and its status word.
ht_status collect_results(ht_multi* m, bool persistent) {
    const size_t G = m->groups.size();
    std::vector<std::vector<unsigned long long>> tot(G), gen(G), sz(G);
    std::vector<std::vector<unsigned int>> lvl(G), done(G), flags(G);
    std::vector<unsigned long long> steps(G, 0);
    std::vector<unsigned int> status(G, 0);
    for (size_t gi = 0; gi < G; ++gi) {
        Group& g = m->groups[gi];
        const uint64_t n = g.members.size();
        tot[gi].resize(n);
        gen[gi].resize(n);
        sz[gi].resize(n * m->max_levels);
        lvl[gi].resize(n);
        done[gi].resize(n);
        flags[gi].resize(n);
        multi_flags_kernel<<<uint32_t((n + 255) / 256), 256, 0, m->stream>>>(g.dev.tables, uint32_t(n), g.d_flags);
        if (cudaGetLastError() != cudaSuccess ||
            cudaMemcpyAsync(flags[gi].data(), g.d_flags, n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaMemcpyAsync(tot[gi].data(), g.dev.total, n * 8, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaMemcpyAsync(gen[gi].data(), g.dev.gen, n * 8, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaMemcpyAsync(lvl[gi].data(), g.dev.level, n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaMemcpyAsync(done[gi].data(), g.dev.done, n * 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
            cudaMemcpyAsync(sz[gi].data(), g.dev.level_sizes, n * m->max_levels * 8, cudaMemcpyDeviceToHost,
                            m->stream) != cudaSuccess)
            return HT_ERR_CUDA;
        if (persistent &&
            (cudaMemcpyAsync(&steps[gi], g.dev.steps, 8, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess ||
             cudaMemcpyAsync(&status[gi], g.dev.status, 4, cudaMemcpyDeviceToHost, m->stream) != cudaSuccess))
            return HT_ERR_CUDA;
    }
    if (cudaStreamSynchronize(m->stream) != cudaSuccess) return HT_ERR_CUDA;
    ht_status st = HT_OK;
    for (size_t gi = 0; gi < G; ++gi) {
        Group& g = m->groups[gi];
        if (persistent) {
            m->steps = std::max<uint64_t>(m->steps, steps[gi]);
            if (status[gi] & kMultiTimeout) return HT_ERR_TIMEOUT;
            if (status[gi] & kMultiBadInit) return HT_ERR_INVALID;
        }
        for (uint64_t i = 0; i < g.members.size(); ++i) {
            const uint32_t e = g.members[i];
            // A table that dropped a key makes the exploration inexact.
            if (flags[gi][i] & kFlagDropped) st = HT_ERR_FULL;
            m->res_complete[e] = done[gi][i] == 1;
            m->res_states[e] = std::min<uint64_t>(tot[gi][i], m->states_cap[e]);
            m->res_levels[e] = tot[gi][i] ? uint64_t(lvl[gi][i]) + 1 : 0;
            m->res_gen[e] = gen[gi][i];
            std::copy(sz[gi].begin() + i * m->max_levels, sz[gi].begin() + (i + 1) * m->max_levels,
                      m->res_sizes.begin() + uint64_t(e) * m->max_levels);
        }
    }
    return st;
}

}  // namespace

extern "C" {

ht_status ht_multi_create(uint32_t count, const ht_model* h_models, const uint64_t* h_s0, const uint64_t* h_capacity,
                          const ht_params* h_params, uint32_t max_levels, void* stream, ht_multi** out) {
    return ht_multi_create_ex(count, h_models, h_s0, h_capacity, nullptr, h_params, max_levels, stream, out);
}

ht_status ht_multi_create_ex(uint32_t count, const ht_model* h_models, const uint64_t* h_s0,
                             const uint64_t* h_capacity, const ht_scheme* h_schemes, const ht_params* h_params,
                             uint32_t max_levels, void* stream, ht_multi** out) {
    if (!out || count == 0 || count > (1u << 16) || !h_models || !h_s0 || !h_capacity || max_levels == 0 ||
        max_levels > 65536)
        return HT_ERR_INVALID;
    if (h_schemes)
        for (uint32_t e = 0; e < count; ++e)
            if (h_schemes[e] != HT_BUCKET && h_schemes[e] != HT_CUCKOO) return HT_ERR_INVALID;
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
    // One table per exploration (h_schemes[e], bucket if NULL), key width
    // from the model.
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
                           ? ht_create(h_capacity[e], h_schemes ? h_schemes[e] : HT_BUCKET, kws[e], p, m->stream, &t)
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
    // Group explorations by (scheme, bucket shape).  Key widths share a
    // group: the group's kernels address every table as a 64-bit key table
    // (a 32-bit set table holds key k as the word k, the same word) and read
    // and write each exploration's states in its own width.
    for (uint32_t e = 0; e < count; ++e) {
        const ht_scheme sch = table_scheme(m->tables[e]);
        BucketCfg c = table_bucket_cfg(m->tables[e]);
        c.kw = 64;
        if (sch == HT_CUCKOO) c.bucket_slots = c.lanes = 0;    // no bucket shape
        Group* g = nullptr;
        for (auto& x : m->groups)
            if (x.scheme == sch && x.cfg.kw == c.kw && x.cfg.bucket_slots == c.bucket_slots && x.cfg.lanes == c.lanes)
                g = &x;
        if (!g) {
            m->groups.emplace_back();
            g = &m->groups.back();
            g->cfg = c;
            g->scheme = sch;
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
        g.budget = uint64_t(1) << HT_MULTI_BUDGET_LOG2;
        const uint64_t succ_cap = g.budget + n * (32 + most) + 32;
        const uint64_t bytes = 18 * ((n * 8 + 255) / 256 * 256) + ((n * max_levels * 8 + 255) / 256 * 256) +
                               8 * 256 + n * sizeof(DevTable) + 256 + n * sizeof(PreparedModel) + 256 +
                               n * sizeof(void*) + 256 + n * sizeof(DevScratch) + 256 + n + 256;
        // Cuckoo: one winner record per successor of a step at most.
        if (g.scheme == HT_CUCKOO && cudaMalloc(&g.dev.win, succ_cap * sizeof(MultiWinner)) != cudaSuccess) {
            destroy_multi(m);
            return HT_ERR_OOM;
        }
        g.dev.win_cap = g.scheme == HT_CUCKOO ? succ_cap : 0;
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
        d.win_count = carve<unsigned long long>(p, 1);
        d.bar = carve<unsigned int>(p, 2);
        d.status = carve<unsigned int>(p, 1);
        d.steps = carve<unsigned long long>(p, 1);      // last of the zeroed counters
        d.barrier_ns = kDefaultBarrierNs;
        d.absent_block = -1;
        // Constant per-exploration data.
        unsigned long long* caps = carve<unsigned long long>(p, n);
        unsigned long long* ms = carve<unsigned long long>(p, n);
        unsigned long long* s0 = carve<unsigned long long>(p, n);
        d.level_sizes = carve<unsigned long long>(p, n * max_levels);
        DevTable* tabs = carve<DevTable>(p, n);
        PreparedModel* mods = carve<PreparedModel>(p, n);
        void** sts = carve<void*>(p, n);
        DevScratch* scr = carve<DevScratch>(p, n);
        unsigned long long* tcap = carve<unsigned long long>(p, n);
        uint8_t* nar = carve<uint8_t>(p, n);
        d.narrow = nar;
        d.scratch = g.scheme == HT_CUCKOO ? scr : nullptr;
        d.take_cap = g.scheme == HT_CUCKOO ? tcap : nullptr;
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
        std::vector<DevScratch> hsc(n);
        std::vector<unsigned long long> htc(n, 0);
        std::vector<uint8_t> hnar(n);
        for (uint64_t i = 0; i < n; ++i) {
            const uint32_t e = g.members[i];
            hc[i] = m->states_cap[e];
            hm[i] = msucc[e];
            hs[i] = h_s0[e];
            ht[i] = table_dev(m->tables[e]);
            hp[i] = prepare_model(h_models[e]);
            hst[i] = m->states[e];
            hnar[i] = kws[e] == 32;
            if (g.scheme == HT_CUCKOO) {
                // A step's distinct absent keys are at most the states the
                // exploration can still hold, and the claim set has twice
                // win_cap slots: when win_cap covers the states array, the
                // set stays at most half full whatever the step's size.
                // Otherwise (a table larger than its claim set, max_batch
                // below its size) a step expands at most as many states as
                // keep its successors within win_cap, as the single-table
                // path chunks a batch.
                hsc[i] = table_scratch(m->tables[e]);
                if (hsc[i].win_cap < m->states_cap[e]) htc[i] = std::max<uint64_t>(1, hsc[i].win_cap / msucc[e]);
            }
        }
        cudaStream_t s = m->stream;
        if (cudaMemcpyAsync(caps, hc.data(), n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(ms, hm.data(), n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(s0, hs.data(), n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(tabs, ht.data(), n * sizeof(DevTable), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(mods, hp.data(), n * sizeof(PreparedModel), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(sts, hst.data(), n * sizeof(void*), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(scr, hsc.data(), n * sizeof(DevScratch), cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(tcap, htc.data(), n * 8, cudaMemcpyHostToDevice, s) != cudaSuccess ||
            cudaMemcpyAsync(nar, hnar.data(), n, cudaMemcpyHostToDevice, s) != cudaSuccess ||
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
    if (!m || mode < 0 || mode > 3) return HT_ERR_INVALID;
    if (mode == 1 || mode == 3)
        for (auto& g : m->groups)
            if (g.scheme != HT_BUCKET) return HT_ERR_INVALID;     // per-step kernels: bucket tables only
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
    } else if (st == HT_OK && mode == 0) {
        // One persistent launch per group, one after another on the stream
        // (each fills the device, so they would not overlap anyway).
        const uint64_t limit = max_steps ? max_steps : (uint64_t(1) << 22);
        for (auto& g : m->groups) {
            if (cudaMemsetAsync(g.dev.win_count, 0, 256 * 4, m->stream) != cudaSuccess ||   // win_count .. steps
                multi_persistent(g.scheme, g.cfg, g.dev, g.budget, limit, g.max_work, g.max_tiles, m->stream) !=
                    cudaSuccess) {
                st = HT_ERR_CUDA;
                break;
            }
        }
    } else if (st == HT_OK) {
        for (auto& g : m->groups)
            if (multi_bucket_init(g.cfg, g.dev, m->stream) != cudaSuccess) st = HT_ERR_CUDA;
        if (st == HT_OK && mode == 3 && !m->graph) {
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
            if (mode == 3) {
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
    }
    if (st == HT_OK && mode != 2) st = collect_results(m, mode == 0);
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

ht_status ht_multi_test_hooks(ht_multi* m, uint64_t barrier_timeout_ns, int32_t absent_block) {
    if (!m || absent_block < -1) return HT_ERR_INVALID;
    for (auto& g : m->groups) {
        g.dev.barrier_ns = barrier_timeout_ns ? barrier_timeout_ns : kDefaultBarrierNs;
        g.dev.absent_block = absent_block;
    }
    return HT_OK;
}

}  // extern "C"
