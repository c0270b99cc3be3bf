// Serving form: a request loop over many device-resident tables.
//
// Requests (find-or-put batches of 64-bit keys for one table) are queued per
// table.  A worker thread forms batches continuously: whenever one of the
// `max_inflight` batch slots is free it takes the head request of every
// table that has no request in flight (so each table's requests complete in
// arrival order and keep their sequential find-or-put meaning), packs their
// keys into that slot's pinned staging buffer, and issues on the slot's own
// stream: one copy in, one packed multi-table kernel for the bucket-scheme
// tables (one 32-key tile per warp, each against its own table), the
// Cuckoo tables' probe/insert launches, and one copy out.  Requests that
// arrive while slots are busy join the next batch, and the slots' streams
// overlap on the device.
//
// Tables are admitted when the free device memory (cudaMemGetInfo, or a
// test value) covers them plus a reserve; requests for a table wait until it
// is admitted.  Every wait the caller makes is bounded by its timeout.
#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ht_internal.cuh"

using namespace ht;

namespace {

using Clock = std::chrono::steady_clock;

struct Req {
    uint32_t table = 0;
    const uint64_t* keys = nullptr;
    uint64_t n = 0;
    uint8_t* out = nullptr;
    Clock::time_point t0, t1;
    bool pinned = false;           // keys are in page-locked host memory
    int state = 0;                 // 0 queued, 1 in flight, 2 done
    ht_status status = HT_OK;
};

struct Tab {
    uint64_t capacity = 0;
    ht_scheme scheme = HT_BUCKET;
    ht_table* t = nullptr;
    uint64_t bytes = 0;
    bool admitted = false, busy = false, closing = false, closed = false;
    cudaEvent_t ready = nullptr;   // recorded on the admission stream after the table's clear
    bool ready_seen = false;       // `ready` has completed
    std::deque<uint64_t> q;
};

struct Slot {
    cudaStream_t s = nullptr;
    cudaEvent_t ev0 = nullptr, ev = nullptr;   // batch start / end on the slot's stream
    uint64_t* h_keys = nullptr;    // pinned staging
    uint8_t* h_flags = nullptr;
    WorkDesc* h_desc = nullptr;
    uint32_t* h_tid = nullptr;     // per request of the batch: its table id ...
    uint32_t* h_flagw = nullptr;   // ... and that table's device status bits after the batch
    uint64_t* d_keys = nullptr;
    uint8_t* d_flags = nullptr;
    WorkDesc* d_desc = nullptr;
    uint32_t* d_tid = nullptr;
    uint32_t* d_flagw = nullptr;
    std::vector<std::pair<uint64_t, uint64_t>> reqs;   // (request id, key offset)
    bool busy = false;
    std::chrono::steady_clock::time_point issued;
};

uint64_t table_bytes(uint64_t capacity, ht_scheme scheme, const ht_params& p) {
    const uint64_t bs = p.bucket_slots ? p.bucket_slots : 16;
    const uint64_t slots = (capacity + bs - 1) / bs * bs;
    uint64_t b = slots * 8 + 4096 * 8 + (1 << 16) * 8 + 4096;
    if (scheme == HT_CUCKOO) {
        const uint64_t chunk = std::min<uint64_t>(p.max_batch ? p.max_batch : (1ull << 22), slots);
        b += 2 * chunk * 8 * 2 + chunk * 16;
    }
    return b;
}

// After a batch: the status bits of each request's table (a key that found
// no place anywhere sets kFlagDropped; a reserved key kFlagInvalidKey).
__global__ void serve_status_kernel(const DevTable* __restrict__ tables, const uint32_t* __restrict__ tid,
                                    uint32_t n, uint32_t* __restrict__ out) {
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) out[i] = __ldcg(&tables[tid[i]].ctr->flags);
}

}  // namespace

struct ht_server {
    ht_server_config cfg{};
    int device = 0;
    std::mutex mu;
    std::condition_variable cv_work, cv_done;
    std::thread worker;
    bool stop = false;
    std::vector<Tab> tabs;
    std::unordered_map<uint64_t, Req> reqs;
    uint64_t next_id = 1;
    std::vector<Slot> slots;
    DevTable* d_tables = nullptr;
    DevTable* h_tables = nullptr;  // pinned source of the descriptor copies (asynchronous)
    cudaStream_t admin = nullptr;
    uint64_t admitted_bytes = 0;
    uint64_t pool_threshold = 0;   // the default pool's release threshold before this server
    bool pool_kept = false;
    size_t rr = 0;                 // round-robin start over tables
    uint32_t first_waiting = 0;    // tables below this id are admitted or closed
    std::vector<double> lat_us;
    uint64_t keys_done = 0, batches = 0, requests_done = 0, tables_created = 0;
    double admit_s = 0, pack_s = 0, finish_s = 0, batch_us = 0, batch_gpu_us = 0;
    double inflight_s = 0;         // wall time with a batch in flight
    uint64_t table_bytes = 0;      // bytes of the tables created
    uint32_t inflight = 0;         // batches in flight
    Clock::time_point inflight_t0;
    Clock::time_point stats_t0;
    ht_status fault = HT_OK;
};

namespace {

constexpr uint32_t kMaxServerTables = 1u << 16;
// Requests at least this large whose keys are in page-locked memory are
// copied to the device straight from the caller's buffer (no staging copy).
constexpr uint64_t kDirectCopyKeys = 1u << 16;

uint64_t free_bytes(ht_server* sv) {
    if (sv->cfg.fake_free_bytes) {
        return sv->cfg.fake_free_bytes > sv->admitted_bytes ? sv->cfg.fake_free_bytes - sv->admitted_bytes : 0;
    }
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) return 0;
    // Memory freed by closed tables stays cached in the device's
    // stream-ordered pool, where new tables' allocations reuse it.
    cudaMemPool_t pool;
    uint64_t reserved = 0, used = 0;
    if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReservedMemCurrent, &reserved) == cudaSuccess &&
        cudaMemPoolGetAttribute(pool, cudaMemPoolAttrUsedMemCurrent, &used) == cudaSuccess && reserved > used)
        fr += reserved - used;
    return fr;
}

// Hands the pool's cached memory back to the driver (when a table's
// allocation failed although the cached memory looked large enough).
void trim_pool(ht_server* sv) {
    cudaStreamSynchronize(sv->admin);
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess) cudaMemPoolTrimTo(pool, 0);
}

// Admits waiting tables, in id order, while free memory covers them.  The
// free memory is queried once per pass (a device query costs tens of
// microseconds) and reduced by each table admitted in the pass; a table
// that then fails to allocate waits for the next pass.
bool admit(ht_server* sv) {
    bool any = false;
    const auto t0 = Clock::now();
    bool queried = false;
    uint64_t avail = 0;
    for (uint32_t id = sv->first_waiting; id < sv->tabs.size(); ++id) {
        Tab& tb = sv->tabs[id];
        if (tb.admitted || tb.closed) {
            if (id == sv->first_waiting) ++sv->first_waiting;    // every table before it is settled
            continue;
        }
        if (!queried) {
            avail = free_bytes(sv);
            queried = true;
        }
        if (avail < tb.bytes + sv->cfg.hbm_reserve_bytes) break;   // keep admission in order
        ht_params p = sv->cfg.table_params;
        if (tb.scheme == HT_CUCKOO) {
            const uint64_t seed = p.seed;
            ht_default_params(HT_CUCKOO, &p);
            p.seed = seed;
        }
        ht_table* t = nullptr;
        ht_status st = ht_create(tb.capacity, tb.scheme, 64, &p, sv->admin, &t);
        if (st == HT_ERR_OOM && !sv->cfg.fake_free_bytes) {
            trim_pool(sv);
            st = ht_create(tb.capacity, tb.scheme, 64, &p, sv->admin, &t);
        }
        if (st == HT_OK) {
            sv->h_tables[id] = table_dev(t);     // ids are never reused: the source stays valid
            if (cudaMemcpyAsync(sv->d_tables + id, sv->h_tables + id, sizeof(DevTable), cudaMemcpyHostToDevice,
                                sv->admin) != cudaSuccess)
                st = HT_ERR_CUDA;
        }
        // No wait here: a table joins batches once `ready` has completed, so
        // admission never stalls behind the batches in flight, and requests
        // of ready tables never wait for another table's clear.
        if (st == HT_OK && !tb.ready && cudaEventCreateWithFlags(&tb.ready, cudaEventDisableTiming) != cudaSuccess)
            st = HT_ERR_CUDA;
        if (st == HT_OK && cudaEventRecord(tb.ready, sv->admin) != cudaSuccess) st = HT_ERR_CUDA;
        if (st != HT_OK) {
            if (t) table_release(t, sv->admin);
            if (st == HT_ERR_OOM) break;          // try again when memory frees up
            sv->fault = st;
            break;
        }
        tb.t = t;
        tb.ready_seen = false;
        tb.admitted = true;
        sv->admitted_bytes += tb.bytes;
        sv->table_bytes += tb.bytes;
        avail -= std::min(avail, tb.bytes);
        sv->tables_created += 1;
        any = true;
    }
    if (any) sv->admit_s += std::chrono::duration<double>(Clock::now() - t0).count();
    return any;
}

void finish(ht_server* sv, Slot& sl) {
    const auto now = Clock::now();
    sv->batch_us += std::chrono::duration<double, std::micro>(now - sl.issued).count();
    float gpu_ms = 0.f;
    if (cudaEventElapsedTime(&gpu_ms, sl.ev0, sl.ev) == cudaSuccess) sv->batch_gpu_us += 1e3 * double(gpu_ms);
    for (size_t j = 0; j < sl.reqs.size(); ++j) {
        const auto& pr = sl.reqs[j];
        auto it = sv->reqs.find(pr.first);
        if (it == sv->reqs.end()) continue;
        Req& r = it->second;
        if (r.out) std::memcpy(r.out, sl.h_flags + pr.second, r.n);
        r.t1 = now;
        r.state = 2;
        // Sticky per table: once a key of the table found no place, its
        // requests report HT_ERR_FULL (nothing is dropped silently).
        const uint32_t fl = sl.h_flagw[j];
        r.status = sv->fault != HT_OK ? sv->fault
                   : (fl & kFlagDropped) ? HT_ERR_FULL
                   : (fl & kFlagInvalidKey) ? HT_ERR_INVALID
                                            : HT_OK;
        sv->tabs[r.table].busy = false;
        sv->keys_done += r.n;
        sv->requests_done += 1;
        sv->lat_us.push_back(std::chrono::duration<double, std::micro>(now - r.t0).count());
    }
    sl.reqs.clear();
    sl.busy = false;
    if (--sv->inflight == 0) sv->inflight_s += std::chrono::duration<double>(now - sv->inflight_t0).count();
    sv->finish_s += std::chrono::duration<double>(Clock::now() - now).count();
}

// Packs the head request of every ready table into slot `sl` and issues it.
bool launch(ht_server* sv, Slot& sl) {
    const auto t0 = Clock::now();
    const uint64_t budget = sv->cfg.batch_key_budget;
    uint64_t off = 0, tiles = 0;
    uint32_t nb = 0;
    struct CuckooJob {
        uint32_t table;
        uint64_t off, n;
    };
    std::vector<CuckooJob> cuckoo;
    struct Copy {
        uint64_t off, n;
        const uint64_t* src;          // caller's pinned keys, or null: from the staging buffer
    };
    std::vector<Copy> staged, direct;
    const size_t nt = sv->tabs.size();
    const uint32_t max_reqs = sv->cfg.pack ? sv->cfg.max_requests_per_batch : 1u;
    for (size_t k = 0; k < nt && sl.reqs.size() < max_reqs; ++k) {
        const uint32_t id = uint32_t((sv->rr + k) % nt);
        Tab& tb = sv->tabs[id];
        if (!tb.admitted || tb.busy || tb.q.empty()) continue;
        if (!tb.ready_seen) {
            if (cudaEventQuery(tb.ready) != cudaSuccess) continue;     // still being cleared
            tb.ready_seen = true;
        }
        Req& r = sv->reqs[tb.q.front()];
        if (off + r.n > budget && off > 0) continue;
        if (r.pinned && r.n >= kDirectCopyKeys) {
            direct.push_back(Copy{off, r.n, r.keys});
        } else {
            std::memcpy(sl.h_keys + off, r.keys, r.n * 8);
            if (!staged.empty() && staged.back().off + staged.back().n == off) staged.back().n += r.n;
            else staged.push_back(Copy{off, r.n, nullptr});
        }
        if (tb.scheme == HT_BUCKET) {
            sl.h_desc[nb].keys = sl.d_keys + off;
            sl.h_desc[nb].flags = sl.d_flags + off;
            sl.h_desc[nb].n = r.n;
            sl.h_desc[nb].tile_off = tiles;
            sl.h_desc[nb].table = id;
            sl.h_desc[nb].pad_ = 0;
            tiles += (r.n + 31) / 32;
            ++nb;
        } else {
            cuckoo.push_back(CuckooJob{id, off, r.n});
        }
        sl.h_tid[sl.reqs.size()] = id;
        sl.reqs.emplace_back(tb.q.front(), off);
        r.state = 1;
        tb.q.pop_front();
        tb.busy = true;
        off += r.n;
    }
    if (sl.reqs.empty()) return false;
    sv->rr = (sv->rr + 1) % std::max<size_t>(nt, 1);
    cudaError_t e = cudaEventRecord(sl.ev0, sl.s);
    for (const Copy& c : staged)
        if (e == cudaSuccess)
            e = cudaMemcpyAsync(sl.d_keys + c.off, sl.h_keys + c.off, c.n * 8, cudaMemcpyHostToDevice, sl.s);
    for (const Copy& c : direct)
        if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_keys + c.off, c.src, c.n * 8, cudaMemcpyHostToDevice, sl.s);
    if (e == cudaSuccess && nb) e = cudaMemcpyAsync(sl.d_desc, sl.h_desc, nb * sizeof(WorkDesc), cudaMemcpyHostToDevice, sl.s);
    if (e == cudaSuccess && nb)
        e = packed_bucket_find_or_put(table_bucket_cfg(sv->tabs[sl.h_desc[0].table].t), sv->d_tables, sl.d_desc, nb,
                                      tiles, sl.s);
    for (const auto& c : cuckoo) {
        if (e != cudaSuccess) break;
        if (ht_find_or_put(sv->tabs[c.table].t, sl.d_keys + c.off, c.n, sl.d_flags + c.off, sl.s) != HT_OK)
            e = cudaErrorLaunchFailure;
    }
    const uint32_t nr = uint32_t(sl.reqs.size());
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.d_tid, sl.h_tid, nr * sizeof(uint32_t), cudaMemcpyHostToDevice, sl.s);
    if (e == cudaSuccess) {
        serve_status_kernel<<<(nr + 255) / 256, 256, 0, sl.s>>>(sv->d_tables, sl.d_tid, nr, sl.d_flagw);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_flagw, sl.d_flagw, nr * sizeof(uint32_t), cudaMemcpyDeviceToHost, sl.s);
    if (e == cudaSuccess) e = cudaMemcpyAsync(sl.h_flags, sl.d_flags, off, cudaMemcpyDeviceToHost, sl.s);
    if (e == cudaSuccess) e = cudaEventRecord(sl.ev, sl.s);
    if (e != cudaSuccess) sv->fault = HT_ERR_CUDA;
    sl.busy = true;
    sl.issued = Clock::now();
    if (sv->inflight++ == 0) sv->inflight_t0 = sl.issued;
    sv->batches += 1;
    sv->pack_s += std::chrono::duration<double>(sl.issued - t0).count();
    return true;
}

void close_idle(ht_server* sv) {
    bool freed = false;
    for (auto& tb : sv->tabs) {
        if (!tb.closing || tb.closed || tb.busy || !tb.q.empty()) continue;
        if (tb.t) {
            // Idle: every batch that used it has completed (its event fired).
            table_release(tb.t, sv->admin);
            tb.t = nullptr;
            freed = true;
        }
        if (tb.admitted) sv->admitted_bytes -= tb.bytes;
        tb.admitted = false;
        tb.closed = true;
    }
    (void)freed;   // the freed memory stays in the pool for the next tables (see free_bytes)
}

void worker_loop(ht_server* sv) {
    cudaSetDevice(sv->device);
    std::unique_lock<std::mutex> lk(sv->mu);
    while (!sv->stop) {
        bool progress = false, any_busy = false;
        for (auto& sl : sv->slots) {
            if (sl.busy) {
                const cudaError_t q = cudaEventQuery(sl.ev);
                if (q == cudaSuccess) {
                    finish(sv, sl);
                    progress = true;
                } else if (q != cudaErrorNotReady) {
                    sv->fault = HT_ERR_CUDA;
                    finish(sv, sl);
                    progress = true;
                } else {
                    any_busy = true;
                }
            }
        }
        if (progress) sv->cv_done.notify_all();
        close_idle(sv);
        if (admit(sv)) progress = true;
        for (auto& sl : sv->slots)
            if (!sl.busy && launch(sv, sl)) progress = any_busy = true;
        if (!progress) {
            // Short waits while work is on the device: batches in flight, or
            // admitted tables with requests whose clear is still running.
            for (const auto& tb : sv->tabs) {
                if (any_busy) break;
                any_busy = tb.admitted && !tb.ready_seen && !tb.q.empty();
            }
            if (any_busy) sv->cv_work.wait_for(lk, std::chrono::microseconds(20));
            else sv->cv_work.wait_for(lk, std::chrono::milliseconds(1));
        }
    }
}

void destroy_server(ht_server* sv) {
    {
        std::lock_guard<std::mutex> g(sv->mu);
        sv->stop = true;
    }
    sv->cv_work.notify_all();
    if (sv->worker.joinable()) sv->worker.join();
    cudaSetDevice(sv->device);
    for (auto& sl : sv->slots) {
        if (sl.s) cudaStreamSynchronize(sl.s);
        cudaFreeHost(sl.h_keys);
        cudaFreeHost(sl.h_flags);
        cudaFreeHost(sl.h_desc);
        cudaFreeHost(sl.h_tid);
        cudaFreeHost(sl.h_flagw);
        cudaFree(sl.d_tid);
        cudaFree(sl.d_flagw);
        cudaFree(sl.d_keys);
        cudaFree(sl.d_flags);
        cudaFree(sl.d_desc);
        if (sl.ev) cudaEventDestroy(sl.ev);
        if (sl.ev0) cudaEventDestroy(sl.ev0);
        if (sl.s) cudaStreamDestroy(sl.s);
    }
    for (auto& tb : sv->tabs) {
        if (tb.t) ht_destroy(tb.t);
        if (tb.ready) cudaEventDestroy(tb.ready);
    }
    cudaFree(sv->d_tables);
    cudaFreeHost(sv->h_tables);
    if (sv->admin) cudaStreamDestroy(sv->admin);
    if (sv->pool_kept) {
        cudaMemPool_t pool;
        if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess) {
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &sv->pool_threshold);
            cudaMemPoolTrimTo(pool, 0);
        }
    }
    delete sv;
}

}  // namespace

extern "C" {

ht_status ht_server_default_config(ht_server_config* c) {
    if (!c) return HT_ERR_INVALID;
    std::memset(c, 0, sizeof(*c));
    c->max_inflight = 4;
    c->batch_key_budget = 1ull << 22;
    c->max_requests_per_batch = 4096;
    c->hbm_reserve_bytes = 1ull << 30;
    c->pack = 1;
    ht_default_params(HT_BUCKET, &c->table_params);
    return HT_OK;
}

ht_status ht_server_create(const ht_server_config* cfg, ht_server** out) {
    if (!out) return HT_ERR_INVALID;
    *out = nullptr;
    ht_server_config c;
    ht_server_default_config(&c);
    if (cfg) c = *cfg;
    if (c.max_inflight < 1 || c.max_inflight > 64 || c.batch_key_budget < 32 || c.batch_key_budget > (1ull << 28) ||
        c.max_requests_per_batch < 1 || c.max_requests_per_batch > (1u << 20))
        return HT_ERR_INVALID;
    ht_server* sv = new (std::nothrow) ht_server();
    if (!sv) return HT_ERR_OOM;
    sv->cfg = c;
    cudaGetDevice(&sv->device);
    sv->stats_t0 = Clock::now();
    {
        // Keep memory freed by closed tables in the device's default
        // stream-ordered pool while the server runs: the next tables reuse
        // it without mapping fresh memory (for a 2^30-slot table that cut
        // create + release from ~19 ms to ~1.4 ms).  It goes back to the
        // driver when an allocation fails (trim_pool) and when the server
        // is destroyed, which also restores the previous threshold.
        cudaMemPool_t pool;
        uint64_t keep = ~0ull;
        if (cudaDeviceGetDefaultMemPool(&pool, sv->device) == cudaSuccess &&
            cudaMemPoolGetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &sv->pool_threshold) == cudaSuccess &&
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess)
            sv->pool_kept = true;
    }
    bool ok = cudaStreamCreateWithFlags(&sv->admin, cudaStreamNonBlocking) == cudaSuccess &&
              cudaMalloc(&sv->d_tables, kMaxServerTables * sizeof(DevTable)) == cudaSuccess &&
              cudaMallocHost(&sv->h_tables, kMaxServerTables * sizeof(DevTable)) == cudaSuccess;
    sv->slots.resize(c.max_inflight);
    const uint64_t nreq = c.max_requests_per_batch;
    for (auto& sl : sv->slots) {
        if (!ok) break;
        ok = cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) == cudaSuccess &&
             cudaEventCreate(&sl.ev0) == cudaSuccess && cudaEventCreate(&sl.ev) == cudaSuccess &&
             cudaMallocHost(&sl.h_keys, c.batch_key_budget * 8) == cudaSuccess &&
             cudaMallocHost(&sl.h_flags, c.batch_key_budget) == cudaSuccess &&
             cudaMallocHost(&sl.h_desc, nreq * sizeof(WorkDesc)) == cudaSuccess &&
             cudaMallocHost(&sl.h_tid, nreq * sizeof(uint32_t)) == cudaSuccess &&
             cudaMallocHost(&sl.h_flagw, nreq * sizeof(uint32_t)) == cudaSuccess &&
             cudaMalloc(&sl.d_tid, nreq * sizeof(uint32_t)) == cudaSuccess &&
             cudaMalloc(&sl.d_flagw, nreq * sizeof(uint32_t)) == cudaSuccess &&
             cudaMalloc(&sl.d_keys, c.batch_key_budget * 8) == cudaSuccess &&
             cudaMalloc(&sl.d_flags, c.batch_key_budget) == cudaSuccess &&
             cudaMalloc(&sl.d_desc, nreq * sizeof(WorkDesc)) == cudaSuccess;
    }
    if (!ok) {
        destroy_server(sv);
        return HT_ERR_OOM;
    }
    sv->worker = std::thread(worker_loop, sv);
    *out = sv;
    return HT_OK;
}

ht_status ht_server_destroy(ht_server* sv) {
    if (!sv) return HT_OK;
    destroy_server(sv);
    return HT_OK;
}

ht_status ht_server_open_table(ht_server* sv, uint64_t capacity, ht_scheme scheme, uint32_t* table_id) {
    if (!sv || !table_id || capacity == 0 || capacity > (1ull << 40) || (scheme != HT_BUCKET && scheme != HT_CUCKOO))
        return HT_ERR_INVALID;
    std::lock_guard<std::mutex> g(sv->mu);
    if (sv->tabs.size() >= kMaxServerTables) return HT_ERR_INVALID;
    Tab tb;
    tb.capacity = capacity;
    tb.scheme = scheme;
    tb.bytes = table_bytes(capacity, scheme, sv->cfg.table_params);
    sv->tabs.push_back(tb);
    *table_id = uint32_t(sv->tabs.size() - 1);
    sv->cv_work.notify_all();
    return HT_OK;
}

ht_status ht_server_close_table(ht_server* sv, uint32_t table_id) {
    if (!sv) return HT_ERR_INVALID;
    std::lock_guard<std::mutex> g(sv->mu);
    if (table_id >= sv->tabs.size() || sv->tabs[table_id].closing) return HT_ERR_INVALID;
    sv->tabs[table_id].closing = true;
    sv->cv_work.notify_all();
    return HT_OK;
}

ht_status ht_server_table_state(ht_server* sv, uint32_t table_id, int32_t* admitted, uint64_t* size) {
    if (!sv) return HT_ERR_INVALID;
    std::lock_guard<std::mutex> g(sv->mu);
    if (table_id >= sv->tabs.size()) return HT_ERR_INVALID;
    Tab& tb = sv->tabs[table_id];
    if (admitted) *admitted = tb.admitted ? 1 : (tb.closed ? -1 : 0);
    if (size) {
        *size = 0;
        if (tb.t && !tb.busy) {
            // The table is idle; its clear (on the admission stream) may still run.
            if (!tb.ready_seen && cudaEventSynchronize(tb.ready) != cudaSuccess) return HT_ERR_CUDA;
            DevCounters c;
            if (cudaMemcpy(&c, table_dev(tb.t).ctr, sizeof(c), cudaMemcpyDeviceToHost) != cudaSuccess) return HT_ERR_CUDA;
            *size = c.size;
        }
    }
    return HT_OK;
}

ht_status ht_server_submit(ht_server* sv, uint32_t table_id, const uint64_t* h_keys, uint64_t n, uint8_t* h_is_new,
                           uint64_t* request_id) {
    if (!sv || !request_id || (n && !h_keys) || n > sv->cfg.batch_key_budget) return HT_ERR_INVALID;
    std::lock_guard<std::mutex> g(sv->mu);
    if (table_id >= sv->tabs.size() || sv->tabs[table_id].closing || sv->tabs[table_id].closed) return HT_ERR_INVALID;
    const uint64_t id = sv->next_id++;
    Req& r = sv->reqs[id];
    r.table = table_id;
    r.keys = h_keys;
    r.n = n;
    r.out = h_is_new;
    if (n >= kDirectCopyKeys) {
        cudaPointerAttributes a;
        if (cudaPointerGetAttributes(&a, h_keys) == cudaSuccess) r.pinned = a.type == cudaMemoryTypeHost;
        else cudaGetLastError();
    }
    r.t0 = Clock::now();
    sv->tabs[table_id].q.push_back(id);
    *request_id = id;
    sv->cv_work.notify_all();
    return HT_OK;
}

ht_status ht_server_wait(ht_server* sv, uint64_t request_id, uint32_t timeout_ms, double* latency_us) {
    if (!sv) return HT_ERR_INVALID;
    std::unique_lock<std::mutex> lk(sv->mu);
    auto it = sv->reqs.find(request_id);
    if (it == sv->reqs.end()) return HT_ERR_INVALID;
    const bool done = sv->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] {
        auto jt = sv->reqs.find(request_id);
        return jt == sv->reqs.end() || jt->second.state == 2;
    });
    if (!done) return HT_ERR_TIMEOUT;
    it = sv->reqs.find(request_id);
    const ht_status st = it->second.status;
    if (latency_us) *latency_us = std::chrono::duration<double, std::micro>(it->second.t1 - it->second.t0).count();
    sv->reqs.erase(it);
    return st;
}

ht_status ht_server_get_stats(ht_server* sv, ht_server_stats* out, int reset) {
    if (!sv || !out) return HT_ERR_INVALID;
    std::lock_guard<std::mutex> g(sv->mu);
    std::memset(out, 0, sizeof(*out));
    out->requests = sv->requests_done;
    out->keys = sv->keys_done;
    out->batches = sv->batches;
    out->seconds = std::chrono::duration<double>(Clock::now() - sv->stats_t0).count();
    std::vector<double> v = sv->lat_us;
    if (!v.empty()) {
        std::sort(v.begin(), v.end());
        auto pct = [&](double q) { return v[std::min<size_t>(v.size() - 1, size_t(q * (v.size() - 1) + 0.5))]; };
        out->p50_us = pct(0.50);
        out->p99_us = pct(0.99);
        out->max_us = v.back();
        double s = 0;
        for (double x : v) s += x;
        out->mean_us = s / double(v.size());
    }
    uint32_t adm = 0;
    for (const auto& tb : sv->tabs) adm += tb.admitted;
    out->tables_admitted = adm;
    out->admitted_bytes = sv->admitted_bytes;
    out->status = sv->fault;
    out->admit_seconds = sv->admit_s;
    out->pack_seconds = sv->pack_s;
    out->finish_seconds = sv->finish_s;
    out->batch_us_mean = sv->batches ? sv->batch_us / double(sv->batches) : 0.0;
    out->batch_gpu_us_mean = sv->batches ? sv->batch_gpu_us / double(sv->batches) : 0.0;
    out->tables_created = sv->tables_created;
    out->inflight_seconds = sv->inflight_s;
    out->table_bytes_created = sv->table_bytes;
    if (reset) {
        sv->lat_us.clear();
        sv->admit_s = sv->pack_s = sv->finish_s = sv->batch_us = sv->batch_gpu_us = sv->inflight_s = 0;
        sv->tables_created = 0;
        sv->table_bytes = 0;
        sv->requests_done = sv->keys_done = sv->batches = 0;
        sv->stats_t0 = Clock::now();
    }
    return HT_OK;
}

}  // extern "C"
