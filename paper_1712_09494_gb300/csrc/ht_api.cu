// Host side of the C ABI: table lifecycle, batching, rebuild and status.
#include <algorithm>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include "ht_internal.cuh"

using namespace ht;

struct ht_table {
    int device;
    ht_scheme scheme;
    uint32_t kw;
    ht_params p;
    DevTable dt;
    DevScratch sc;
    uint64_t chunk;              // Cuckoo keys per probe/insert launch pair
    uint32_t parity;
    uint32_t rebuilds;
    bool rebuild_exhausted;
    ht_status sticky;            // HT_ERR_FULL once a key was dropped
    uint64_t seed_base;
    L2Window win;                // l2_persist: the slots (or the Cuckoo claim set)
};

namespace {

constexpr uint64_t kMaxCapacity = 1ull << 40;

uint64_t next_pow2(uint64_t x) {
    uint64_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

void derive_seeds(ht_table* t) {
    for (int a = 0; a < kMaxHashes; ++a) t->dt.seed[a] = mix64(t->seed_base + uint64_t(a + 1) * 0x9E3779B97F4A7C15ull);
    t->dt.aux_seed = mix64(t->seed_base ^ 0xD1B54A32D192ED03ull);
}

bool is_long(uint32_t kw) { return kw > 128; }

BucketCfg bucket_cfg(const ht_table* t) {
    return BucketCfg{int(t->kw), int(t->p.bucket_slots), int(t->p.lanes_per_key)};
}

cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }

ht_status cuda_status(cudaError_t e) {
    if (e == cudaSuccess) return HT_OK;
    if (e == cudaErrorMemoryAllocation) return HT_ERR_OOM;
    return HT_ERR_CUDA;
}

#define HT_TRY(expr)                                 \
    do {                                             \
        cudaError_t e_ = (expr);                     \
        if (e_ != cudaSuccess) return cuda_status(e_); \
    } while (0)

struct DeviceGuard {
    int prev = -1;
    explicit DeviceGuard(int dev) {
        cudaGetDevice(&prev);
        if (prev != dev) cudaSetDevice(dev);
        else prev = -1;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};

ht_status clear_table(ht_table* t, cudaStream_t s) {
    // Words per slot: 2 for 128-bit keys and long-key Cuckoo entries.
    const uint64_t w = (t->kw == 128 || (is_long(t->kw) && t->scheme == HT_CUCKOO)) ? 2 : 1;
    const uint64_t wo = t->kw >= 128 ? 2 : 1;    // words per overflow entry
    HT_TRY(fill_words(t->dt.slots, t->dt.nslots * w, kEmpty, s));
    HT_TRY(fill_words(t->dt.stash, t->dt.stash_slots, kEmpty, s));
    HT_TRY(fill_words(t->dt.ovf, t->dt.ovf_slots * wo, kEmpty, s));
    HT_TRY(cudaMemsetAsync(t->dt.ctr, 0, sizeof(DevCounters), s));
    return HT_OK;
}

// Every stored key (and value) to the caller's buffers, any key width.
cudaError_t export_any(ht_table* t, void* keys, uint32_t* vals, unsigned long long* cnt, uint64_t cap,
                       cudaStream_t s) {
    if (t->kw == 128) return wide_export(t->dt, keys, cnt, cap, s);
    if (is_long(t->kw)) return long_export(t->dt, t->scheme == HT_CUCKOO, keys, cnt, cap, s);
    return table_export(int(t->kw), t->dt, keys, vals, cnt, cap, s);
}

// Runs find-or-put / insert over a batch without touching rebuild state.
ht_status run_put(ht_table* t, const void* keys, const uint32_t* vals, uint64_t n, uint8_t* is_new,
                  void* new_out, unsigned long long* new_count, cudaStream_t s,
                  const unsigned long long* d_n = nullptr, uint64_t new_cap = ~0ull) {
    if (n == 0) return HT_OK;
    if (is_long(t->kw)) {
        if (vals || new_out || d_n) return HT_ERR_INVALID;
        if (t->scheme == HT_BUCKET) return cuda_status(long_find_or_put(t->dt, keys, n, is_new, s));
        const size_t ksz = t->kw / 8;
        for (uint64_t off = 0; off < n; off += t->chunk) {
            const uint64_t m = std::min(t->chunk, n - off);
            HT_TRY(long_cuckoo_probe(t->dt, t->sc, t->parity, static_cast<const char*>(keys) + off * ksz, m,
                                     is_new ? is_new + off : nullptr, s));
            HT_TRY(long_cuckoo_insert(t->dt, t->sc, t->parity, std::min<uint64_t>(m, t->sc.win_cap), s));
            t->parity ^= 1u;
        }
        return HT_OK;
    }
    if (t->kw == 128) {
        if (vals) return HT_ERR_INVALID;
        if (t->scheme == HT_BUCKET)
            return cuda_status(wide_find_or_put(int(t->p.lanes_per_key), t->dt, keys, n, d_n, is_new, new_out,
                                                new_count, new_cap, s));
        for (uint64_t off = 0; off < n; off += t->chunk) {
            const uint64_t m = std::min(t->chunk, n - off);
            HT_TRY(wide_cuckoo_probe(t->dt, t->sc, t->parity, static_cast<const char*>(keys) + off * 16, m, d_n, off,
                                     is_new ? is_new + off : nullptr, s, new_out != nullptr));
            HT_TRY(wide_cuckoo_insert(t->dt, t->sc, t->parity, new_out, new_count, new_cap,
                                      std::min<uint64_t>(m, t->sc.win_cap), s));
            t->parity ^= 1u;
        }
        return HT_OK;
    }
    if (t->scheme == HT_BUCKET) {
        return cuda_status(bucket_find_or_put(bucket_cfg(t), t->dt, keys, vals, n, d_n, is_new, new_out,
                                              new_count, new_cap, s, t->win));
    }
    const size_t ksz = t->kw / 8;
    for (uint64_t off = 0; off < n; off += t->chunk) {
        const uint64_t m = std::min(t->chunk, n - off);
        const void* k = static_cast<const char*>(keys) + off * ksz;
        HT_TRY(cuckoo_probe(int(t->kw), t->dt, t->sc, t->parity, k, vals ? vals + off : nullptr, m, d_n,
                            off, is_new ? is_new + off : nullptr, s, t->win, new_out != nullptr));
        HT_TRY(cuckoo_insert(int(t->kw), t->dt, t->sc, t->parity, new_out, new_count, new_cap,
                             std::min<uint64_t>(m, t->sc.win_cap), s, t->win));
        t->parity ^= 1u;
    }
    return HT_OK;
}

ht_status read_counters(ht_table* t, DevCounters* c, cudaStream_t s) {
    HT_TRY(cudaMemcpyAsync(c, t->dt.ctr, sizeof(DevCounters), cudaMemcpyDeviceToHost, s));
    HT_TRY(cudaStreamSynchronize(s));
    return HT_OK;
}

// Section 4.1: when the stash is full and an insertion fails, rebuild the
// table with new hash constants.  All stored words (table, stash, overflow
// set) are copied out, the table is cleared, the constants are re-drawn and
// the words are inserted again; repeated up to max_rebuilds times.
ht_status rebuild(ht_table* t, cudaStream_t s) {
    DevCounters c;
    ht_status st = read_counters(t, &c, s);
    if (st != HT_OK) return st;
    const uint64_t n = c.size;
    void* keys = nullptr;
    uint32_t* vals = nullptr;
    unsigned long long* cnt = nullptr;
    HT_TRY(cudaMalloc(&keys, std::max<uint64_t>(n, 1) * (t->kw / 8)));
    if (t->kw == 32 && cudaMalloc(&vals, std::max<uint64_t>(n, 1) * 4) != cudaSuccess) {
        cudaFree(keys);
        return HT_ERR_OOM;
    }
    if (cudaMalloc(&cnt, sizeof(unsigned long long)) != cudaSuccess) {
        cudaFree(keys);
        cudaFree(vals);
        return HT_ERR_OOM;
    }
    st = HT_OK;
    do {
        if (cudaMemsetAsync(cnt, 0, sizeof(*cnt), s) != cudaSuccess ||
            export_any(t, keys, vals, cnt, n, s) != cudaSuccess) {
            st = HT_ERR_CUDA;
            break;
        }
        unsigned long long got = 0;
        if (cudaMemcpyAsync(&got, cnt, sizeof(got), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = HT_ERR_CUDA;
            break;
        }
        const unsigned long long dropped = c.dropped;
        const uint32_t keep_flags = c.flags & (kFlagDropped | kFlagInvalidKey);
        bool ok = false;
        for (uint32_t attempt = 0; attempt < t->p.max_rebuilds; ++attempt) {
            t->rebuilds += 1;
            t->seed_base = mix64(t->seed_base + 0x9E3779B97F4A7C15ull * t->rebuilds);
            derive_seeds(t);
            if ((st = clear_table(t, s)) != HT_OK) break;
            if ((st = run_put(t, keys, vals, got, nullptr, nullptr, nullptr, s)) != HT_OK) break;
            if ((st = read_counters(t, &c, s)) != HT_OK) break;
            if (!(c.flags & (kFlagRebuild | kFlagDropped))) {
                ok = true;
                break;
            }
        }
        if (st != HT_OK) break;
        if (!ok) {
            // Keep the last attempt only if it lost nothing; otherwise the
            // table is over-full for its capacity.
            if (c.flags & kFlagDropped) t->sticky = HT_ERR_FULL;
            t->rebuild_exhausted = true;
        }
        // Carry the sticky facts of the old table over.
        if (dropped || keep_flags) {
            DevCounters nc = c;
            nc.dropped += dropped;
            nc.flags |= keep_flags;
            cudaMemcpyAsync(t->dt.ctr, &nc, sizeof(nc), cudaMemcpyHostToDevice, s);
            cudaStreamSynchronize(s);
        }
    } while (false);
    cudaFree(keys);
    cudaFree(vals);
    cudaFree(cnt);
    return st;
}

ht_status grow_to(ht_table* t, uint64_t new_capacity, cudaStream_t s);

ht_status sync_and_status(ht_table* t, cudaStream_t s) {
    DevCounters c;
    ht_status st = read_counters(t, &c, s);
    if (st != HT_OK) return st;
    if (t->p.grow_load_permille && !(c.flags & kFlagDropped)) {
        // Growth instead of rebuilds: double while above the load or while
        // keys sit in the overflow set (bounded: capacity doubles each time).
        while ((c.size * 1000 > t->dt.nslots * uint64_t(t->p.grow_load_permille) || (c.flags & kFlagRebuild)) &&
               t->dt.nslots * 2 <= kMaxCapacity) {
            st = grow_to(t, t->dt.nslots * 2, s);
            if (st != HT_OK) return st;
            st = read_counters(t, &c, s);
            if (st != HT_OK) return st;
        }
    }
    if ((c.flags & kFlagRebuild) && !t->rebuild_exhausted) {
        st = rebuild(t, s);
        if (st != HT_OK) return st;
        st = read_counters(t, &c, s);
        if (st != HT_OK) return st;
    }
    if (c.flags & kFlagDropped) t->sticky = HT_ERR_FULL;
    if (c.flags & kFlagTimeout) t->sticky = HT_ERR_TIMEOUT;
    if (c.flags & kFlagInvalidKey) {
        // Reported once, then cleared.
        unsigned int f = c.flags & ~kFlagInvalidKey;
        HT_TRY(cudaMemcpyAsync(&t->dt.ctr->flags, &f, sizeof(f), cudaMemcpyHostToDevice, s));
        HT_TRY(cudaStreamSynchronize(s));
        return t->sticky != HT_OK ? t->sticky : HT_ERR_INVALID;
    }
    return t->sticky;
}

bool valid_params(ht_scheme scheme, const ht_params& p) {
    if (p.grow_load_permille != 0 && (p.grow_load_permille < 100 || p.grow_load_permille > 1000)) return false;
    if (scheme == HT_BUCKET) {
        if (p.num_hashes < 1 || p.num_hashes > uint32_t(kMaxHashes)) return false;
        if (p.bucket_slots != 8 && p.bucket_slots != 16 && p.bucket_slots != 32) return false;
        const uint32_t g = p.lanes_per_key;
        // (bucket_slots, lanes) pairs the bucket kernels are instantiated for.
        static const uint32_t kShapes[][2] = {{8, 2}, {8, 4}, {8, 8}, {16, 2}, {16, 4}, {16, 8},
                                              {16, 16}, {32, 4}, {32, 8}, {32, 16}, {32, 32}};
        bool shape_ok = false;
        for (const auto& sh : kShapes) shape_ok |= sh[0] == p.bucket_slots && sh[1] == g;
        if (!shape_ok) return false;
    } else {
        if (p.num_hashes < 2 || p.num_hashes > uint32_t(kMaxCuckooHashes)) return false;
        if (p.max_evictions < 1 || p.max_evictions > 4096) return false;
        if (p.bucket_slots != 8 && p.bucket_slots != 16 && p.bucket_slots != 32) return false;
    }
    if (p.cuckoo_chain_h1 > 1) return false;
    if (p.stash_slots > 4096) return false;
    if (p.max_batch < 1 || p.max_batch > (1ull << 26)) return false;
    if (p.max_rebuilds > 64) return false;
    return true;
}

ht_params complete_params(ht_scheme scheme, const ht_params* in) {
    ht_params d;
    ht_default_params(scheme, &d);
    if (!in) return d;
    ht_params p = *in;
    if (!p.num_hashes) p.num_hashes = d.num_hashes;
    if (!p.max_evictions) p.max_evictions = d.max_evictions;
    if (!p.stash_slots) p.stash_slots = d.stash_slots;
    if (!p.bucket_slots) p.bucket_slots = d.bucket_slots;
    if (!p.lanes_per_key) p.lanes_per_key = 2;
    if (!p.max_rebuilds) p.max_rebuilds = d.max_rebuilds;
    if (!p.max_batch) p.max_batch = d.max_batch;
    return p;
}

// Tables holding an L2 access-policy window, per device, and the context's
// persisting set-aside before the first of them raised it.  When the last
// one is freed the set-aside goes back to that value and persisting lines
// turn normal: a set-aside left behind would shrink the L2 of all later work
// in the process (a 128-bit bucket fill took 9.0 instead of 5.4 ms after a
// Cuckoo table with a window had come and gone).
std::mutex g_win_mu;
int g_win_tables[64];
size_t g_win_prev[64];

void window_acquire(int dev, size_t before) {
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> g(g_win_mu);
    if (g_win_tables[dev]++ == 0) g_win_prev[dev] = before;
}

void window_release(int dev) {
    if (dev < 0 || dev >= 64) return;
    std::lock_guard<std::mutex> g(g_win_mu);
    if (g_win_tables[dev] > 0 && --g_win_tables[dev] == 0) {
        cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, g_win_prev[dev]);
        cudaCtxResetPersistingL2Cache();
    }
}

// Table memory is stream-ordered (cudaMallocAsync / cudaFreeAsync), so a
// table can be released without synchronising the whole device.
void free_table(ht_table* t, cudaStream_t s) {
    if (!t) return;
    if (t->win.base) window_release(t->device);
    void* ptrs[] = {t->dt.slots, t->dt.stash, t->dt.ovf, t->dt.ctr, t->sc.set, t->sc.win, t->dt.kstore};
    for (void* p : ptrs)
        if (p) cudaFreeAsync(p, s);
    delete t;
}

}  // namespace

namespace {

// Copies every stored word out, inserts them into new storage of
// new_capacity slots with the current hash constants, and swaps the storage
// in; on any failure the table is left as it was.
ht_status grow_to(ht_table* t, uint64_t new_capacity, cudaStream_t s) {
    DevCounters c;
    ht_status st = read_counters(t, &c, s);
    if (st != HT_OK) return st;
    ht_params p = t->p;
    p.seed = t->seed_base;                // the constants in use (after any rebuild)
    ht_table* nt = nullptr;
    st = ht_create(new_capacity, t->scheme, t->kw, &p, s, &nt);
    if (st != HT_OK) return st;
    const uint64_t n = c.size;
    void* keys = nullptr;
    uint32_t* vals = nullptr;
    unsigned long long* cnt = nullptr;
    cudaError_t e = cudaMalloc(&keys, std::max<uint64_t>(n, 1) * (t->kw / 8));
    if (e == cudaSuccess && t->kw == 32) e = cudaMalloc(&vals, std::max<uint64_t>(n, 1) * 4);   // 32-bit maps
    if (e == cudaSuccess) e = cudaMalloc(&cnt, sizeof(*cnt));
    if (e == cudaSuccess) e = cudaMemsetAsync(cnt, 0, sizeof(*cnt), s);
    if (e == cudaSuccess) e = export_any(t, keys, vals, cnt, n, s);
    unsigned long long got = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&got, cnt, sizeof(got), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    st = cuda_status(e);
    if (st == HT_OK) st = run_put(nt, keys, vals, std::min<uint64_t>(got, n), nullptr, nullptr, nullptr, s);
    if (st == HT_OK) {
        nt->p.grow_load_permille = 0;     // the new storage must hold them as it is
        st = sync_and_status(nt, s);
        nt->p.grow_load_permille = t->p.grow_load_permille;
    }
    cudaFree(keys);
    cudaFree(vals);
    cudaFree(cnt);
    if (st != HT_OK) {
        cudaStreamSynchronize(s);
        free_table(nt, s);
        return st == HT_ERR_INVALID ? HT_ERR_FULL : st;
    }
    // Carry the sticky facts over (dropped keys stay counted), then swap.
    if (c.dropped || (c.flags & (kFlagDropped | kFlagInvalidKey))) {
        DevCounters nc;
        if ((st = read_counters(nt, &nc, s)) == HT_OK) {
            nc.dropped += c.dropped;
            nc.flags |= c.flags & (kFlagDropped | kFlagInvalidKey);
            cudaMemcpyAsync(nt->dt.ctr, &nc, sizeof(nc), cudaMemcpyHostToDevice, s);
        }
    }
    std::swap(t->dt, nt->dt);
    std::swap(t->sc, nt->sc);
    std::swap(t->chunk, nt->chunk);
    std::swap(t->parity, nt->parity);
    std::swap(t->win, nt->win);
    t->rebuild_exhausted = false;
    cudaStreamSynchronize(s);
    free_table(nt, s);                    // the old storage
    return HT_OK;
}

// Bucket-scheme items of one ht_multi_find_or_put call that share a key
// width and bucket shape (one packed launch).
struct PackGroup {
    BucketCfg cfg;
    std::vector<DevTable> tabs;
    std::vector<uint32_t> slot_of;   // table index -> position in tabs (or ~0)
    std::vector<WorkDesc> items;
    uint64_t tiles = 0;
};

}  // namespace

extern "C" {

const char* ht_status_str(ht_status s) {
    switch (s) {
        case HT_OK: return "ok";
        case HT_ERR_INVALID: return "invalid argument or reserved key";
        case HT_ERR_OOM: return "device allocation failed";
        case HT_ERR_FULL: return "table full: keys could not be placed";
        case HT_ERR_CUDA: return "CUDA error";
        case HT_ERR_TIMEOUT: return "bounded device wait timed out";
    }
    return "unknown status";
}

ht_status ht_default_params(ht_scheme scheme, ht_params* p) {
    if (!p || (scheme != HT_BUCKET && scheme != HT_CUCKOO)) return HT_ERR_INVALID;
    std::memset(p, 0, sizeof(*p));
    p->num_hashes = scheme == HT_BUCKET ? 16 : 4;
    p->max_evictions = 256;
    p->stash_slots = 101;
    p->bucket_slots = 16;
    p->lanes_per_key = 2;
    p->max_rebuilds = 8;
    // Cuckoo: 2^22 keys per launch pair.  Each insert launch ends with its
    // longest eviction chain, so fewer, larger launches pay fewer tails (a
    // BFS of 10^8 states: insert 41.7 -> 24.1 ms); 2^23 keys would put the
    // claim set past the persisting L2 (fill of 2^27 keys: 15.9 ms at 2^22,
    // 16.5 at 2^21, 24.5 at 2^23).
    p->max_batch = 1ull << 22;
    p->seed = 0x243F6A8885A308D3ull;
    // Off by default for both schemes.  Most new Cuckoo keys no longer claim
    // in the dedup set, and the persisting set-aside a window raises stays
    // reserved for the context after the table is gone: with it on, the
    // Cuckoo fill of 2^27 keys took 15.9 instead of 14.8 ms, and a later
    // 128-bit bucket fill 9.0 instead of 5.4 ms.
    p->l2_persist = 0;
    return HT_OK;
}

ht_status ht_create(uint64_t capacity, ht_scheme scheme, uint32_t key_width, const ht_params* params,
                    void* stream, ht_table** out) {
    if (!out) return HT_ERR_INVALID;
    *out = nullptr;
    if (capacity == 0 || capacity > kMaxCapacity) return HT_ERR_INVALID;
    if (scheme != HT_BUCKET && scheme != HT_CUCKOO) return HT_ERR_INVALID;
    const bool long_keys = is_long(key_width) && key_width % 64 == 0 && key_width / 64 >= kLongMinWords &&
                           key_width / 64 <= kLongMaxWords;
    if (key_width != 32 && key_width != 64 && key_width != 128 && !long_keys) return HT_ERR_INVALID;
    ht_params p = complete_params(scheme, params);
    if (p.digest_bits > 64 || (p.digest_bits && !long_keys)) return HT_ERR_INVALID;
    if (long_keys) {
        // Bucket scheme: 16 header words per bucket, one thread per key
        // (lanes_per_key unused).  Cuckoo: 16-byte entries, no stash.
        if (scheme == HT_BUCKET) {
            if (!params || !params->bucket_slots) p.bucket_slots = kLongBucketSlots;
            if (p.bucket_slots != kLongBucketSlots) return HT_ERR_INVALID;
        }
        p.stash_slots = 0;
    }
    if (key_width == 128) {
        // 16-byte slots; no stash (the overflow set takes what does not fit).
        // Bucket scheme: buckets of 8 (one 128-byte line), 2 or 4 lanes.
        if (!params) p.bucket_slots = 8;      // lanes_per_key stays 2 (measured faster than 4)
        if (scheme == HT_BUCKET && (p.bucket_slots != 8 || (p.lanes_per_key != 2 && p.lanes_per_key != 4)))
            return HT_ERR_INVALID;
        p.stash_slots = 0;
    }
    if (!valid_params(scheme, p)) return HT_ERR_INVALID;

    ht_table* t = new (std::nothrow) ht_table();
    if (!t) return HT_ERR_OOM;
    std::memset(&t->dt, 0, sizeof(t->dt));
    std::memset(&t->sc, 0, sizeof(t->sc));
    t->scheme = scheme;
    t->kw = key_width;
    t->p = p;
    t->sticky = HT_OK;
    t->seed_base = p.seed;
    if (cudaGetDevice(&t->device) != cudaSuccess) {
        delete t;
        return HT_ERR_CUDA;
    }
    const uint64_t bs = p.bucket_slots;
    t->dt.nslots = (capacity + bs - 1) / bs * bs;             // whole buckets for both schemes
    t->dt.nbuckets = t->dt.nslots / bs;
    t->dt.stash_slots = p.stash_slots;
    t->dt.ovf_slots = uint32_t(std::min<uint64_t>(kOvfSlots, std::max<uint64_t>(1024, next_pow2(t->dt.nslots / 64))));
    t->dt.k = p.num_hashes;
    t->dt.max_evict = p.max_evictions;
    t->dt.chain_h1 = p.cuckoo_chain_h1;
    t->dt.spin_limit = p.publish_wait_polls ? p.publish_wait_polls : kDefaultSpinLimit;
    derive_seeds(t);

    const cudaStream_t cs = as_stream(stream);
    auto fail = [&](cudaError_t e) {
        free_table(t, cs);
        return cuda_status(e);
    };
    cudaError_t e;
    const uint64_t slot_bytes = (key_width == 128 || (long_keys && scheme == HT_CUCKOO)) ? 16 : 8;
    const uint64_t ovf_bytes = key_width >= 128 ? 16 : 8;
    if ((e = cudaMallocAsync(&t->dt.slots, t->dt.nslots * slot_bytes, cs)) != cudaSuccess) return fail(e);
    if ((e = cudaMallocAsync(&t->dt.stash, std::max<uint32_t>(t->dt.stash_slots, 1) * 8, cs)) != cudaSuccess) return fail(e);
    if ((e = cudaMallocAsync(&t->dt.ovf, uint64_t(t->dt.ovf_slots) * ovf_bytes, cs)) != cudaSuccess) return fail(e);
    t->dt.digest_mask = p.digest_bits == 0 || p.digest_bits == 64 ? ~0ull : (1ull << p.digest_bits) - 1;
    if (long_keys) {
        // Key store: one row per slot (bucket scheme), or one per key the
        // table, its overflow set included, can hold (Cuckoo).
        t->dt.words = key_width / 64;
        t->dt.row_words = (t->dt.words + 1) & ~1u;
        t->dt.kstore_rows = t->dt.nslots + (scheme == HT_CUCKOO ? t->dt.ovf_slots : 0);
        if ((e = cudaMallocAsync(&t->dt.kstore, t->dt.kstore_rows * t->dt.row_words * 8, cs)) != cudaSuccess)
            return fail(e);
    }
    if ((e = cudaMallocAsync(&t->dt.ctr, sizeof(DevCounters), cs)) != cudaSuccess) return fail(e);
    if (scheme == HT_CUCKOO) {
        // Keys per probe/insert launch pair: max_batch.  Unless the table
        // overflows, a chunk's distinct absent keys (its winners) are no more
        // than the table can hold, so the dedup set (twice that, for short
        // probe runs) and the winner list are sized by the smaller of the
        // two; a chunk that exceeds them would overflow the table anyway and
        // reports its keys as dropped.
        t->chunk = p.max_batch;
        const uint64_t sc_cap =
            std::min<uint64_t>(p.max_batch, next_pow2(t->dt.nslots + t->dt.stash_slots + t->dt.ovf_slots));
        const uint64_t sslots = next_pow2(2 * sc_cap);
        t->sc.mask = sslots - 1;
        t->sc.win_cap = sc_cap;
        const uint64_t set_words = key_width >= 128 ? 2 : 1;
        const uint64_t win_bytes = key_width >= 128 ? kWideWinnerBytes : sizeof(Winner);
        if ((e = cudaMallocAsync(&t->sc.set, sslots * 8 * set_words, cs)) != cudaSuccess) return fail(e);
        if ((e = cudaMallocAsync(&t->sc.win, sc_cap * win_bytes, cs)) != cudaSuccess) return fail(e);
        if ((e = fill_words(t->sc.set, sslots * set_words, kEmpty, cs)) != cudaSuccess) return fail(e);
    }
    ht_status st = clear_table(t, cs);
    if (st != HT_OK) {
        free_table(t, cs);
        return st;
    }
    if (p.l2_persist) {
        // The slot array when it fits the device's persisting L2, else (Cuckoo)
        // the dedup claim set, which every absent key of a batch touches.
        int dev = 0, max_persist = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev);
        const size_t table_bytes = t->dt.nslots * slot_bytes;
        size_t before = 0;
        cudaDeviceGetLimit(&before, cudaLimitPersistingL2CacheSize);
        if (table_bytes <= size_t(max_persist)) t->win = l2_window(t->dt.slots, table_bytes);
        else if (scheme == HT_CUCKOO) t->win = l2_window(t->sc.set, (t->sc.mask + 1) * (key_width >= 128 ? 16 : 8));
        if (t->win.base) window_acquire(dev, before);
    }
    *out = t;
    return HT_OK;
}

ht_status ht_destroy(ht_table* t) {
    if (!t) return HT_OK;
    DeviceGuard g(t->device);
    cudaDeviceSynchronize();          // the table may have been used on any stream
    free_table(t, nullptr);
    cudaStreamSynchronize(nullptr);
    return HT_OK;
}

static ht_status put_common(ht_table* t, const void* keys, const uint32_t* vals, uint64_t n,
                            uint8_t* is_new, void* new_out, unsigned long long* new_count, void* stream) {
    if (!t) return HT_ERR_INVALID;
    if (n && !keys) return HT_ERR_INVALID;
    if (vals && t->kw != 32) return HT_ERR_INVALID;
    if ((new_out == nullptr) != (new_count == nullptr)) return HT_ERR_INVALID;
    if (is_long(t->kw) && (new_out || (reinterpret_cast<uintptr_t>(keys) & 7))) return HT_ERR_INVALID;
    DeviceGuard g(t->device);
    return run_put(t, keys, vals, n, is_new, new_out, new_count, as_stream(stream));
}

ht_status ht_find_or_put(ht_table* t, const void* d_keys, uint64_t n, uint8_t* d_is_new, void* stream) {
    return put_common(t, d_keys, nullptr, n, d_is_new, nullptr, nullptr, stream);
}

ht_status ht_find_or_put_append(ht_table* t, const void* d_keys, uint64_t n, uint8_t* d_is_new,
                                void* d_new_keys, unsigned long long* d_new_count, void* stream) {
    if (!d_new_keys || !d_new_count) return HT_ERR_INVALID;
    return put_common(t, d_keys, nullptr, n, d_is_new, d_new_keys, d_new_count, stream);
}

ht_status ht_insert(ht_table* t, const void* d_keys, const uint32_t* d_values, uint64_t n, void* stream) {
    return put_common(t, d_keys, d_values, n, nullptr, nullptr, nullptr, stream);
}

ht_status ht_lookup(ht_table* t, const void* d_keys, uint64_t n, uint32_t* d_values, uint8_t* d_found,
                    void* stream) {
    if (!t || (n && !d_keys)) return HT_ERR_INVALID;
    if (n == 0) return HT_OK;
    DeviceGuard g(t->device);
    const cudaStream_t s = as_stream(stream);
    if (is_long(t->kw)) {
        if (d_values || (reinterpret_cast<uintptr_t>(d_keys) & 7)) return HT_ERR_INVALID;
        if (t->scheme == HT_CUCKOO) return cuda_status(long_cuckoo_lookup(t->dt, d_keys, n, d_found, s));
        return cuda_status(long_lookup(t->dt, d_keys, n, d_found, s));
    }
    if (t->kw == 128) {
        if (d_values) return HT_ERR_INVALID;
        if (t->scheme == HT_CUCKOO) return cuda_status(wide_cuckoo_lookup(t->dt, d_keys, n, d_found, s));
        return cuda_status(wide_lookup(int(t->p.lanes_per_key), t->dt, d_keys, n, d_found, s));
    }
    if (t->scheme == HT_BUCKET)
        return cuda_status(bucket_lookup(bucket_cfg(t), t->dt, d_keys, n, d_values, d_found, s, t->win));
    return cuda_status(cuckoo_lookup(int(t->kw), t->dt, d_keys, n, d_values, d_found, s, t->win));
}

ht_status ht_multi_find_or_put(ht_table* const* tables, uint32_t ntables, const ht_work* list, uint32_t m,
                               void* stream) {
    if (m && (!tables || !list)) return HT_ERR_INVALID;
    for (uint32_t i = 0; i < m; ++i) {
        if (list[i].table >= ntables || !tables[list[i].table] || tables[list[i].table]->kw >= 128)
            return HT_ERR_INVALID;
        if (list[i].n && !list[i].d_keys) return HT_ERR_INVALID;
    }
    if (!m) return HT_OK;
    DeviceGuard g(tables[list[0].table]->device);
    const cudaStream_t s = as_stream(stream);
    // Bucket items, grouped by key width and bucket shape: one packed launch
    // per group.  A group's tables and items go to the device in one
    // stream-ordered scratch block.
    std::vector<PackGroup> groups;
    for (uint32_t i = 0; i < m; ++i) {
        const ht_work& w = list[i];
        ht_table* t = tables[w.table];
        if (t->scheme != HT_BUCKET || w.n == 0) continue;
        const BucketCfg c = bucket_cfg(t);
        PackGroup* gp = nullptr;
        for (auto& gr : groups)
            if (gr.cfg.kw == c.kw && gr.cfg.bucket_slots == c.bucket_slots && gr.cfg.lanes == c.lanes) gp = &gr;
        if (!gp) {
            groups.emplace_back();
            gp = &groups.back();
            gp->cfg = c;
            gp->slot_of.assign(ntables, ~0u);
        }
        if (gp->slot_of[w.table] == ~0u) {
            gp->slot_of[w.table] = uint32_t(gp->tabs.size());
            gp->tabs.push_back(t->dt);
        }
        WorkDesc d;
        d.keys = w.d_keys;
        d.flags = w.d_is_new;
        d.n = w.n;
        d.tile_off = gp->tiles;
        d.table = gp->slot_of[w.table];
        d.pad_ = 0;
        gp->items.push_back(d);
        gp->tiles += (w.n + 31) / 32;
    }
    for (auto& gr : groups) {
        const size_t tb = gr.tabs.size() * sizeof(DevTable), ib = gr.items.size() * sizeof(WorkDesc);
        const size_t toff = (ib + 255) / 256 * 256;
        char* scratch = nullptr;
        HT_TRY(cudaMallocAsync(&scratch, toff + tb, s));
        // Pageable sources: each copy has read its source when the call returns.
        cudaError_t e = cudaMemcpyAsync(scratch, gr.items.data(), ib, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = cudaMemcpyAsync(scratch + toff, gr.tabs.data(), tb, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess)
            e = packed_bucket_find_or_put(gr.cfg, reinterpret_cast<const DevTable*>(scratch + toff),
                                          reinterpret_cast<const WorkDesc*>(scratch), uint32_t(gr.items.size()),
                                          gr.tiles, s);
        cudaFreeAsync(scratch, s);
        if (e != cudaSuccess) return cuda_status(e);
    }
    // Cuckoo items, in list order.
    for (uint32_t i = 0; i < m; ++i) {
        const ht_work& w = list[i];
        ht_table* t = tables[w.table];
        if (t->scheme != HT_CUCKOO || w.n == 0) continue;
        const ht_status st = run_put(t, w.d_keys, nullptr, w.n, w.d_is_new, nullptr, nullptr, s);
        if (st != HT_OK) return st;
    }
    return HT_OK;
}

ht_status ht_sync(ht_table* t, void* stream) {
    if (!t) return HT_ERR_INVALID;
    DeviceGuard g(t->device);
    return sync_and_status(t, as_stream(stream));
}

ht_status ht_size(ht_table* t, uint64_t* out, void* stream) {
    if (!t || !out) return HT_ERR_INVALID;
    DeviceGuard g(t->device);
    const cudaStream_t s = as_stream(stream);
    ht_status st = sync_and_status(t, s);
    DevCounters c;
    ht_status st2 = read_counters(t, &c, s);
    if (st2 != HT_OK) return st2;
    *out = c.size;
    return st;
}

ht_status ht_export(ht_table* t, void* d_keys_out, uint32_t* d_values_out, uint64_t cap, uint64_t* count,
                    void* stream) {
    if (!t || !count || (cap && !d_keys_out) || (d_values_out && t->kw != 32)) return HT_ERR_INVALID;
    DeviceGuard g(t->device);
    const cudaStream_t s = as_stream(stream);
    ht_status st = sync_and_status(t, s);
    if (st == HT_ERR_CUDA) return st;
    unsigned long long* cnt = nullptr;
    HT_TRY(cudaMalloc(&cnt, sizeof(*cnt)));
    cudaError_t e = cudaMemsetAsync(cnt, 0, sizeof(*cnt), s);
    if (e == cudaSuccess) e = export_any(t, d_keys_out, d_values_out, cnt, cap, s);
    unsigned long long got = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&got, cnt, sizeof(got), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(cnt);
    if (e != cudaSuccess) return cuda_status(e);
    *count = got;
    if (got > cap) return HT_ERR_INVALID;
    return st;
}

ht_status ht_clear(ht_table* t, void* stream) {
    if (!t) return HT_ERR_INVALID;
    DeviceGuard g(t->device);
    t->sticky = HT_OK;
    t->rebuild_exhausted = false;
    return clear_table(t, as_stream(stream));
}

ht_status ht_grow(ht_table* t, uint64_t new_capacity, void* stream) {
    if (!t || new_capacity == 0 || new_capacity > kMaxCapacity) return HT_ERR_INVALID;
    DeviceGuard g(t->device);
    return grow_to(t, new_capacity, as_stream(stream));
}

ht_status ht_stats(ht_table* t, ht_table_stats* out, void* stream) {
    if (!t || !out) return HT_ERR_INVALID;
    DevCounters c;
    const ht_status st = read_counters(t, &c, static_cast<cudaStream_t>(stream));
    if (st != HT_OK) return st;
    std::memset(out, 0, sizeof(*out));
    out->size = c.size;
    out->dropped = c.dropped;
    out->exchanges = c.exchanges;
    out->probes = c.probes;
    out->probe_misses = c.probe_misses;
    out->probe_miss_reads = c.probe_miss_reads;
    out->probe_cas = c.probe_cas;
    out->stash_used = c.stash_used;
    out->overflow_used = c.ovf_used;
    out->rebuilds = t->rebuilds;
    out->flags = c.flags;
    return HT_OK;
}

ht_status ht_table_words(const ht_table* t, void** d_slots, uint64_t* bytes) {
    if (!t || !d_slots || !bytes) return HT_ERR_INVALID;
    const uint64_t slot_bytes = (t->kw == 128 || (is_long(t->kw) && t->scheme == HT_CUCKOO)) ? 16 : 8;
    *d_slots = t->dt.slots;
    *bytes = t->dt.nslots * slot_bytes;
    return HT_OK;
}

ht_status ht_info(const ht_table* t, uint64_t* slots, uint32_t* num_hashes, uint32_t* rebuilds) {
    if (!t) return HT_ERR_INVALID;
    if (slots) *slots = t->dt.nslots;
    if (num_hashes) *num_hashes = t->dt.k;
    if (rebuilds) *rebuilds = t->rebuilds;
    return HT_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// State-space exploration.
// ---------------------------------------------------------------------------
namespace {

}  // namespace

// Checks the model's fields against the layout documented in ht.h and
// returns the largest number of successors one state can have (0 = invalid).
uint64_t ht::model_max_successors(const ht_model* m, uint32_t key_width) {
    if (!m || m->num_components < 1 || m->num_components > 16 || m->num_pairs < 0 || m->num_pairs > 8) return 0;
    if (key_width != 32 && key_width != 64 && key_width != 128) return 0;
    uint32_t bits = 0;
    for (int c = 0; c < m->num_components; ++c) {
        if (m->bits[c] < 1 || m->bits[c] > 5) return 0;
        bits += m->bits[c];
    }
    if (bits > (key_width == 32 ? 31u : key_width == 64 ? 63u : 127u)) return 0;
    for (int p = 0; p < m->num_pairs; ++p)
        if (m->pair_c1[p] >= m->num_components || m->pair_c2[p] >= m->num_components ||
            m->pair_c1[p] == m->pair_c2[p])
            return 0;
    uint64_t total = 0;
    for (int c = 0; c < m->num_components; ++c) {
        uint32_t most = 0;
        for (uint32_t u = 0; u < (1u << m->bits[c]); ++u) {
            if (m->deg[c][u] > 4) return 0;
            uint32_t local = 0;
            for (int j = 0; j < m->deg[c][u]; ++j) {
                if (m->tgt[c][u][j] >= (1u << m->bits[c]) || m->lab[c][u][j] > m->num_pairs) return 0;
                local += m->lab[c][u][j] == 0;
            }
            most = std::max(most, local);
        }
        total += most;
    }
    for (int p = 0; p < m->num_pairs; ++p) {
        uint32_t most[2] = {0, 0};
        const int cs[2] = {m->pair_c1[p], m->pair_c2[p]};
        for (int side = 0; side < 2; ++side)
            for (uint32_t u = 0; u < (1u << m->bits[cs[side]]); ++u) {
                uint32_t k = 0;
                for (int j = 0; j < m->deg[cs[side]][u]; ++j) k += m->lab[cs[side]][u][j] == p + 1;
                most[side] = std::max(most[side], k);
            }
        total += uint64_t(most[0]) * most[1];
    }
    return total ? total : 1;
}

const DevTable& ht::table_dev(const ht_table* t) { return t->dt; }
const DevScratch& ht::table_scratch(const ht_table* t) { return t->sc; }
void ht::table_release(ht_table* t, cudaStream_t s) {
    if (!t) return;
    DeviceGuard g(t->device);
    free_table(t, s);
}
BucketCfg ht::table_bucket_cfg(const ht_table* t) { return bucket_cfg(t); }
ht_scheme ht::table_scheme(const ht_table* t) { return t->scheme; }
uint32_t ht::table_key_width(const ht_table* t) { return t->kw; }

namespace {

struct DevBuf {
    void* p = nullptr;
    ~DevBuf() { cudaFree(p); }
};

}  // namespace

extern "C" {

ht_status ht_successors(const ht_model* h_model, uint32_t key_width, const void* d_states, uint64_t n,
                        void* d_succ, uint64_t cap, unsigned long long* d_count, void* stream) {
    if ((key_width != 32 && key_width != 64 && key_width != 128) || !d_count || (n && (!d_states || !d_succ)))
        return HT_ERR_INVALID;
    if (!model_max_successors(h_model, key_width)) return HT_ERR_INVALID;
    if (n == 0) return HT_OK;
    const cudaStream_t s = as_stream(stream);
    DevBuf dm;
    const PreparedModel pm = prepare_model(*h_model);
    HT_TRY(cudaMalloc(&dm.p, sizeof(PreparedModel)));
    HT_TRY(cudaMemcpyAsync(dm.p, &pm, sizeof(pm), cudaMemcpyHostToDevice, s));
    HT_TRY(successors(int(key_width), static_cast<const PreparedModel*>(dm.p), d_states, n, nullptr, 0, d_succ, cap,
                      d_count, nullptr, s));
    HT_TRY(cudaStreamSynchronize(s));        // the model copy is freed on return
    return HT_OK;
}

static ht_status bfs_common(ht_table* t, const ht_model* h_model, uint64_t s0, uint32_t max_levels,
                            uint64_t* h_level_sizes, void* d_states, uint64_t states_cap, ht_bfs_result* result,
                            void* stream, bool fused) {
    if (!t || !result) return HT_ERR_INVALID;
    if (fused && (t->scheme != HT_BUCKET || t->kw == 128)) return HT_ERR_INVALID;
    const uint64_t msucc = model_max_successors(h_model, t->kw);
    if (!msucc) return HT_ERR_INVALID;
    if (t->kw == 32 ? s0 >= 0xFFFFFFFFull : (s0 >> 63) != 0) return HT_ERR_INVALID;
    DeviceGuard g(t->device);
    const cudaStream_t s = as_stream(stream);
    std::memset(result, 0, sizeof(*result));
    const size_t ksz = t->kw / 8;
    if (!d_states) {
        if (!states_cap) states_cap = t->dt.nslots + t->dt.stash_slots + t->dt.ovf_slots;
    } else if (!states_cap) {
        return HT_ERR_INVALID;
    }
    // Successor buffer (split form): up to 2^26 vectors per find-or-put
    // launch sequence; the fused form has none.
    const uint64_t succ_cap =
        fused ? 1 : std::min<uint64_t>(1ull << 26, std::max<uint64_t>(msucc, (t->dt.nslots + 1) * msucc));
    const uint64_t chunk_states = std::max<uint64_t>(1, succ_cap / msucc);
    DevBuf dm, states_own, succ, ctr;
    const PreparedModel pm = prepare_model(*h_model);
    HT_TRY(cudaMalloc(&dm.p, sizeof(PreparedModel)));
    HT_TRY(cudaMemcpyAsync(dm.p, &pm, sizeof(pm), cudaMemcpyHostToDevice, s));
    if (!d_states) {
        HT_TRY(cudaMalloc(&states_own.p, states_cap * ksz));
        d_states = states_own.p;
    }
    HT_TRY(cudaMalloc(&succ.p, succ_cap * ksz));
    // ctr[0]: states stored so far; ctr[1]: successors of the current chunk;
    // ctr[2]: successors generated in total; ctr[4..5]: the initial state
    // (16-byte aligned; for 128-bit tables s0 is its low word, the high word 0).
    HT_TRY(cudaMalloc(&ctr.p, 6 * sizeof(unsigned long long)));
    unsigned long long* c = static_cast<unsigned long long*>(ctr.p);
    unsigned long long init[6] = {0, 0, 0, 0, s0, 0};
    HT_TRY(cudaMemcpyAsync(c, init, sizeof(init), cudaMemcpyHostToDevice, s));
    // Level 0: the initial state (the open set starts with it).
    ht_status st = run_put(t, t->kw == 32 ? static_cast<const void*>(reinterpret_cast<const uint32_t*>(c + 4))
                                          : static_cast<const void*>(c + 4),
                           nullptr, 1, nullptr, d_states, c, s, nullptr, states_cap);
    if (st != HT_OK) return st;
    char* states = static_cast<char*>(d_states);
    uint64_t lo = 0;
    uint32_t level = 0;
    for (;;) {
        unsigned long long hi = 0;
        HT_TRY(cudaMemcpyAsync(&hi, c, sizeof(hi), cudaMemcpyDeviceToHost, s));
        HT_TRY(cudaStreamSynchronize(s));
        if (hi > states_cap) {               // the states buffer overflowed: stop
            result->states = states_cap;
            result->levels = level;
            break;
        }
        const uint64_t nd = hi - lo;
        if (nd == 0) {
            result->complete = 1;
            result->states = hi;
            result->levels = level;
            break;
        }
        if (level >= max_levels) {
            result->states = hi;
            result->levels = level;
            break;
        }
        if (h_level_sizes) h_level_sizes[level] = nd;
        if (fused) {
            HT_TRY(bfs_fused_level(bucket_cfg(t), static_cast<const PreparedModel*>(dm.p), states + lo * ksz, nd,
                                   t->dt, d_states, c, states_cap, c + 2, s));
            lo = hi;
            ++level;
            continue;
        }
        for (uint64_t c0 = lo; c0 < hi; c0 += chunk_states) {
            const uint64_t m = std::min<uint64_t>(chunk_states, hi - c0);
            HT_TRY(cudaMemsetAsync(c + 1, 0, sizeof(unsigned long long), s));
            HT_TRY(successors(int(t->kw), static_cast<const PreparedModel*>(dm.p), states + c0 * ksz, m, nullptr, 0, succ.p,
                              succ_cap, c + 1, c + 2, s));
            st = run_put(t, succ.p, nullptr, std::min<uint64_t>(succ_cap, m * msucc), nullptr, d_states, c, s, c + 1,
                         states_cap);
            if (st != HT_OK) return st;
        }
        lo = hi;
        ++level;
    }
    unsigned long long gen = 0;
    HT_TRY(cudaMemcpyAsync(&gen, c + 2, sizeof(gen), cudaMemcpyDeviceToHost, s));
    HT_TRY(cudaStreamSynchronize(s));
    result->successors = gen;
    const ht_status ts = sync_and_status(t, s);
    return ts;
}

ht_status ht_bfs(ht_table* t, const ht_model* h_model, uint64_t s0, uint32_t max_levels, uint64_t* h_level_sizes,
                 void* d_states, uint64_t states_cap, ht_bfs_result* result, void* stream) {
    return bfs_common(t, h_model, s0, max_levels, h_level_sizes, d_states, states_cap, result, stream, false);
}

ht_status ht_bfs_fused(ht_table* t, const ht_model* h_model, uint64_t s0, uint32_t max_levels,
                       uint64_t* h_level_sizes, void* d_states, uint64_t states_cap, ht_bfs_result* result,
                       void* stream) {
    return bfs_common(t, h_model, s0, max_levels, h_level_sizes, d_states, states_cap, result, stream, true);
}

}  // extern "C"
