// Kernels shared by both schemes: export, fill, frontier compaction, the
// random-read roofline probe; plus launch sizing and event timing.
#include <algorithm>
#include <mutex>
#include <unordered_map>
#include <vector>

#include "ht_internal.cuh"

namespace ht {
namespace {

__device__ __forceinline__ unsigned long long warp_reserve(bool pred, unsigned long long* counter,
                                                          unsigned* mask_out) {
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
    *mask_out = mask;
    if (!mask) return 0;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    return base + __popc(mask & ((1u << lane) - 1));
}

// Every non-empty word of slots[], stash[] and ovf[] (one index space).
template <int KW>
__global__ void __launch_bounds__(kBlock)
export_kernel(const DevTable t, typename Keys<KW>::T* __restrict__ keys_out,
              uint32_t* __restrict__ vals_out, unsigned long long* __restrict__ count, uint64_t cap) {
    using K = Keys<KW>;
    const uint64_t total = t.nslots + t.stash_slots + t.ovf_slots;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t rounds = (total + stride - 1) / stride;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x + r * stride;
        uint64_t w = kEmpty;
        if (i < t.nslots) w = __ldcg(reinterpret_cast<const unsigned long long*>(t.slots + i));
        else if (i < t.nslots + t.stash_slots) w = __ldcg(reinterpret_cast<const unsigned long long*>(t.stash + (i - t.nslots)));
        else if (i < total) w = __ldcg(reinterpret_cast<const unsigned long long*>(t.ovf + (i - t.nslots - t.stash_slots)));
        const bool keep = !K::empty(w);
        unsigned m;
        const unsigned long long at = warp_reserve(keep, count, &m);
        if (keep && at < cap) {
            keys_out[at] = typename K::T(K::keyof(w));
            if (vals_out) vals_out[at] = K::value(w);
        }
    }
}

__global__ void __launch_bounds__(kBlock) fill_kernel(uint64_t* __restrict__ p, uint64_t n, uint64_t v) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t n2 = n / 2;
    ulonglong2* q = reinterpret_cast<ulonglong2*>(p);
    for (uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x; i < n2; i += stride)
        q[i] = make_ulonglong2(v, v);
    if ((n & 1) && blockIdx.x == 0 && threadIdx.x == 0) p[n - 1] = v;
}

template <typename T>
__global__ void __launch_bounds__(kBlock)
compact_kernel(const T* __restrict__ keys, const uint8_t* __restrict__ flags, uint64_t n,
               T* __restrict__ out, unsigned long long* __restrict__ count) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t rounds = (n + stride - 1) / stride;
    __shared__ T s_keep[kBlock / 32][kStageCap];
    WarpStage<T, kStageCap> stage(s_keep[threadIdx.x >> 5]);
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x + r * stride;
        const bool keep = i < n && flags[i] != 0;
        T k = keep ? keys[i] : T(0);
        stage.push(keep, k, out, count, ~0ull);
    }
    stage.flush(out, count, ~0ull);
}

// Random-read probe (the denominator of the hash probes' roofline).
//   GRAN 8:   each thread keeps 8 independent 8-byte loads in flight
//             (a Cuckoo slot probe);
//   GRAN 32:  each thread keeps 4 independent 32-byte (256-bit) loads in flight;
//   GRAN 128: each group of 8 lanes reads one 128-byte line with one
//             coalesced 16-byte load per lane, 4 lines in flight per group
//             (a bucket probe).
// Offsets come from a 32-bit mixer so address arithmetic stays cheap.
__device__ __forceinline__ uint32_t mix32(uint32_t x) {
    x ^= x >> 16;
    x *= 0x7FEB352Du;
    x ^= x >> 15;
    x *= 0x846CA68Bu;
    x ^= x >> 16;
    return x;
}

template <int GRAN>
__global__ void __launch_bounds__(kBlock)
probe_read_kernel(const uint64_t* __restrict__ buf, uint32_t nblocks, uint64_t n_access, uint32_t seed,
                  unsigned long long* __restrict__ sink) {
    constexpr int U = GRAN == 8 ? 8 : 4;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nthreads = uint64_t(gridDim.x) * blockDim.x;
    // Accesses handled per "unit": a thread (8, 32) or an 8-lane group (128).
    const uint64_t unit = GRAN == 128 ? tid / 8 : tid;
    const uint64_t units = GRAN == 128 ? nthreads / 8 : nthreads;
    const uint64_t iters = (n_access + units * U - 1) / (units * U);
    uint64_t acc = 0;
    for (uint64_t it = 0; it < iters; ++it) {
        uint64_t v[U][2];
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t a = (it * units + unit) * U + u;
            const uint32_t b = __umulhi(mix32(uint32_t(a) * 0x9E3779B9u + uint32_t(a >> 32) + seed), nblocks);
            const uint64_t* p = buf + uint64_t(b) * (GRAN / 8);
            v[u][0] = v[u][1] = 0;
            if (a < n_access) {
                if constexpr (GRAN == 8) {
                    v[u][0] = __ldcg(reinterpret_cast<const unsigned long long*>(p));
                } else if constexpr (GRAN == 32) {
                    unsigned long long x0, x1, x2, x3;
                    asm volatile("ld.global.cg.v4.u64 {%0,%1,%2,%3}, [%4];"
                                 : "=l"(x0), "=l"(x1), "=l"(x2), "=l"(x3) : "l"(p));
                    v[u][0] = x0 ^ x2;
                    v[u][1] = x1 ^ x3;
                } else {
                    const ulonglong2 x = __ldcg(reinterpret_cast<const ulonglong2*>(p) + (threadIdx.x & 7));
                    v[u][0] = x.x;
                    v[u][1] = x.y;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < U; ++u) acc ^= v[u][0] ^ v[u][1];
    }
    for (int o = 16; o; o >>= 1) acc ^= __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc == 0x9E3779B97F4A7C15ull) atomicXor(sink, acc);
}

// Random read-modify-write: n_access 8-byte atomic adds at uniformly random
// 128-byte-aligned offsets, eight in flight per thread.  Each one makes L2
// fetch a line from DRAM and, once evicted, write it back: the cost of a
// claim in a random line.
__global__ void __launch_bounds__(kBlock)
probe_rmw_kernel(unsigned long long* __restrict__ buf, uint32_t nlines, uint64_t n_access, uint32_t seed) {
    constexpr int U = 8;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nthreads = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t iters = (n_access + nthreads * U - 1) / (nthreads * U);
    for (uint64_t it = 0; it < iters; ++it) {
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const uint64_t a = (it * nthreads + tid) * U + u;
            const uint32_t b = __umulhi(mix32(uint32_t(a) * 0x9E3779B9u + uint32_t(a >> 32) + seed), nlines);
            if (a < n_access) atomicAdd(buf + uint64_t(b) * 16, 1ull);
        }
    }
}

// ------------------------------------------------------------- profiling
struct ProfRec {
    uint32_t id;
    cudaEvent_t a, b;
};

struct Prof {
    std::mutex mu;
    bool on = false;
    std::vector<ProfRec> pending;
    std::vector<std::pair<cudaEvent_t, cudaEvent_t>> pool;
    uint64_t launches[kKNumKernels] = {};
    double ms[kKNumKernels] = {};
};

Prof& prof() {
    static Prof* p = new Prof();
    return *p;
}

const char* kNames[kKNumKernels] = {
    "bucket_find_or_put", "bucket_lookup", "cuckoo_probe", "cuckoo_insert", "cuckoo_lookup",
    "export", "clear", "compact", "probe_random_read", "successors", "probe_random_rmw",
    "multi_persistent",
};

}  // namespace

ProfScope::ProfScope(uint32_t id, cudaStream_t s) : id_(id), s_(s), slot_(-1) {
    Prof& p = prof();
    if (!p.on) return;
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return;
    std::lock_guard<std::mutex> g(p.mu);
    ProfRec r;
    r.id = id;
    if (!p.pool.empty()) {
        r.a = p.pool.back().first;
        r.b = p.pool.back().second;
        p.pool.pop_back();
    } else {
        cudaEventCreate(&r.a);
        cudaEventCreate(&r.b);
    }
    cudaEventRecord(r.a, s);
    p.pending.push_back(r);
    slot_ = int(p.pending.size()) - 1;
}

ProfScope::~ProfScope() {
    if (slot_ < 0) return;
    Prof& p = prof();
    std::lock_guard<std::mutex> g(p.mu);
    if (slot_ < int(p.pending.size())) cudaEventRecord(p.pending[slot_].b, s_);
}

int launch_blocks(const void* kernel, int block, size_t smem) {
    static std::mutex mu;
    static std::unordered_map<const void*, int> cache[64];
    int dev = 0;
    cudaGetDevice(&dev);
    std::lock_guard<std::mutex> g(mu);
    auto& c = cache[dev & 63];
    auto it = c.find(kernel);
    if (it != c.end()) return it->second;
    int sms = 0, per = 0;
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, smem);
    const int grid = (sms > 0 ? sms : 1) * (per > 0 ? per : 1);
    c.emplace(kernel, grid);
    return grid;
}

L2Window l2_window(const void* base, size_t bytes) {
    L2Window w;
    if (!base || !bytes) return w;
    static std::mutex mu;
    std::lock_guard<std::mutex> g(mu);
    int dev = 0, max_persist = 0, max_window = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_persist, cudaDevAttrMaxPersistingL2CacheSize, dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&max_window, cudaDevAttrMaxAccessPolicyWindowSize, dev) != cudaSuccess ||
        max_persist <= 0 || max_window <= 0)
        return w;
    size_t cur = 0;
    cudaDeviceGetLimit(&cur, cudaLimitPersistingL2CacheSize);
    const size_t want = std::min<size_t>(bytes, size_t(max_persist));
    if (cur < want && cudaDeviceSetLimit(cudaLimitPersistingL2CacheSize, want) == cudaSuccess) cur = want;
    if (!cur) return w;
    w.base = base;
    w.bytes = std::min<size_t>(bytes, size_t(max_window));
    w.hit = float(std::min<double>(1.0, double(cur) / double(w.bytes)));
    return w;
}

cudaError_t table_export(int kw, const DevTable& t, void* keys_out, uint32_t* vals_out,
                         unsigned long long* count, uint64_t cap, cudaStream_t s) {
    ProfScope ps(kKExport, s);
    if (kw == 32) {
        auto k = export_kernel<32>;
        k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, static_cast<uint32_t*>(keys_out), vals_out, count, cap);
    } else {
        auto k = export_kernel<64>;
        k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, static_cast<uint64_t*>(keys_out), vals_out, count, cap);
    }
    return cudaGetLastError();
}

cudaError_t fill_words(uint64_t* p, uint64_t n, uint64_t v, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ProfScope ps(kKClear, s);
    fill_kernel<<<launch_blocks((const void*)fill_kernel, kBlock), kBlock, 0, s>>>(p, n, v);
    return cudaGetLastError();
}

cudaError_t compact(int kw, const void* keys, const uint8_t* flags, uint64_t n, void* out,
                    unsigned long long* count, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ProfScope ps(kKCompact, s);
    if (kw == 32) {
        auto k = compact_kernel<uint32_t>;
        k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(static_cast<const uint32_t*>(keys), flags, n, static_cast<uint32_t*>(out), count);
    } else {
        auto k = compact_kernel<uint64_t>;
        k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(static_cast<const uint64_t*>(keys), flags, n, static_cast<uint64_t*>(out), count);
    }
    return cudaGetLastError();
}

cudaError_t probe_random_read(const void* buf, uint64_t bytes, uint32_t gran, uint64_t n_access,
                              uint64_t seed, unsigned long long* sink, cudaStream_t s) {
    ProfScope ps(kKProbeRead, s);
    const uint32_t nblocks = uint32_t(std::min<uint64_t>(bytes / gran, 0xFFFFFFFFull));
    const uint64_t* b = static_cast<const uint64_t*>(buf);
#define L(G)                                                                                           \
    {                                                                                                  \
        auto k = probe_read_kernel<G>;                                                                 \
        k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(b, nblocks, n_access, uint32_t(seed), sink); \
    }
    if (gran == 8) L(8) else if (gran == 32) L(32) else L(128)
#undef L
    return cudaGetLastError();
}

cudaError_t probe_random_rmw(void* buf, uint64_t bytes, uint64_t n_access, uint64_t seed, cudaStream_t s) {
    ProfScope ps(kKProbeRmw, s);
    const uint32_t nlines = uint32_t(std::min<uint64_t>(bytes / 128, 0xFFFFFFFFull));
    auto k = probe_rmw_kernel;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(static_cast<unsigned long long*>(buf), nlines,
                                                              n_access, uint32_t(seed));
    return cudaGetLastError();
}

}  // namespace ht

extern "C" {

ht_status ht_prof_enable(int on) {
    ht::prof().on = on != 0;
    return HT_OK;
}

ht_status ht_prof_reset(void) {
    ht::Prof& p = ht::prof();
    std::lock_guard<std::mutex> g(p.mu);
    for (auto& r : p.pending) {
        cudaEventSynchronize(r.b);
        p.pool.emplace_back(r.a, r.b);
    }
    p.pending.clear();
    for (int i = 0; i < ht::kKNumKernels; ++i) {
        p.launches[i] = 0;
        p.ms[i] = 0.0;
    }
    return HT_OK;
}

uint32_t ht_prof_num_kernels(void) { return ht::kKNumKernels; }

const char* ht_prof_kernel_name(uint32_t id) { return id < ht::kKNumKernels ? ht::kNames[id] : nullptr; }

ht_status ht_prof_read(uint32_t id, uint64_t* launches, double* total_ms) {
    if (id >= ht::kKNumKernels) return HT_ERR_INVALID;
    ht::Prof& p = ht::prof();
    std::lock_guard<std::mutex> g(p.mu);
    ht_status st = HT_OK;
    for (auto& r : p.pending) {
        float ms = 0.f;
        if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&ms, r.a, r.b) != cudaSuccess)
            st = HT_ERR_CUDA;
        p.launches[r.id] += 1;
        p.ms[r.id] += ms;
        p.pool.emplace_back(r.a, r.b);
    }
    p.pending.clear();
    if (launches) *launches = p.launches[id];
    if (total_ms) *total_ms = p.ms[id];
    return st;
}

ht_status ht_compact(const void* d_keys, const uint8_t* d_flags, uint64_t n, uint32_t key_width,
                     void* d_out, unsigned long long* d_count, void* stream) {
    if ((key_width != 32 && key_width != 64) || (n && (!d_keys || !d_flags || !d_out || !d_count)))
        return HT_ERR_INVALID;
    return ht::compact(int(key_width), d_keys, d_flags, n, d_out, d_count,
                       static_cast<cudaStream_t>(stream)) == cudaSuccess ? HT_OK : HT_ERR_CUDA;
}

ht_status ht_probe_random_read(const void* d_buf, uint64_t bytes, uint32_t gran, uint64_t n_access,
                               uint64_t seed, unsigned long long* d_sink, void* stream) {
    if (!d_buf || !d_sink || (gran != 8 && gran != 32 && gran != 128) || bytes < gran)
        return HT_ERR_INVALID;
    return ht::probe_random_read(d_buf, bytes, gran, n_access, seed, d_sink,
                                 static_cast<cudaStream_t>(stream)) == cudaSuccess ? HT_OK : HT_ERR_CUDA;
}

ht_status ht_probe_random_rmw(void* d_buf, uint64_t bytes, uint64_t n_access, uint64_t seed, void* stream) {
    if (!d_buf || bytes < 128 || (reinterpret_cast<uintptr_t>(d_buf) & 127)) return HT_ERR_INVALID;
    return ht::probe_random_rmw(d_buf, bytes, n_access, seed, static_cast<cudaStream_t>(stream)) == cudaSuccess
               ? HT_OK
               : HT_ERR_CUDA;
}

}  // extern "C"
