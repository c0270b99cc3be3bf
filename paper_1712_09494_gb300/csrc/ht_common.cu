// Kernels shared by both schemes: export, fill, frontier compaction, the
// random-read roofline probe; plus launch sizing and event timing.
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
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x + r * stride;
        const bool keep = i < n && flags[i] != 0;
        T k = keep ? keys[i] : T(0);
        warp_append<T>(keep, k, out, count);
    }
}

// Random reads of `gran` bytes at gran-aligned offsets; four independent
// reads in flight per thread.
template <int GRAN>
__global__ void __launch_bounds__(kBlock)
probe_read_kernel(const uint64_t* __restrict__ buf, uint64_t nblocks, uint64_t n_access, uint64_t seed,
                  unsigned long long* __restrict__ sink) {
    constexpr int W = GRAN / 16;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    uint64_t acc = 0;
    for (uint64_t i = tid * 4; i < n_access; i += stride * 4) {
        ulonglong2 v[4][W];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const uint64_t b = __umul64hi(mix64(seed ^ (i + u)), nblocks);
            const ulonglong2* p = reinterpret_cast<const ulonglong2*>(buf + b * (GRAN / 8));
#pragma unroll
            for (int w = 0; w < W; ++w) v[u][w] = (i + u < n_access) ? __ldcg(p + w) : make_ulonglong2(0, 0);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
            for (int w = 0; w < W; ++w) acc ^= v[u][w].x ^ v[u][w].y;
    }
    for (int o = 16; o; o >>= 1) acc ^= __shfl_down_sync(0xFFFFFFFFu, acc, o);
    if ((threadIdx.x & 31) == 0 && acc == 0x9E3779B97F4A7C15ull) atomicXor(sink, acc);
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
    "export", "clear", "compact", "probe_random_read", "successors",
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
    const uint64_t nblocks = bytes / gran;
    const uint64_t* b = static_cast<const uint64_t*>(buf);
#define L(G)                                                                                  \
    {                                                                                         \
        auto k = probe_read_kernel<G>;                                                        \
        k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(b, nblocks, n_access, seed, sink); \
    }
    if (gran == 32) L(32) else if (gran == 64) L(64) else L(128)
#undef L
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
    if (!d_buf || !d_sink || (gran != 32 && gran != 64 && gran != 128) || bytes < gran)
        return HT_ERR_INVALID;
    return ht::probe_random_read(d_buf, bytes, gran, n_access, seed, d_sink,
                                 static_cast<cudaStream_t>(stream)) == cudaSuccess ? HT_OK : HT_ERR_CUDA;
}

}  // extern "C"
