// ht_cuckoo_find_or_put_noalloc: Cuckoo find-or-put for callers that cannot
// allocate device memory.
//
// Some callers own all of their device memory up front -- an arena carved out
// at start-up, a framework whose caching allocator already holds the GPU's
// memory, or code on a path where cudaMalloc is not allowed (it may
// synchronise the device, and it is refused while a stream is being
// captured).  They can give the table memory themselves, but not the
// per-batch dedup set and winner list that Cuckoo find-or-put needs.  This
// entry point takes that scratch from one static device array of fixed size
// instead, and runs the same probe and insert kernels as ht_find_or_put.
//
// The array belongs to the library: every GPU on which the library is used
// holds it (8 MiB) until the process exits.  All calls share it, so calls
// whose work overlaps on the GPU (different streams, or several host threads)
// race on it; callers must order them.
#include <cstring>

#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr uint64_t kNoallocMaxBatch = 1ull << 18;        // keys per call
constexpr uint64_t kNoallocSetSlots = 2 * kNoallocMaxBatch;
constexpr uint64_t kNoallocWords = kNoallocSetSlots + kNoallocMaxBatch * (sizeof(Winner) / 8);

// Dedup set (kNoallocSetSlots words) followed by the winner list.
static __device__ __align__(256) uint64_t g_noalloc_scratch[kNoallocWords];

// Layout of the caller's state block (HT_NOALLOC_STATE_BYTES bytes).
constexpr uint64_t kStateCtrWords = 16;       // DevCounters, padded to 128 bytes
constexpr uint32_t kStateStash = 101;
constexpr uint64_t kStateStashWords = 128;
constexpr uint32_t kStateOvf = 64;            // power of two
static_assert(sizeof(DevCounters) <= kStateCtrWords * 8, "counters fit the header");
static_assert((kStateCtrWords + kStateStashWords + kStateOvf) * 8 <= HT_NOALLOC_STATE_BYTES, "state fits");

// The array's device address on the current device.  The name is only a
// host-side stand-in, so the address is looked up on every call (a host-side
// lookup, no allocation): a cached address would go stale when the module is
// loaded again after a device reset.
cudaError_t scratch_on_current_device(uint64_t** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess) return e;
    *out = static_cast<uint64_t*>(p);
    return cudaSuccess;
}

}  // namespace
}  // namespace ht

extern "C" ht_status ht_cuckoo_find_or_put_noalloc(uint64_t* d_slots, uint64_t nslots, void* d_state,
                                                   uint64_t seed, const uint64_t* d_keys, uint64_t n,
                                                   uint8_t* d_is_new, int reset, void* stream) {
    using namespace ht;
    if (!d_slots || !d_state || nslots == 0 || nslots > (1ull << 40)) return HT_ERR_INVALID;
    if (n > kNoallocMaxBatch || (n && !d_keys)) return HT_ERR_INVALID;
    if ((reinterpret_cast<uintptr_t>(d_slots) | reinterpret_cast<uintptr_t>(d_keys)) & 7) return HT_ERR_INVALID;
    if (reinterpret_cast<uintptr_t>(d_state) & 15) return HT_ERR_INVALID;
    const cudaStream_t s = static_cast<cudaStream_t>(stream);
    uint64_t* scratch = nullptr;
    if (scratch_on_current_device(&scratch) != cudaSuccess) return HT_ERR_CUDA;

    uint64_t* state = static_cast<uint64_t*>(d_state);
    DevTable t;
    memset(&t, 0, sizeof(t));
    t.slots = d_slots;
    t.nslots = nslots;
    t.nbuckets = nslots;
    t.ctr = reinterpret_cast<DevCounters*>(state);
    t.stash = state + kStateCtrWords;
    t.stash_slots = kStateStash;
    t.ovf = state + kStateCtrWords + kStateStashWords;
    t.ovf_slots = kStateOvf;
    t.k = 4;
    t.max_evict = 256;
    for (int a = 0; a < kMaxHashes; ++a) t.seed[a] = mix64(seed + uint64_t(a + 1) * 0x9E3779B97F4A7C15ull);
    t.aux_seed = mix64(seed ^ 0xD1B54A32D192ED03ull);
    DevScratch sc;
    sc.set = scratch;
    sc.mask = kNoallocSetSlots - 1;
    sc.win = reinterpret_cast<Winner*>(scratch + kNoallocSetSlots);
    sc.win_cap = kNoallocMaxBatch;

    if (reset) {
        if (fill_words(d_slots, nslots, kEmpty, s) != cudaSuccess ||
            fill_words(t.stash, kStateStashWords + kStateOvf, kEmpty, s) != cudaSuccess ||
            cudaMemsetAsync(t.ctr, 0, kStateCtrWords * 8, s) != cudaSuccess)
            return HT_ERR_CUDA;
    }
    if (n == 0) return HT_OK;
    // The array keeps whatever the previous call left: empty the dedup set
    // and zero this call's winner count before the probe.
    if (fill_words(sc.set, kNoallocSetSlots, kEmpty, s) != cudaSuccess ||
        cudaMemsetAsync(&t.ctr->winners[0], 0, sizeof(unsigned int), s) != cudaSuccess)
        return HT_ERR_CUDA;
    if (cuckoo_probe(64, t, sc, 0, d_keys, nullptr, n, nullptr, 0, d_is_new, s, L2Window(), false) != cudaSuccess)
        return HT_ERR_CUDA;
    if (cuckoo_insert(64, t, sc, 0, nullptr, nullptr, 0, n, s) != cudaSuccess) return HT_ERR_CUDA;
    return HT_OK;
}
