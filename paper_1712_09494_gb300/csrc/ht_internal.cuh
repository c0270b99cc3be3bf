// Internal definitions shared by the CUDA translation units of libht.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <utility>

#include "../../include/ht.h"

namespace ht {

constexpr uint64_t kEmpty = ~0ull;          // an empty slot: every bit set
constexpr int kMaxHashes = 16;              // bucket scheme upper bound
constexpr int kMaxCuckooHashes = 8;
constexpr uint32_t kOvfSlots = 1u << 16;    // overflow set behind the stash
constexpr int kBlock = 256;
constexpr uint32_t kDefaultSpinLimit = 1u << 20;   // long-key publish wait, polls (~0.1 s)

// Sticky device flags.
enum : uint32_t {
    kFlagInvalidKey = 1u,   // a reserved key was seen
    kFlagRebuild = 2u,      // the stash overflowed: rebuild with new constants
    kFlagDropped = 4u,      // a key found no place at all (table full)
    kFlagTimeout = 8u,      // a bounded wait for a claimed slot's publish gave up
};

struct DevCounters {
    unsigned long long size;      // keys stored (table + stash + overflow)
    unsigned long long dropped;   // keys that could not be placed
    unsigned int stash_used;
    unsigned int ovf_used;
    unsigned int flags;
    unsigned int winners[2];      // Cuckoo dedup winners per chunk parity
    unsigned int pad0_;
    unsigned long long exchanges; // Cuckoo: atomic exchanges made by insert chains
    unsigned long long probes;    // Cuckoo: slots the probes read (bucket scheme: not counted)
    unsigned long long ids;       // long-key Cuckoo: key-store rows handed out
    unsigned long long probe_misses;      // Cuckoo: probed keys found nowhere (64-bit path)
    unsigned long long probe_miss_reads;  // ... and the slots those keys' probes read
    unsigned long long probe_cas; // Cuckoo (32/64/128-bit keys): CASes of absent keys into table slots
};
static_assert(sizeof(DevCounters) == 88, "counter block layout");

// Everything a kernel needs to address a table; passed by value.
struct DevTable {
    uint64_t* slots;
    uint64_t nslots;          // capacity in slots
    uint64_t nbuckets;        // nslots / bucket_slots (bucket scheme)
    uint64_t* stash;
    uint64_t* ovf;
    DevCounters* ctr;
    uint32_t stash_slots;
    uint32_t ovf_slots;
    uint32_t k;               // hash functions
    uint32_t max_evict;       // Cuckoo eviction bound
    uint64_t aux_seed;        // stash / overflow / dedup start positions
    uint64_t seed[kMaxHashes];
    // Keys of more than two words (ht_long.cu): the key store (rows of
    // row_words words: the key's words, then a zero word when the count is
    // odd, so that rows are 16-byte aligned), its rows, and the mask applied
    // to every key digest (all ones except in tests that force digest
    // collisions).
    uint64_t* kstore;
    uint64_t kstore_rows;
    uint64_t digest_mask;
    uint32_t words;
    uint32_t row_words;
    // Cuckoo: 1 starts every insertion chain at h_1 (Section 4.1); 0 at the
    // first slot the probe saw empty.
    uint32_t chain_h1;
    // Long-key bucket scheme: polls of a claimed, unpublished header before
    // a reader gives up (kFlagTimeout).
    uint32_t spin_limit;
};

// A Cuckoo insertion job: the packed word, where its dedup claim sits, and
// the hash index its eviction chain starts at (0 = h_1).
struct Winner {
    uint64_t word;
    uint32_t spos;
    uint32_t start;
};

// Dedup scratch of one Cuckoo table: a linear-probing set of keys.
struct DevScratch {
    uint64_t* set;
    uint64_t mask;            // slots - 1 (power of two)
    Winner* win;
    uint64_t win_cap;         // entries of win
};

// ---------------------------------------------------------------------------
// Hash family.  h_a(k) = floor(mix64(k xor s_a) * m / 2^64): the SplitMix64
// output finaliser (Steele, Lea & Flood 2014) as the mixer and Lemire's
// multiply-high range reduction.  The paper names only "hash constants"
// copied to the GPU (Section 5); s_a are those constants.
// ---------------------------------------------------------------------------
__host__ __device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

__device__ __forceinline__ uint64_t hidx(uint64_t key, uint64_t s, uint64_t m) {
    return __umul64hi(mix64(key ^ s), m);
}

// Key <-> slot word.  32-bit keys sit in the low word with the value above;
// 64-bit keys fill the word.  keyof(kEmpty) is the reserved key, so
// "keyof(w) == reserved" means "empty".
template <int KW> struct Keys;
template <> struct Keys<32> {
    using T = uint32_t;
    static constexpr uint64_t kMask = 0xFFFFFFFFull;
    __device__ __forceinline__ static uint64_t keyof(uint64_t w) { return w & kMask; }
    __device__ __forceinline__ static bool empty(uint64_t w) { return (w & kMask) == kMask; }
    __device__ __forceinline__ static bool reserved(uint64_t k) { return k == kMask; }
    __device__ __forceinline__ static uint64_t word(uint64_t k, uint32_t v) { return (uint64_t(v) << 32) | k; }
    __device__ __forceinline__ static uint32_t value(uint64_t w) { return uint32_t(w >> 32); }
    __device__ __forceinline__ static uint64_t load(const void* p, uint64_t i) {
        return static_cast<const uint32_t*>(p)[i];
    }
};
template <> struct Keys<64> {
    using T = uint64_t;
    __device__ __forceinline__ static uint64_t keyof(uint64_t w) { return w; }
    __device__ __forceinline__ static bool empty(uint64_t w) { return w == kEmpty; }
    __device__ __forceinline__ static bool reserved(uint64_t k) { return (k >> 63) != 0; }
    __device__ __forceinline__ static uint64_t word(uint64_t k, uint32_t) { return k; }
    __device__ __forceinline__ static uint32_t value(uint64_t) { return 0u; }
    __device__ __forceinline__ static uint64_t load(const void* p, uint64_t i) {
        return static_cast<const uint64_t*>(p)[i];
    }
};

// 16-byte atomics on a 16-byte-aligned pair of words (sm_90 and later):
// compare-and-swap from EMPTY (all ones in both words), and exchange.
__device__ __forceinline__ void cas128(uint64_t* addr, uint64_t new_lo, uint64_t new_hi, uint64_t& old_lo,
                                       uint64_t& old_hi) {
    asm volatile(
        "{\n"
        " .reg .b128 d, c, n;\n"
        " mov.b128 c, {%2, %3};\n"
        " mov.b128 n, {%4, %5};\n"
        " atom.global.cas.b128 d, [%6], c, n;\n"
        " mov.b128 {%0, %1}, d;\n"
        "}\n"
        : "=l"(old_lo), "=l"(old_hi)
        : "l"(kEmpty), "l"(kEmpty), "l"(new_lo), "l"(new_hi), "l"(addr)
        : "memory");
}

__device__ __forceinline__ void exch128(uint64_t* addr, uint64_t lo, uint64_t hi, uint64_t& old_lo,
                                        uint64_t& old_hi) {
    asm volatile(
        "{\n"
        " .reg .b128 d, n;\n"
        " mov.b128 n, {%2, %3};\n"
        " atom.global.exch.b128 d, [%4], n;\n"
        " mov.b128 {%0, %1}, d;\n"
        "}\n"
        : "=l"(old_lo), "=l"(old_hi)
        : "l"(lo), "l"(hi), "l"(addr)
        : "memory");
}

__device__ __forceinline__ void set_flag(DevCounters* c, uint32_t f) {
    if ((*(volatile unsigned int*)&c->flags & f) != f) atomicOr(&c->flags, f);
}

// Linear-probing set with CAS claims (the stash, the overflow set, the dedup
// scratch).  Slots only ever go from empty to a fixed word, and every caller
// scans the same fixed order from the same start, so a key is claimed at
// most once: a later claimant passes the earlier claim's slot first.
// Returns 1 if `word` was stored here, 0 if its key was already present,
// -1 if all `n` slots are taken by other keys.
template <int KW>
__device__ __forceinline__ int lp_insert(uint64_t* arr, uint32_t n, uint64_t start,
                                         uint64_t key, uint64_t word, uint32_t* at) {
    uint32_t p = uint32_t(start);
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t w = __ldcg(reinterpret_cast<const unsigned long long*>(arr + p));
        if (Keys<KW>::empty(w)) {
            w = atomicCAS(reinterpret_cast<unsigned long long*>(arr + p), kEmpty, word);
            if (w == kEmpty) { if (at) *at = p; return 1; }
        }
        if (Keys<KW>::keyof(w) == key) { if (at) *at = p; return 0; }
        p = (p + 1 == n) ? 0 : p + 1;
    }
    return -1;
}

// Lookup in a linear-probing set: stops at the first empty slot.
template <int KW>
__device__ __forceinline__ bool lp_find(const uint64_t* arr, uint32_t n, uint64_t start,
                                        uint64_t key, uint64_t* out) {
    uint32_t p = uint32_t(start);
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t w = __ldcg(reinterpret_cast<const unsigned long long*>(arr + p));
        if (Keys<KW>::empty(w)) return false;
        if (Keys<KW>::keyof(w) == key) { *out = w; return true; }
        p = (p + 1 == n) ? 0 : p + 1;
    }
    return false;
}

__device__ __forceinline__ uint64_t stash_start(const DevTable& t, uint64_t key) {
    return mix64(key ^ t.aux_seed) % t.stash_slots;
}
__device__ __forceinline__ uint64_t ovf_start(const DevTable& t, uint64_t key) {
    return mix64(key ^ ~t.aux_seed) & (t.ovf_slots - 1);
}

// Places a word that found no slot in the main table: stash first, then the
// overflow set (which asks the host for a rebuild), else it is dropped.
// Returns 1 stored, 0 key already present, -1 dropped.
template <int KW>
__device__ __forceinline__ int place_spill(const DevTable& t, uint64_t key, uint64_t word) {
    int r = -1;
    if (t.stash_slots) {
        r = lp_insert<KW>(t.stash, t.stash_slots, stash_start(t, key), key, word, nullptr);
        if (r == 1) atomicAdd(&t.ctr->stash_used, 1u);
    }
    if (r < 0) {
        r = lp_insert<KW>(t.ovf, t.ovf_slots, ovf_start(t, key), key, word, nullptr);
        if (r == 1) {
            atomicAdd(&t.ctr->ovf_used, 1u);
            set_flag(t.ctr, kFlagRebuild);
        }
    }
    if (r < 0) {
        atomicAdd(&t.ctr->dropped, 1ull);
        set_flag(t.ctr, kFlagDropped);
    }
    return r;
}

// Looks a key up in the stash and then the overflow set.
template <int KW>
__device__ __forceinline__ bool find_spill(const DevTable& t, uint64_t key, uint32_t stash_used,
                                           uint32_t ovf_used, uint64_t* w) {
    if (stash_used && lp_find<KW>(t.stash, t.stash_slots, stash_start(t, key), key, w)) return true;
    if (ovf_used && lp_find<KW>(t.ovf, t.ovf_slots, ovf_start(t, key), key, w)) return true;
    return false;
}

// Warp-aggregated append of `v` (when `pred`) to out[] at *counter.  Slots at
// or past `cap` are not written (the counter still counts them).
template <typename T>
__device__ __forceinline__ void warp_append(bool pred, T v, T* out, unsigned long long* counter,
                                            uint64_t cap = ~0ull) {
    const unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
    if (!mask) return;
    const int lane = threadIdx.x & 31;
    const int leader = __ffs(mask) - 1;
    unsigned long long base = 0;
    if (lane == leader) base = atomicAdd(counter, (unsigned long long)__popc(mask));
    base = __shfl_sync(0xFFFFFFFFu, base, leader);
    const unsigned long long at = base + __popc(mask & ((1u << lane) - 1));
    if (pred && at < cap) out[at] = v;
}

// Warp-aggregated append staged in shared memory: the warp collects up to
// CAP entries in `buf` (its own CAP slots) and moves them out with one atomic
// on the counter per flush, instead of one atomic per 32-entry tile -- many
// warps appending to one counter otherwise serialise on its L2 slice.  Every
// lane of the warp calls push/flush together; flush must end the warp's
// work.  Entries past `cap` are not written (the counter still counts them).
template <typename T, int CAP>
struct WarpStage {
    T* buf;
    uint32_t pend;
    __device__ __forceinline__ explicit WarpStage(T* b) : buf(b), pend(0) {}
    __device__ __forceinline__ void flush(T* out, unsigned long long* counter, uint64_t cap) {
        __syncwarp();
        if (pend) {
            const int lane = threadIdx.x & 31;
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(counter, (unsigned long long)pend);
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            for (uint32_t j = lane; j < pend; j += 32)
                if (base + j < cap) out[base + j] = buf[j];
        }
        __syncwarp();
        pend = 0;
    }
    __device__ __forceinline__ void push(bool pred, T v, T* out, unsigned long long* counter, uint64_t cap) {
        const unsigned mask = __ballot_sync(0xFFFFFFFFu, pred);
        const uint32_t c = __popc(mask);
        if (pend + c > uint32_t(CAP)) flush(out, counter, cap);
        const int lane = threadIdx.x & 31;
        if (pred) buf[pend + __popc(mask & ((1u << lane) - 1))] = v;
        pend += c;
    }
};
constexpr int kStageCap = 256;   // entries per warp (8 tiles of 32)

// ---------------------------------------------------------------------------
// Kernel timing (ht_prof_*).
// ---------------------------------------------------------------------------
enum KernelId : uint32_t {
    kKBucketFop = 0,
    kKBucketLookup,
    kKCuckooProbe,
    kKCuckooInsert,
    kKCuckooLookup,
    kKExport,
    kKClear,
    kKCompact,
    kKProbeRead,
    kKSuccessors,
    kKProbeRmw,
    kKMultiPersistent,
    kKNumKernels
};

struct ProfScope {
    ProfScope(uint32_t id, cudaStream_t s);
    ~ProfScope();
    uint32_t id_;
    cudaStream_t s_;
    int slot_;
};

int launch_blocks(const void* kernel, int block, size_t smem = 0);

// L2 residency: an access-policy window that marks a range persisting in L2
// for the launches that carry it (bytes 0 = none).
struct L2Window {
    const void* base = nullptr;
    size_t bytes = 0;
    float hit = 0.f;
};

// Window over [base, base + bytes) if the device supports persisting L2:
// raises the context's persisting set-aside (cudaLimitPersistingL2CacheSize,
// a per-process setting that ends with the process) to cover it, up to the
// device maximum; hit < 1 when the range is larger than that.
L2Window l2_window(const void* base, size_t bytes);

template <typename... KArgs, typename... Args>
cudaError_t launch_win(void (*kernel)(KArgs...), int grid, int block, cudaStream_t s, const L2Window& w,
                       Args&&... args) {
    if (!w.bytes) {
        kernel<<<grid, block, 0, s>>>(std::forward<Args>(args)...);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeAccessPolicyWindow;
    at[0].val.accessPolicyWindow.base_ptr = const_cast<void*>(w.base);
    at[0].val.accessPolicyWindow.num_bytes = w.bytes;
    at[0].val.accessPolicyWindow.hitRatio = w.hit;
    at[0].val.accessPolicyWindow.hitProp = cudaAccessPropertyPersisting;
    at[0].val.accessPolicyWindow.missProp = cudaAccessPropertyStreaming;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

// ---------------------------------------------------------------------------
// Launchers implemented by the scheme translation units.  All return the
// cudaGetLastError() of the launch.
// ---------------------------------------------------------------------------
struct BucketCfg {
    int kw;
    int bucket_slots;
    int lanes;
};

// d_n (nullable): the batch size lives on the device; n is then an upper bound.
cudaError_t bucket_find_or_put(const BucketCfg& c, const DevTable& t, const void* keys,
                               const uint32_t* vals, uint64_t n, const unsigned long long* d_n,
                               uint8_t* is_new, void* new_out, unsigned long long* new_count,
                               uint64_t new_cap, cudaStream_t s, const L2Window& w = L2Window());
cudaError_t bucket_lookup(const BucketCfg& c, const DevTable& t, const void* keys, uint64_t n,
                          uint32_t* vals, uint8_t* found, cudaStream_t s, const L2Window& w = L2Window());

// d_n (nullable): the batch size lives on the device; this launch covers keys
// [off, off + n) of it.  list_stored: list the keys the probe stored itself
// in the winner list too (for an insert that appends every new key).
cudaError_t cuckoo_probe(int kw, const DevTable& t, const DevScratch& sc, uint32_t parity,
                         const void* keys, const uint32_t* vals, uint64_t n,
                         const unsigned long long* d_n, uint64_t off, uint8_t* is_new,
                         cudaStream_t s, const L2Window& w = L2Window(), bool list_stored = true);
cudaError_t cuckoo_insert(int kw, const DevTable& t, const DevScratch& sc, uint32_t parity,
                          void* new_out, unsigned long long* new_count, uint64_t new_cap,
                          uint64_t max_winners, cudaStream_t s, const L2Window& w = L2Window());
cudaError_t cuckoo_lookup(int kw, const DevTable& t, const void* keys, uint64_t n,
                          uint32_t* vals, uint8_t* found, cudaStream_t s, const L2Window& w = L2Window());

cudaError_t table_export(int kw, const DevTable& t, void* keys_out, uint32_t* vals_out,
                         unsigned long long* count, uint64_t cap, cudaStream_t s);
cudaError_t fill_words(uint64_t* p, uint64_t n, uint64_t v, cudaStream_t s);
cudaError_t compact(int kw, const void* keys, const uint8_t* flags, uint64_t n, void* out,
                    unsigned long long* count, cudaStream_t s);
cudaError_t probe_random_read(const void* buf, uint64_t bytes, uint32_t gran, uint64_t n_access,
                              uint64_t seed, unsigned long long* sink, cudaStream_t s);
cudaError_t probe_random_rmw(void* buf, uint64_t bytes, uint64_t n_access, uint64_t seed, cudaStream_t s);

// A model with its bit offsets precomputed (device copy; the single-table
// successor kernel stages it in shared memory).
// A model's transitions regrouped for successor generation: per component
// and local state the targets of its local (unlabelled) transitions, and per
// synchronising pair, member (0: pc1, 1: pc2) and local state the targets of
// that member's transitions carrying the pair's label.
struct PreparedModel {
    uint8_t nloc[16][32];
    uint8_t loc[16][32][4];
    uint8_t nsyn[8][2][32];
    uint8_t syn[8][2][32][4];
    uint8_t off[16];
    uint8_t bits[16];
    uint8_t pc1[8];
    uint8_t pc2[8];
    int C;
    int P;
};

PreparedModel prepare_model(const ht_model& m);

// Successor enumeration over a prepared model (state vectors of up to 64
// bits; component c's local state is bits [off[c], off[c] + bits[c])).
// S is the state vector's type: uint64_t, or unsigned __int128 for models
// wider than 63 bits.
template <class S>
__device__ __forceinline__ uint32_t local_of(const PreparedModel& m, S s, int c) {
    return uint32_t(s >> m.off[c]) & ((1u << m.bits[c]) - 1u);
}

template <class S>
__device__ __forceinline__ S with_local(const PreparedModel& m, S s, int c, uint32_t v) {
    const S mask = ((S(1) << m.bits[c]) - S(1)) << m.off[c];
    return (s & ~mask) | (S(v) << m.off[c]);
}

// Visits every successor of s: local actions of each component, then every
// combination of the two members' transitions of each synchronising pair.
template <class S, class F>
__device__ __forceinline__ void for_each_successor(const PreparedModel& m, S s, F&& emit) {
    for (int c = 0; c < m.C; ++c) {
        const uint32_t u = local_of(m, s, c);
        const int d = m.nloc[c][u];
        for (int j = 0; j < d; ++j) emit(with_local(m, s, c, m.loc[c][u][j]));
    }
    for (int p = 0; p < m.P; ++p) {
        const int c1 = m.pc1[p], c2 = m.pc2[p];
        const uint32_t u1 = local_of(m, s, c1), u2 = local_of(m, s, c2);
        const int d1 = m.nsyn[p][0][u1], d2 = m.nsyn[p][1][u2];
        for (int j1 = 0; j1 < d1; ++j1) {
            const S s1 = with_local(m, s, c1, m.syn[p][0][u1][j1]);
            for (int j2 = 0; j2 < d2; ++j2) emit(with_local(m, s1, c2, m.syn[p][1][u2][j2]));
        }
    }
}

// The number of successors of s (what for_each_successor visits).
template <class S>
__device__ __forceinline__ uint32_t count_successors(const PreparedModel& m, S s) {
    uint32_t n = 0;
    for (int c = 0; c < m.C; ++c) n += m.nloc[c][local_of(m, s, c)];
    for (int p = 0; p < m.P; ++p)
        n += uint32_t(m.nsyn[p][0][local_of(m, s, m.pc1[p])]) * m.nsyn[p][1][local_of(m, s, m.pc2[p])];
    return n;
}

// Largest number of successors of one state, or 0 for a malformed model.
uint64_t model_max_successors(const ht_model* m, uint32_t key_width);

// One BFS level fused: successors of frontier[0..n) generated and
// found-or-put into a bucket-scheme table in one launch; new states appended
// to out at *count (entries past cap not written); *gen += successors.
cudaError_t bfs_fused_level(const BucketCfg& c, const PreparedModel* model, const void* frontier, uint64_t n,
                            const DevTable& t, void* out, unsigned long long* count, uint64_t cap,
                            unsigned long long* gen, cudaStream_t s);

// Bucket-scheme tables of 128-bit keys (ht_wide.cu): keys are 16-byte pairs
// (low word, high word), 16-byte aligned; slots are 16 bytes, buckets 8 slots.
cudaError_t wide_find_or_put(int lanes, const DevTable& t, const void* keys, uint64_t n,
                             const unsigned long long* d_n, uint8_t* is_new, void* new_out,
                             unsigned long long* new_count, uint64_t new_cap, cudaStream_t s);
cudaError_t wide_lookup(int lanes, const DevTable& t, const void* keys, uint64_t n, uint8_t* found,
                        cudaStream_t s);
cudaError_t wide_export(const DevTable& t, void* keys, unsigned long long* count, uint64_t cap, cudaStream_t s);
// Cuckoo tables of 128-bit keys: probe (stores into the first empty slot,
// dedup of the keys with every slot full, winners of `parity`; list_stored:
// list the stored keys too, for an insert that appends every new key),
// insert (eviction chains; winners appended to new_out when non-null),
// lookup.  The claim set holds 16-byte entries and the winner list 32-byte
// records.
cudaError_t wide_cuckoo_probe(const DevTable& t, const DevScratch& sc, uint32_t parity, const void* keys, uint64_t n,
                              const unsigned long long* d_n, uint64_t off, uint8_t* is_new, cudaStream_t s,
                              bool list_stored = true);
cudaError_t wide_cuckoo_insert(const DevTable& t, const DevScratch& sc, uint32_t parity, void* new_out,
                               unsigned long long* new_count, uint64_t new_cap, uint64_t max_winners,
                               cudaStream_t s);
cudaError_t wide_cuckoo_lookup(const DevTable& t, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s);
constexpr uint64_t kWideWinnerBytes = 32;

// Tables of keys of W = 3..8 64-bit words (ht_long.cu).  Keys are rows of W
// words, 8-byte aligned.  Bucket scheme: `slots` holds one header word per
// slot and the key store one row per slot; Cuckoo: `slots` holds 16-byte
// (digest, row) entries and the key store one row per key placed.
constexpr uint32_t kLongMinWords = 3;
constexpr uint32_t kLongMaxWords = 8;
constexpr uint32_t kLongBucketSlots = 16;
cudaError_t long_find_or_put(const DevTable& t, const void* keys, uint64_t n, uint8_t* is_new, cudaStream_t s);
cudaError_t long_lookup(const DevTable& t, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s);
cudaError_t long_cuckoo_probe(const DevTable& t, const DevScratch& sc, uint32_t parity, const void* keys, uint64_t n,
                              uint8_t* is_new, cudaStream_t s);
cudaError_t long_cuckoo_insert(const DevTable& t, const DevScratch& sc, uint32_t parity, uint64_t max_winners,
                               cudaStream_t s);
cudaError_t long_cuckoo_lookup(const DevTable& t, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s);
// Every stored key of a long-key table of either scheme to keys (rows).
cudaError_t long_export(const DevTable& t, bool cuckoo, void* keys, unsigned long long* count, uint64_t cap,
                        cudaStream_t s);

// Read-only views of a table for the batched form (ht_api.cu).
const DevTable& table_dev(const ht_table* t);
const DevScratch& table_scratch(const ht_table* t);
BucketCfg table_bucket_cfg(const ht_table* t);
ht_scheme table_scheme(const ht_table* t);
uint32_t table_key_width(const ht_table* t);
// Frees an idle table's memory in the order of stream s, without a device
// synchronisation (the caller guarantees no work on the table is pending).
void table_release(ht_table* t, cudaStream_t s);

// State-space successors (ht_bfs.cu).  `model` is a device copy of ht_model.
// count: reservation counter for succ[]; total (nullable): running count of
// successors generated.
cudaError_t successors(int kw, const PreparedModel* model, const void* states, uint64_t n,
                       const unsigned long long* d_n, uint64_t off, void* succ, uint64_t cap,
                       unsigned long long* count, unsigned long long* total, cudaStream_t s);

// ---------------------------------------------------------------------------
// Batched exploration of many models at once (ht_multi.cu).  One step
// processes a slice of every exploration's current BFS level.
// ---------------------------------------------------------------------------
struct MultiWinner;
struct MultiDev {
    uint32_t count;                  // explorations in this group
    uint32_t max_levels;
    const DevTable* tables;          // [count]
    const PreparedModel* models;     // [count]
    void* const* states;             // [count] key-width vectors, level order
    const unsigned long long* states_cap;  // [count]
    const unsigned long long* msucc;       // [count] successors per state bound
    unsigned long long* total;       // [count] states stored (append counters)
    unsigned long long* lo;          // [count] start of the current level
    unsigned long long* hi;          // [count] end of the current level
    unsigned long long* cur;         // [count] next frontier state to expand
    unsigned long long* take;        // [count] states expanded this step
    unsigned long long* work_off;    // [count] prefix of take (states)
    unsigned long long* seg_off;     // [count] start of the successor segment
    unsigned long long* seg_cnt;     // [count] successors written this step
    unsigned long long* gen;         // [count] successors generated in total
    unsigned int* level;             // [count] current level number
    unsigned int* done;              // [count] 1 = finished (2 = hit a limit)
    unsigned long long* level_sizes; // [count * max_levels]
    unsigned long long* work_total;  // [1] states expanded this step, all explorations
    unsigned long long* tiles_total; // [1] 32-key tiles of successors this step
    unsigned int* active;            // [1] explorations not finished
    uint64_t* succ;                  // successor buffer (64-bit words)
    uint64_t succ_cap;
    const unsigned long long* s0;    // [count] initial states
    // Per exploration, the width of its states: 1 = 32-bit words (a model of
    // at most 31 bits), 0 = 64-bit words.  The tables of a group are always
    // addressed as 64-bit key tables: a 32-bit set table holds a key k as
    // the word k (value 0 above it), exactly the word a 64-bit table holds.
    const uint8_t* narrow;           // [count]
    // Cuckoo groups: each table's dedup scratch, a cap on the states one
    // step may expand (0 = none; keeps a step's keys within the table's
    // dedup capacity), and one winner list for all tables of the group.
    const DevScratch* scratch;       // [count] (nullptr for bucket groups)
    const unsigned long long* take_cap;  // [count] (nullptr: no cap)
    MultiWinner* win;                // [win_cap]
    unsigned long long* win_count;   // [1] winners of this step
    uint64_t win_cap;
    // Persistent form: grid barrier words (arrivals, generation), sticky
    // status bits of the run and the number of steps it made.
    unsigned int* bar;               // [2]
    unsigned int* status;            // [1]
    unsigned long long* steps;       // [1]
    uint64_t barrier_ns;             // bound on one barrier wait
    int32_t absent_block;            // failure test: this block leaves before its first barrier (-1: none)
};

// A Cuckoo insertion job of the batched form: the packed word, its claim in
// its table's dedup set, and tag = (exploration << 8) | chain start index.
struct MultiWinner {
    uint64_t word;
    uint32_t spos;
    uint32_t tag;
};

// Status bits of a persistent batched run (MultiDev::status).
enum : uint32_t {
    kMultiTimeout = 1u,     // a grid barrier wait ran past its bound
    kMultiBadInit = 2u,     // an initial state could not be placed (table not empty)
};

// budget: successors the step may generate (the buffer holds budget + slack).
cudaError_t multi_advance(const MultiDev& m, uint64_t budget, cudaStream_t s);
// The whole batched run of one group in one cooperative (co-resident)
// launch: every level of every exploration, with bounded grid barriers
// between the phases of a step (ht_persist.cu).  scheme: HT_BUCKET (c gives
// the bucket shape) or HT_CUCKOO.
cudaError_t multi_persistent(ht_scheme scheme, const BucketCfg& c, const MultiDev& m, uint64_t budget,
                             uint64_t max_steps, uint64_t max_work, uint64_t max_tiles, cudaStream_t s);
cudaError_t multi_successors(int kw, const MultiDev& m, uint64_t max_work, cudaStream_t s);
// Tiles of 32 successors, each against its own exploration's table; new
// states are appended to that exploration's states.
cudaError_t multi_bucket_find_or_put(const BucketCfg& c, const MultiDev& m, uint64_t max_tiles, cudaStream_t s);
// Stores every exploration's initial state (level 0) and resets its cursors.
cudaError_t multi_bucket_init(const BucketCfg& c, const MultiDev& m, cudaStream_t s);

// One packed serving batch: request r's n keys sit at keys[key_off, +n) and
// its tiles of 32 keys start at tile index tile_off (ht_server.cu).
// One item of a packed multi-table find-or-put: n keys (device, the table's
// key width) against tables[table]; flags[i] = is_new (nullable).  Tiles of
// 32 keys are numbered across the items: the item's first is tile_off.
struct WorkDesc {
    const void* keys;
    uint8_t* flags;
    uint64_t n;
    uint64_t tile_off;
    uint32_t table;
    uint32_t pad_;
};
// find-or-put of every item against its own bucket-scheme table (all of the
// key width and bucket shape `c`), one warp per tile, in one launch.
cudaError_t packed_bucket_find_or_put(const BucketCfg& c, const DevTable* tables, const WorkDesc* items,
                                      uint32_t nitems, uint64_t ntiles, cudaStream_t s);

}  // namespace ht
