// Tables of long keys: W = 3..8 64-bit words (192 to 512 bits).  These are
// GPUexplore's multi-word state vectors (Sections 3.2, 4.2) past what one
// 16-byte atomic covers, and the generalisation of Cuckoo hashing to keys of
// any length that Section 7 leaves as future work.
//
// No atomic covers a whole key, so a key cannot go from EMPTY to stored in
// one step; a reader could otherwise see part of a key (the long-element
// race of Section 4.2).  Both schemes therefore claim a short word
// atomically and keep the key's words apart from it.
//
// Bucket scheme: claim, then publish.  A bucket is 16 header words, one
// 128-byte line; the key of slot s is row s of the key store.  A header is
//     EMPTY (all ones) -> BUSY | tag (compare-and-swap claim) -> tag (release store)
// with tag = the key digest's low 62 bits and BUSY = bit 62.  The claimer
// writes the key's words between its two steps and waits on nothing there.
// A reader whose tag matches a header waits (bounded) until the header is
// published, reads it with acquire semantics and then compares the whole
// key.  Claims go in slot order over the slots read as EMPTY, and a claim's
// compare-and-swap returns the header's true state, so the slot-order
// argument of the one-word kernels carries over unchanged: a key is claimed
// in at most one slot, and it sits in bucket h_f only if h_1 .. h_{f-1} were
// full.
//
// Cuckoo: indirection.  A slot is a 16-byte entry (digest, row); the key's
// words sit in row `row` of the key store, written once by the probe kernel
// that elects the key's winner.  Eviction chains move entries with 16-byte
// atomic exchanges and take the next position from the digest alone, so a
// chain reads no key words.  The insert kernel starts after the probe
// kernel has ended, so every row is complete before an entry points to it.
//
// Key-store rows hold the key's words and, for an odd word count, a zero
// word, so every row is 16-byte aligned and is read and written with 16-byte
// accesses.
#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr uint64_t kBusy = 1ull << 62;
constexpr uint64_t kTagMask = kBusy - 1;
constexpr unsigned kFullMask = 0xFFFFFFFFu;
constexpr int kLBS = int(kLongBucketSlots);

struct LongWinner {
    uint64_t digest;
    uint64_t row;
    uint64_t spos;     // its entry in the claim set, cleared by the insert
    uint64_t start;    // the hash index its eviction chain starts at
};
static_assert(sizeof(LongWinner) == kWideWinnerBytes, "winner record size");

// The digest of a key: mix64 chained over its words, seeded with W.  Hash
// positions and tags are taken from the digest; equal digests of different
// keys are told apart by comparing the words.
__device__ __forceinline__ uint64_t digest_of(const uint64_t (&k)[kLongMaxWords], uint32_t W, uint64_t mask) {
    uint64_t h = mix64(0x9E3779B97F4A7C15ull * (W + 1));
#pragma unroll
    for (uint32_t j = 0; j < kLongMaxWords; ++j)
        if (j < W) h = mix64(h ^ k[j]);
    return h & mask;
}

__device__ __forceinline__ void load_key(const uint64_t* __restrict__ keys, uint64_t i, uint32_t W,
                                         uint64_t (&k)[kLongMaxWords]) {
    const uint64_t* p = keys + i * W;
#pragma unroll
    for (uint32_t j = 0; j < kLongMaxWords; ++j) k[j] = j < W ? __ldg(p + j) : 0;
}

// A key of the input batch (W words, 8-byte aligned) against k.
__device__ __forceinline__ bool input_equals(const uint64_t* row, const uint64_t (&k)[kLongMaxWords], uint32_t W) {
    bool eq = true;
#pragma unroll
    for (uint32_t j = 0; j < kLongMaxWords; ++j)
        if (j < W) eq &= __ldg(row + j) == k[j];
    return eq;
}

// A key-store row (RW words, 16-byte aligned; a padding word is 0, as in k)
// against k, with 16-byte loads.
__device__ __forceinline__ bool row_equals(const uint64_t* row, const uint64_t (&k)[kLongMaxWords], uint32_t RW) {
    bool eq = true;
#pragma unroll
    for (uint32_t j = 0; j < kLongMaxWords; j += 2)
        if (j < RW) {
            const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(row + j));
            eq &= v.x == k[j] && v.y == k[j + 1];
        }
    return eq;
}

__device__ __forceinline__ void write_row(uint64_t* row, const uint64_t (&k)[kLongMaxWords], uint32_t RW) {
#pragma unroll
    for (uint32_t j = 0; j < kLongMaxWords; j += 2)
        if (j < RW) *reinterpret_cast<ulonglong2*>(row + j) = make_ulonglong2(k[j], k[j + 1]);
}

// Bit p of x (p < 8) to bit 2p.
__device__ __forceinline__ uint32_t spread8(uint32_t x) {
    x = (x | (x << 4)) & 0x0F0Fu;
    x = (x | (x << 2)) & 0x3333u;
    x = (x | (x << 1)) & 0x5555u;
    return x;
}

__device__ __forceinline__ uint64_t ld_acquire(const uint64_t* p) {
    uint64_t v;
    asm volatile("ld.acquire.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release(uint64_t* p, uint64_t v) {
    asm volatile("st.release.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

// Bucket scheme: does slot `slot`, whose header carries the key's tag, hold
// the key?  Waits until the header is published (bounded: after
// t.spin_limit polls the timeout flag is set and the slot is taken as
// another key's).
__device__ bool slot_holds(const DevTable& t, uint64_t slot, const uint64_t (&k)[kLongMaxWords], uint32_t RW) {
    uint64_t h = ld_acquire(t.slots + slot);
    uint32_t spins = 0;
    while (h & kBusy) {
        if (++spins > t.spin_limit) {
            set_flag(t.ctr, kFlagTimeout);
            return false;
        }
        __nanosleep(100);
        h = ld_acquire(t.slots + slot);
    }
    return row_equals(t.kstore + slot * RW, k, RW);
}

// Bucket-scheme find-or-put (LOOKUP: lookup).  A warp takes 32 keys, one
// per lane.  Each round every lane still searching names its bucket h_f, and
// the warp reads those buckets together: in load j, lanes 8g .. 8g+7 read the
// eight 16-byte pieces of the bucket of lane 4j+g, so a bucket is one
// coalesced 128-byte access; ballots hand each owner its 16-bit masks of
// slots whose tag matches and of EMPTY slots.  The owner then checks the
// matching slots and, if the key is not there and the bucket has EMPTY
// slots, claims them in slot order until one claim succeeds or another copy
// of the key turns up.  A lookup stops at the first bucket with an EMPTY
// slot.
enum : int { kSearching = 0, kClaimed = 1, kFound = 2, kAbsent = 3, kIdle = 4 };

template <bool LOOKUP>
__global__ void __launch_bounds__(kBlock)
long_bucket_kernel(const DevTable t, const uint64_t* __restrict__ keys, uint64_t n, uint8_t* __restrict__ out) {
    const uint32_t W = t.words, RW = t.row_words;
    const int lane = threadIdx.x & 31;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    const uint64_t ntiles = (n + 31) >> 5;
    unsigned long long added = 0;
    for (uint64_t tile = (uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5; tile < ntiles; tile += nwarps) {
        const uint64_t i = tile * 32 + lane;
        const bool act = i < n;
        uint64_t k[kLongMaxWords];
        if (act) {
            load_key(keys, i, W, k);
        } else {
#pragma unroll
            for (uint32_t j = 0; j < kLongMaxWords; ++j) k[j] = 0;
        }
        const uint64_t d = digest_of(k, W, t.digest_mask);
        const uint64_t tag = d & kTagMask;
        int res = act ? kSearching : kIdle;
        uint32_t f = 0;
        // Bounded: a searching lane moves to its next function or settles
        // every round, and there are k functions.
        while (__any_sync(kFullMask, res == kSearching)) {
            const int need = res == kSearching;
            const uint64_t base = need ? hidx(d, t.seed[f], t.nbuckets) * kLBS : 0;
            ulonglong2 v[8];
            int on[8];
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const int owner = 4 * j + (lane >> 3);
                const uint64_t ob = __shfl_sync(kFullMask, base, owner);
                on[j] = __shfl_sync(kFullMask, need, owner);
                v[j] = make_ulonglong2(0, 0);
                if (on[j]) v[j] = __ldcg(reinterpret_cast<const ulonglong2*>(t.slots + ob) + (lane & 7));
            }
            uint32_t match = 0, empty = 0;
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                const uint64_t ot = __shfl_sync(kFullMask, tag, 4 * j + (lane >> 3));
                const bool m0 = on[j] && (v[j].x & ~kBusy) == ot, m1 = on[j] && (v[j].y & ~kBusy) == ot;
                const bool e0 = on[j] && v[j].x == kEmpty, e1 = on[j] && v[j].y == kEmpty;
                const uint32_t bm0 = __ballot_sync(kFullMask, m0), bm1 = __ballot_sync(kFullMask, m1);
                const uint32_t be0 = __ballot_sync(kFullMask, e0), be1 = __ballot_sync(kFullMask, e1);
                if ((lane >> 2) == j) {
                    const int sh = 8 * (lane & 3);
                    match = spread8((bm0 >> sh) & 0xFFu) | (spread8((bm1 >> sh) & 0xFFu) << 1);
                    empty = spread8((be0 >> sh) & 0xFFu) | (spread8((be1 >> sh) & 0xFFu) << 1);
                }
            }
            if (!need) continue;
            while (match && res == kSearching) {
                const int sl = __ffs(match) - 1;
                match &= match - 1;
                if (slot_holds(t, base + sl, k, RW)) res = kFound;
            }
            if (res == kSearching && empty) {
                if (LOOKUP) {
                    res = kAbsent;        // an EMPTY slot: the key would sit in this bucket
                } else {
                    while (empty && res == kSearching) {
                        const int sl = __ffs(empty) - 1;
                        empty &= empty - 1;
                        uint64_t* hdr = t.slots + base + sl;
                        const uint64_t old =
                            atomicCAS(reinterpret_cast<unsigned long long*>(hdr), kEmpty, tag | kBusy);
                        if (old == kEmpty) {
                            write_row(t.kstore + (base + sl) * RW, k, RW);
                            st_release(hdr, tag);
                            res = kClaimed;
                        } else if ((old & ~kBusy) == tag && slot_holds(t, base + sl, k, RW)) {
                            res = kFound;
                        }
                    }
                }
            }
            // Still searching: the bucket is full; the next function, if any.
            if (res == kSearching && ++f >= t.k) res = kAbsent;
        }
        if (!act) continue;
        if (LOOKUP) {
            if (out) out[i] = uint8_t(res == kFound);
        } else {
            if (res == kAbsent) {         // all k buckets full
                set_flag(t.ctr, kFlagDropped);
                atomicAdd(&t.ctr->dropped, 1ull);
            }
            added += res == kClaimed;
            if (out) out[i] = uint8_t(res == kClaimed);
        }
    }
    if (!LOOKUP) {
        for (int o = 16; o; o >>= 1) added += __shfl_down_sync(kFullMask, added, o);
        if (lane == 0 && added) atomicAdd(&t.ctr->size, added);
    }
}

// Cuckoo overflow set: linear probing over 16-byte (digest, row) entries.
__device__ int ovf_insert(const DevTable& t, uint64_t d, uint64_t row) {
    const uint32_t n = t.ovf_slots;
    uint32_t p = uint32_t(mix64(d ^ t.aux_seed) & (n - 1));
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t ol, oh;
        cas128(t.ovf + 2 * uint64_t(p), d, row, ol, oh);
        if (ol == kEmpty && oh == kEmpty) return 1;
        p = (p + 1) & (n - 1);
    }
    return -1;
}

__device__ bool ovf_find(const DevTable& t, uint64_t d, const uint64_t (&k)[kLongMaxWords], uint32_t RW) {
    const uint32_t n = t.ovf_slots;
    uint32_t p = uint32_t(mix64(d ^ t.aux_seed) & (n - 1));
    for (uint32_t i = 0; i < n; ++i) {
        const ulonglong2 e = __ldcg(reinterpret_cast<const ulonglong2*>(t.ovf + 2 * uint64_t(p)));
        if (e.x == kEmpty && e.y == kEmpty) return false;
        if (e.x == d && e.y < t.kstore_rows && row_equals(t.kstore + e.y * RW, k, RW)) return true;
        p = (p + 1) & (n - 1);
    }
    return false;
}

// Cuckoo probe (LOOKUP: lookup), one thread per key.  Section 4.1: the key
// is at one of h_1 .. h_k (or in the overflow set); a chain starts at the
// first slot its probe saw EMPTY (h_1 if none), an evicted entry moves from
// h_a to h_{a+1}, and slots never return to EMPTY, so an EMPTY h_a proves
// the key absent -- and is where a new key's chain starts.  A miss claims the key's
// entry (digest, batch index) in the claim set; an entry of equal digest is
// told apart by comparing the two batch keys.  Winners wait in a per-warp
// stage in shared memory; a flush lists a stage's winners with one atomic on
// the winner count, and a winner listed at position `at` owns key-store row
// ids + at (ids: the rows handed out before this batch, advanced by the
// insert kernel), copies its words there from the batch and writes its
// record.  One atomic per flush instead of two per warp and round: those
// same-address atomics set the probe's pace when every warp issued them.
constexpr int kLongStage = 128;
struct LongStaged {
    uint64_t digest;
    uint64_t i;        // batch index
    uint64_t spos;
    uint64_t start;
};

// The words of batch key i to key-store row `row` (a zero padding word for
// an odd W), with 16-byte stores.
__device__ __forceinline__ void copy_row(uint64_t* row, const uint64_t* __restrict__ key, uint32_t W, uint32_t RW) {
#pragma unroll
    for (uint32_t j = 0; j < kLongMaxWords; j += 2)
        if (j < RW) {
            const uint64_t a = __ldg(key + j);
            const uint64_t b = j + 1 < W ? __ldg(key + j + 1) : 0;
            *reinterpret_cast<ulonglong2*>(row + j) = make_ulonglong2(a, b);
        }
}

template <bool LOOKUP>
__global__ void __launch_bounds__(kBlock)
long_cuckoo_probe_kernel(const DevTable t, const DevScratch sc, uint32_t parity, const uint64_t* __restrict__ keys,
                         uint64_t n, uint8_t* __restrict__ out) {
    const uint32_t W = t.words, RW = t.row_words;
    const uint32_t ovf_used = __ldcg(&t.ctr->ovf_used);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t rounds = (n + stride - 1) / stride;      // warp-uniform trip count
    const uint64_t dseed = t.aux_seed * 3 + 1;
    const int lane = threadIdx.x & 31;
    LongWinner* win = reinterpret_cast<LongWinner*>(sc.win);
    unsigned long long probes = 0;
    constexpr int kStage = LOOKUP ? 1 : kLongStage;
    __shared__ LongStaged s_win[kBlock / 32][kStage];
    LongStaged* stage = s_win[threadIdx.x >> 5];
    uint32_t pend = 0;
    const uint64_t row_base = LOOKUP ? 0 : __ldcg(&t.ctr->ids);
    // Lists the staged winners.  A winner past the list's capacity or past
    // the key store (more keys than the table holds) gives its claim back
    // with one 16-byte atomic (other threads may be comparing against it),
    // is reported dropped and loses its flag; inside the list it leaves a
    // record with row = EMPTY that the insert kernel skips.
    auto flush = [&]() {
        __syncwarp();
        if (pend) {
            unsigned int b = 0;
            if (lane == 0) b = atomicAdd(&t.ctr->winners[parity], pend);
            b = __shfl_sync(kFullMask, b, 0);
            for (uint32_t j = lane; j < pend; j += 32) {
                const LongStaged e = stage[j];
                const uint64_t at = uint64_t(b) + j;
                const uint64_t row = row_base + at;
                const bool listed = at < sc.win_cap, stored = listed && row < t.kstore_rows;
                if (stored) copy_row(t.kstore + row * RW, keys + e.i * W, W, RW);
                if (listed) {
                    LongWinner wn;
                    wn.digest = e.digest;
                    wn.row = stored ? row : kEmpty;
                    wn.spos = e.spos;
                    wn.start = e.start;
                    win[at] = wn;
                }
                if (!stored) {
                    uint64_t ol, oh;
                    exch128(sc.set + 2 * e.spos, kEmpty, kEmpty, ol, oh);
                    set_flag(t.ctr, kFlagDropped);
                    atomicAdd(&t.ctr->dropped, 1ull);
                    if (out) out[e.i] = 0;
                }
            }
        }
        __syncwarp();
        pend = 0;
    };
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = r * stride + tid;
        const bool act = i < n;
        uint64_t k[kLongMaxWords];
        uint64_t d = 0;
        bool found = false;
        uint32_t start = 0;            // the first function whose slot was seen EMPTY (0: none)
        if (act) {
            load_key(keys, i, W, k);
            d = digest_of(k, W, t.digest_mask);
            for (uint32_t a = 0; a < t.k; ++a) {
                const ulonglong2 e =
                    __ldcg(reinterpret_cast<const ulonglong2*>(t.slots + 2 * hidx(d, t.seed[a], t.nslots)));
                ++probes;
                if (e.x == kEmpty && e.y == kEmpty) {
                    start = a;         // the key is not past it; its chain starts there
                    break;
                }
                if (e.x == d && e.y < t.kstore_rows && row_equals(t.kstore + e.y * RW, k, RW)) {
                    found = true;
                    break;
                }
            }
            if (!found && ovf_used) found = ovf_find(t, d, k, RW);
        }
        if (LOOKUP) {
            if (act && out) out[i] = uint8_t(found);
            continue;
        }
        bool winner = false;
        uint64_t spos = 0;
        if (act && !found) {
            spos = mix64(d ^ dseed) & sc.mask;
            bool settled = false;
            for (uint64_t p = 0; p <= sc.mask; ++p) {
                uint64_t ol, oh;
                cas128(sc.set + 2 * spos, d, i, ol, oh);
                if (ol == kEmpty && oh == kEmpty) {
                    winner = settled = true;
                    break;
                }
                if (ol == d && oh < n && input_equals(keys + oh * W, k, W)) {
                    settled = true;                        // another copy of the key won
                    break;
                }
                spos = (spos + 1) & sc.mask;
            }
            if (!settled) {                                // more distinct misses than the set holds
                set_flag(t.ctr, kFlagDropped);
                atomicAdd(&t.ctr->dropped, 1ull);
            }
        }
        if (act && out) out[i] = uint8_t(winner);
        const unsigned wm = __ballot_sync(kFullMask, winner);
        if (wm) {
            if (pend + __popc(wm) > uint32_t(kStage)) flush();
            if (winner) {
                LongStaged& e = stage[pend + __popc(wm & ((1u << lane) - 1))];
                e.digest = d;
                e.i = i;
                e.spos = spos;
                e.start = t.chain_h1 ? 0u : start;
            }
            pend += __popc(wm);
        }
    }
    if (!LOOKUP) {
        flush();
        for (int o = 16; o; o >>= 1) probes += __shfl_down_sync(kFullMask, probes, o);
        if (lane == 0 && probes) atomicAdd(&t.ctr->probes, probes);
    }
}

// Eviction chains of the winners' (digest, row) entries; each thread keeps
// four chains in flight and refills a chain that ends with its next winner.
__global__ void __launch_bounds__(kBlock)
long_cuckoo_insert_kernel(const DevTable t, const DevScratch sc, uint32_t parity, uint64_t max_winners) {
    constexpr int U = 4;
    const uint64_t count = min(uint64_t(__ldcg(&t.ctr->winners[parity])), max_winners);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        t.ctr->winners[parity ^ 1u] = 0;
        // Rows ids .. ids + count - 1 went to this batch's listed winners
        // (those past the key store were dropped); no other thread of this
        // kernel reads ids, and the next probe starts after it ends.
        const unsigned long long ids = t.ctr->ids;
        t.ctr->ids = min(uint64_t(ids) + count, t.kstore_rows);
    }
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const LongWinner* win = reinterpret_cast<const LongWinner*>(sc.win);
    unsigned long long placed = 0, exchanges = 0;
    uint64_t next = tid;
    uint64_t dg[U], row[U], pos[U];
    uint32_t evictions[U];
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        live[u] = false;
        dg[u] = row[u] = pos[u] = 0;
        evictions[u] = 0;
    }
    // Bounded: each winner is taken once and its chain ends after at most
    // max_evictions + 1 exchanges.
    for (;;) {
        bool any = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            while (!live[u] && next < count) {
                const LongWinner wn = win[next];
                next += stride;
                if (wn.row >= t.kstore_rows) continue;     // dropped in the probe; its claim is back
                sc.set[2 * wn.spos] = kEmpty;              // leave the claim set empty for the next batch
                sc.set[2 * wn.spos + 1] = kEmpty;
                dg[u] = wn.digest;
                row[u] = wn.row;
                pos[u] = hidx(wn.digest, t.seed[wn.start < t.k ? wn.start : 0], t.nslots);
                evictions[u] = 0;
                live[u] = true;
            }
            any |= live[u];
        }
        if (!any) break;
        ulonglong2 old[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (live[u]) {
                uint64_t ol, oh;
                exch128(t.slots + 2 * pos[u], dg[u], row[u], ol, oh);
                old[u] = make_ulonglong2(ol, oh);
            }
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!live[u]) continue;
            ++exchanges;
            if (old[u].x == kEmpty && old[u].y == kEmpty) {
                live[u] = false;
                ++placed;
                continue;
            }
            dg[u] = old[u].x;
            row[u] = old[u].y;
            if (++evictions[u] > t.max_evict) {
                // The chain hit the eviction bound: the held entry goes to the overflow set.
                if (ovf_insert(t, dg[u], row[u]) == 1) {
                    ++placed;
                    atomicAdd(&t.ctr->ovf_used, 1u);
                    set_flag(t.ctr, kFlagRebuild);
                } else {
                    set_flag(t.ctr, kFlagDropped);
                    atomicAdd(&t.ctr->dropped, 1ull);
                }
                live[u] = false;
                continue;
            }
            // Section 4.1: the evicted entry sat at h_a(digest) = pos, a the
            // smallest such index; it moves on to h_{a+1} (after h_k: h_1).
            uint32_t a = 0;
            for (; a + 1 < t.k; ++a)
                if (hidx(dg[u], t.seed[a], t.nslots) == pos[u]) break;
            const uint32_t nxt = (a + 1 == t.k) ? 0u : a + 1;
            pos[u] = hidx(dg[u], t.seed[nxt], t.nslots);
        }
    }
    for (int o = 16; o; o >>= 1) {
        placed += __shfl_down_sync(kFullMask, placed, o);
        exchanges += __shfl_down_sync(kFullMask, exchanges, o);
    }
    if ((threadIdx.x & 31) == 0 && placed) atomicAdd(&t.ctr->size, placed);
    if ((threadIdx.x & 31) == 0 && exchanges) atomicAdd(&t.ctr->exchanges, exchanges);
}

// Export: the rows of every published header (bucket scheme) or every
// entry of the table and the overflow set (Cuckoo), appended per warp.
__global__ void __launch_bounds__(kBlock)
long_export_kernel(const DevTable t, bool cuckoo, uint64_t* __restrict__ out, unsigned long long* __restrict__ count,
                   uint64_t cap) {
    const uint32_t W = t.words, RW = t.row_words;
    const uint64_t total = t.nslots + (cuckoo ? t.ovf_slots : 0);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t rounds = (total + stride - 1) / stride;
    const int lane = threadIdx.x & 31;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t s = r * stride + tid;
        bool have = false;
        uint64_t src = 0;
        if (s < total) {
            if (!cuckoo) {
                const uint64_t h = __ldcg(reinterpret_cast<const unsigned long long*>(t.slots + s));
                have = (h >> 62) == 0;
                src = s;
            } else {
                const uint64_t* e = s < t.nslots ? t.slots + 2 * s : t.ovf + 2 * (s - t.nslots);
                const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(e));
                have = !(v.x == kEmpty && v.y == kEmpty);
                src = v.y;
            }
        }
        const unsigned m = __ballot_sync(kFullMask, have);
        if (!m) continue;
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(count, (unsigned long long)__popc(m));
        b = __shfl_sync(kFullMask, b, 0);
        const uint64_t at = b + __popc(m & ((1u << lane) - 1));
        if (have && at < cap && src < t.kstore_rows) {
            const uint64_t* row = t.kstore + src * RW;
            for (uint32_t j = 0; j < W; ++j) out[at * W + j] = __ldcg(reinterpret_cast<const unsigned long long*>(row + j));
        }
    }
}

}  // namespace

cudaError_t long_find_or_put(const DevTable& t, const void* keys, uint64_t n, uint8_t* is_new, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ProfScope ps(kKBucketFop, s);
    auto k = long_bucket_kernel<false>;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, static_cast<const uint64_t*>(keys), n, is_new);
    return cudaGetLastError();
}

cudaError_t long_lookup(const DevTable& t, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ProfScope ps(kKBucketLookup, s);
    auto k = long_bucket_kernel<true>;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, static_cast<const uint64_t*>(keys), n, found);
    return cudaGetLastError();
}

cudaError_t long_cuckoo_probe(const DevTable& t, const DevScratch& sc, uint32_t parity, const void* keys, uint64_t n,
                              uint8_t* is_new, cudaStream_t s) {
    ProfScope ps(kKCuckooProbe, s);
    auto k = long_cuckoo_probe_kernel<false>;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, sc, parity, static_cast<const uint64_t*>(keys), n,
                                                              is_new);
    return cudaGetLastError();
}

cudaError_t long_cuckoo_insert(const DevTable& t, const DevScratch& sc, uint32_t parity, uint64_t max_winners,
                               cudaStream_t s) {
    ProfScope ps(kKCuckooInsert, s);
    auto k = long_cuckoo_insert_kernel;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, sc, parity, max_winners);
    return cudaGetLastError();
}

cudaError_t long_cuckoo_lookup(const DevTable& t, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ProfScope ps(kKCuckooLookup, s);
    DevScratch none{};
    auto k = long_cuckoo_probe_kernel<true>;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, none, 0u, static_cast<const uint64_t*>(keys), n,
                                                              found);
    return cudaGetLastError();
}

cudaError_t long_export(const DevTable& t, bool cuckoo, void* keys, unsigned long long* count, uint64_t cap,
                        cudaStream_t s) {
    ProfScope ps(kKExport, s);
    auto k = long_export_kernel;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, cuckoo, static_cast<uint64_t*>(keys), count, cap);
    return cudaGetLastError();
}

}  // namespace ht
