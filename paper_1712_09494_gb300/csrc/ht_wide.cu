// Bucket-scheme tables of 128-bit keys (state vectors wider than 64 bits;
// the multi-word vectors GPUexplore stores, Sections 3.2 and 4.2).
//
// A slot is 16 bytes: the key's low word, then its high word.  EMPTY is all
// ones in both; a key's top bit (bit 63 of the high word) is reserved, so no
// key is EMPTY.  A bucket is 8 slots (one 128-byte line) read by G lanes.
// A claim is one 16-byte compare-and-swap (atom.cas.b128), so a slot goes
// from EMPTY to a key at once and never changes again.
//
// Reads are plain 16-byte loads, which the memory model does not make
// atomic with respect to that CAS: a reader may see half of a key being
// written.  Since the only write is EMPTY -> key, a torn read always shows
// at least one all-ones word.  So a slot read with neither word all ones is
// a complete key (and stays so); a slot with both all ones, or exactly one,
// is a claim candidate whose true content the claiming CAS returns.  Claims
// go in slot order over the candidates (the slot-order argument of the
// 64-bit kernels: a key is claimed in at most one slot), and only the CAS
// result decides, so stale or torn reads cannot duplicate a key.
#include "ht_internal.cuh"

namespace ht {
namespace {

constexpr int kWideBS = 8;                // slots per bucket
constexpr uint64_t kOnes = ~0ull;
constexpr unsigned kFull = 0xFFFFFFFFu;

__device__ __forceinline__ bool wide_reserved(uint64_t hi) { return (hi >> 63) != 0; }

// The bucket hash of a 128-bit key: the 64-bit family applied to a fold of
// both words (mix64 of the high word, xored into the low word).
__device__ __forceinline__ uint64_t wide_fold(uint64_t lo, uint64_t hi) {
    return lo ^ mix64(hi ^ 0xD1B54A32D192ED03ull);
}

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
        : "l"(kOnes), "l"(kOnes), "l"(new_lo), "l"(new_hi), "l"(addr)
        : "memory");
}

// Slot classes of a read: 2 = a complete key, 1 = a claim candidate.
__device__ __forceinline__ int slot_class(uint64_t lo, uint64_t hi) {
    return (lo != kOnes && hi != kOnes) ? 2 : 1;
}

// Overflow set: linear probing over 16-byte entries; returns 1 stored,
// 0 present, -1 full.  One lane per key.
__device__ int wide_ovf_insert(const DevTable& t, uint64_t lo, uint64_t hi) {
    const uint32_t n = t.ovf_slots;
    uint32_t p = uint32_t(mix64(wide_fold(lo, hi) ^ t.aux_seed) & (n - 1));
    for (uint32_t i = 0; i < n; ++i) {
        uint64_t* s = t.ovf + 2 * uint64_t(p);
        const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(s));
        if (slot_class(v.x, v.y) == 2) {
            if (v.x == lo && v.y == hi) return 0;
        } else {
            uint64_t ol, oh;
            cas128(s, lo, hi, ol, oh);
            if (ol == kOnes && oh == kOnes) return 1;
            if (ol == lo && oh == hi) return 0;
        }
        p = (p + 1) & (n - 1);
    }
    return -1;
}

__device__ bool wide_ovf_find(const DevTable& t, uint64_t lo, uint64_t hi) {
    const uint32_t n = t.ovf_slots;
    uint32_t p = uint32_t(mix64(wide_fold(lo, hi) ^ t.aux_seed) & (n - 1));
    for (uint32_t i = 0; i < n; ++i) {
        const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(t.ovf + 2 * uint64_t(p)));
        if (v.x == kOnes && v.y == kOnes) return false;
        if (v.x == lo && v.y == hi) return true;
        p = (p + 1) & (n - 1);
    }
    return false;
}

// find-or-put: a warp takes 32 keys (lane l loads key l); in round q group
// g (G lanes) serves key q*(32/G)+g through buckets h_1, h_2, ... until the
// key is found, claimed, or (all k buckets full) placed in the overflow set.
// APPEND: the keys new to the table also go to new_out at *new_count
// (staged per warp in shared memory; entries past new_cap not written).
// d_n (nullable): the batch size produced on the device, at most n.
template <int G, bool LOOKUP, bool APPEND>
__global__ void __launch_bounds__(kBlock)
wide_kernel(const DevTable t, const ulonglong2* __restrict__ keys, uint64_t n,
            const unsigned long long* __restrict__ d_n, uint8_t* __restrict__ out,
            ulonglong2* __restrict__ new_out, unsigned long long* __restrict__ new_count, uint64_t new_cap) {
    constexpr int SPL = kWideBS / G;
    constexpr int GPW = 32 / G;
    constexpr uint32_t kGMask = (1u << G) - 1u;
    if (d_n) n = min(n, uint64_t(__ldcg(d_n)));
    const int lane = threadIdx.x & 31;
    const int grp = lane / G, sub = lane % G, gbase = grp * G;
    const uint64_t nwarps = (uint64_t(gridDim.x) * blockDim.x) >> 5;
    unsigned long long stored = 0;
    __shared__ ulonglong2 s_new[APPEND ? kBlock / 32 : 1][APPEND ? kStageCap : 1];
    WarpStage<ulonglong2, kStageCap> stage(s_new[APPEND ? (threadIdx.x >> 5) : 0]);
    for (uint64_t base = ((uint64_t(blockIdx.x) * blockDim.x + threadIdx.x) >> 5) * 32; base < n;
         base += nwarps * 32) {
        const bool mine = base + lane < n;
        ulonglong2 mk = make_ulonglong2(0, 0);
        if (mine) mk = keys[base + lane];
        const bool myok = mine && !wide_reserved(mk.y);
        if (mine && !myok) set_flag(t.ctr, kFlagInvalidKey);
        uint32_t res_all = 0;                       // bit q: the group's key of round q was stored / found
        for (int q = 0; q < G; ++q) {
            const int kidx = q * GPW + grp;
            const uint64_t lo = __shfl_sync(kFull, mk.x, kidx);
            const uint64_t hi = __shfl_sync(kFull, mk.y, kidx);
            const bool ok = __shfl_sync(kFull, myok, kidx);
            const uint64_t fold = wide_fold(lo, hi);
            uint32_t f = 0;
            uint64_t b = hidx(fold, t.seed[0], t.nbuckets);
            int state = ok ? 0 : 3;                 // 0 read, 1 decide, 2 spill, 3 done
            uint32_t cand = 0, match = 0, res = 0;
            // Bounded: each pass ends the key, spends a candidate slot of
            // this bucket (<= 8) or moves to the next of k buckets.
            while (__any_sync(kFull, state != 3)) {
                if (state == 0) {
                    cand = match = 0;
#pragma unroll
                    for (int j = 0; j < SPL; ++j) {
                        const ulonglong2 v = __ldcg(reinterpret_cast<const ulonglong2*>(
                            t.slots + 2 * (b * kWideBS + uint64_t(sub * SPL + j))));
                        if (LOOKUP) {
                            // No writer runs beside a lookup: reads are
                            // complete, and only all ones is empty.
                            if (v.x == lo && v.y == hi) match |= 1u << j;
                            else if (v.x == kOnes && v.y == kOnes) cand |= 1u << j;
                        } else if (slot_class(v.x, v.y) == 2) {
                            if (v.x == lo && v.y == hi) match |= 1u << j;
                        } else {
                            cand |= 1u << j;
                        }
                    }
                    state = 1;
                }
                const uint32_t M = (__ballot_sync(kFull, state == 1 && match != 0) >> gbase) & kGMask;
                const uint32_t C = (__ballot_sync(kFull, state == 1 && cand != 0) >> gbase) & kGMask;
                int owner = -1;
                if (state == 1) {
                    if (M) {
                        state = 3;
                        res = LOOKUP ? 1u : 0u;
                    } else if (C) {
                        if (LOOKUP) {
                            // An empty slot: a key moves on to its next
                            // bucket only from a full one, so it is absent.
                            state = 3;
                            res = 0;
                        } else {
                            owner = gbase + __ffs(C) - 1;
                        }
                    } else if (++f < t.k) {
                        b = hidx(fold, t.seed[f], t.nbuckets);
                        state = 0;
                    } else {
                        state = 2;
                    }
                }
                uint32_t code = 0;
                if (!LOOKUP && lane == owner) {
                    const int j = __ffs(cand) - 1;
                    uint64_t ol, oh;
                    cas128(t.slots + 2 * (b * kWideBS + uint64_t(sub * SPL + j)), lo, hi, ol, oh);
                    code = (ol == kOnes && oh == kOnes) ? 0u : ((ol == lo && oh == hi) ? 1u : 2u);
                    cand &= ~(1u << j);
                }
                code = __shfl_sync(kFull, code, owner >= 0 ? owner : lane);
                if (owner >= 0 && code != 2u) {
                    state = 3;
                    res = code == 0u;
                }
                if (state == 2) {
                    if (sub == 0) {
                        if (LOOKUP) {
                            res = wide_ovf_find(t, lo, hi) ? 1u : 0u;
                        } else {
                            const int r = wide_ovf_insert(t, lo, hi);
                            res = r == 1;
                            if (r == 1) atomicAdd(&t.ctr->ovf_used, 1u);
                            if (r < 0) {
                                set_flag(t.ctr, kFlagDropped);
                                atomicAdd(&t.ctr->dropped, 1ull);
                            }
                        }
                    }
                    state = 3;
                }
            }
            res = __shfl_sync(kFull, res, gbase);
            res_all |= res << q;
        }
        const uint32_t my = (__shfl_sync(kFull, res_all, (lane % GPW) * G) >> (lane / GPW)) & 1u;
        if (mine && out) out[base + lane] = uint8_t(my);
        if (APPEND) stage.push(mine && my, mk, new_out, new_count, new_cap);
        if (!LOOKUP) stored += __popc(__ballot_sync(kFull, my != 0));
    }
    if (APPEND) stage.flush(new_out, new_count, new_cap);
    if (!LOOKUP && lane == 0 && stored) atomicAdd(&t.ctr->size, stored);
}

// Every stored key (table, then overflow set) to out[2 * i .. 2 * i + 1].
__global__ void __launch_bounds__(kBlock)
wide_export_kernel(const DevTable t, uint64_t* __restrict__ out, unsigned long long* __restrict__ count,
                   uint64_t cap) {
    const uint64_t total = t.nslots + t.ovf_slots;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t rounds = (total + stride - 1) / stride;
    const int lane = threadIdx.x & 31;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = r * stride + uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
        ulonglong2 v = make_ulonglong2(kOnes, kOnes);
        if (i < t.nslots) v = __ldcg(reinterpret_cast<const ulonglong2*>(t.slots + 2 * i));
        else if (i < total) v = __ldcg(reinterpret_cast<const ulonglong2*>(t.ovf + 2 * (i - t.nslots)));
        const bool keep = !(v.x == kOnes && v.y == kOnes);
        const unsigned m = __ballot_sync(kFull, keep);
        if (!m) continue;
        unsigned long long b = 0;
        if (lane == 0) b = atomicAdd(count, (unsigned long long)__popc(m));
        b = __shfl_sync(kFull, b, 0);
        const unsigned long long at = b + __popc(m & ((1u << lane) - 1));
        if (keep && at < cap) {
            out[2 * at] = v.x;
            out[2 * at + 1] = v.y;
        }
    }
}

template <int G, bool LOOKUP, bool APPEND>
cudaError_t launch_wide(const DevTable& t, const void* keys, uint64_t n, const unsigned long long* d_n,
                        uint8_t* out, void* new_out, unsigned long long* new_count, uint64_t new_cap,
                        cudaStream_t s) {
    auto k = wide_kernel<G, LOOKUP, APPEND>;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, static_cast<const ulonglong2*>(keys), n, d_n, out,
                                                              static_cast<ulonglong2*>(new_out), new_count, new_cap);
    return cudaGetLastError();
}

}  // namespace

cudaError_t wide_find_or_put(int lanes, const DevTable& t, const void* keys, uint64_t n,
                             const unsigned long long* d_n, uint8_t* is_new, void* new_out,
                             unsigned long long* new_count, uint64_t new_cap, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ProfScope ps(kKBucketFop, s);
#define L(G)                                                                                                 \
    return new_out ? launch_wide<G, false, true>(t, keys, n, d_n, is_new, new_out, new_count, new_cap, s)     \
                   : launch_wide<G, false, false>(t, keys, n, d_n, is_new, nullptr, nullptr, 0, s);
    if (lanes == 2) L(2)
    if (lanes == 4) L(4)
#undef L
    return cudaErrorInvalidValue;
}

cudaError_t wide_lookup(int lanes, const DevTable& t, const void* keys, uint64_t n, uint8_t* found,
                        cudaStream_t s) {
    if (!n) return cudaSuccess;
    ProfScope ps(kKBucketLookup, s);
    if (lanes == 2) return launch_wide<2, true, false>(t, keys, n, nullptr, found, nullptr, nullptr, 0, s);
    if (lanes == 4) return launch_wide<4, true, false>(t, keys, n, nullptr, found, nullptr, nullptr, 0, s);
    return cudaErrorInvalidValue;
}

cudaError_t wide_export(const DevTable& t, void* keys, unsigned long long* count, uint64_t cap, cudaStream_t s) {
    ProfScope ps(kKExport, s);
    auto k = wide_export_kernel;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, static_cast<uint64_t*>(keys), count, cap);
    return cudaGetLastError();
}

}  // namespace ht
