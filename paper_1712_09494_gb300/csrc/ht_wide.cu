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

// ---------------------------------------------------------------------------
// Cuckoo hashing of 128-bit keys (Section 4.1 with 16-byte slots; the
// generalisation to longer keys is the paper's own future work, Section 7).
// The same two kernels as for 64-bit keys.  The probe finds keys in h_1
// (then h_2..h_k when h_1 is occupied); an absent key that met a slot
// without a complete key stores itself there with a 16-byte CAS from EMPTY,
// going on in slot order when another key took it first; a key whose k
// slots all hold complete keys claims its key in a claim set of 16-byte
// entries, and the one claimant runs an eviction chain from h_1 with
// 16-byte atomic exchanges in the insert kernel.
//
// The probe's reads are plain 16-byte loads while its CASes write: a read
// can show half of a key being stored (one all-ones word).  As in the
// bucket kernels, only a read with neither word all ones counts as a
// complete key (found, or occupied by another key); any other read is a
// candidate that the CAS settles, returning the slot's true content.  So a
// copy never passes a slot where another copy is storing its key, the
// slot-order argument holds, and a copy that saw k complete keys read each
// slot after it was filled (no copy stores the key in the table during the
// probe).  Lookups run with no writer, so their reads are complete.

struct WideWinner {
    uint64_t lo, hi;
    uint64_t spos;                        // its claim-set entry (cleared by the insert)
    uint64_t start;                       // the hash index its eviction chain starts at
};
// The start field of a record whose key the probe stored itself (listed
// only for a caller that collects the new keys).
constexpr uint64_t kWidePlaced = ~0ull;

constexpr int kWU = 4;                    // keys (probe) or chains (insert) in flight per thread

#ifndef HT_WIDE_PROBE_MIN_BLOCKS
#define HT_WIDE_PROBE_MIN_BLOCKS 2
#endif
template <bool LOOKUP>
__global__ void __launch_bounds__(kBlock, HT_WIDE_PROBE_MIN_BLOCKS)
wide_cuckoo_probe_kernel(const DevTable t, const DevScratch sc, uint32_t parity, const ulonglong2* __restrict__ keys,
                         uint64_t n, const unsigned long long* __restrict__ d_n, uint64_t off,
                         uint8_t* __restrict__ out, bool list_stored) {
    if (d_n) {
        const uint64_t total = __ldcg(d_n);
        n = total > off ? min(n, total - off) : 0;
    }
    const uint32_t ovf_used = __ldcg(&t.ctr->ovf_used);
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t rounds = (n + stride * kWU - 1) / (stride * kWU);   // warp-uniform trip count
    const int lane = threadIdx.x & 31;
    const uint64_t dseed = t.aux_seed * 3 + 1;
    WideWinner* win = reinterpret_cast<WideWinner*>(sc.win);
    unsigned long long stored_here = 0, cas_count = 0;
    for (uint64_t r = 0; r < rounds; ++r) {
        ulonglong2 k[kWU];
        uint64_t fold[kWU];
        bool act[kWU], ok[kWU], found[kWU], more[kWU], cand[kWU];
        uint32_t at[kWU];                     // the slot a search stopped at (a candidate)
#pragma unroll
        for (int u = 0; u < kWU; ++u) {
            const uint64_t i = (r * kWU + u) * stride + tid;
            act[u] = i < n;
            k[u] = act[u] ? keys[i] : make_ulonglong2(0, 0);
            ok[u] = act[u] && !wide_reserved(k[u].y);
            if (act[u] && !ok[u]) set_flag(t.ctr, kFlagInvalidKey);
            fold[u] = wide_fold(k[u].x, k[u].y);
            found[u] = cand[u] = false;
            more[u] = ok[u];
            at[u] = 0;
        }
        // h_1, h_2, ... one function at a time (16-byte words of four keys in
        // flight per thread), each key until it is found or meets a slot
        // without a complete key.  An EMPTY h_a proves the key absent (a key
        // stored at h_j has h_1..h_(j-1) occupied: slots never return to
        // EMPTY and a key is stored only past slots seen occupied).
        for (uint32_t a = 0; a < t.k; ++a) {
            ulonglong2 w[kWU];
#pragma unroll
            for (int u = 0; u < kWU; ++u)
                if (more[u])
                    w[u] = __ldcg(reinterpret_cast<const ulonglong2*>(t.slots + 2 * hidx(fold[u], t.seed[a], t.nslots)));
#pragma unroll
            for (int u = 0; u < kWU; ++u) {
                if (!more[u]) continue;
                const bool same = w[u].x == k[u].x && w[u].y == k[u].y;
                const bool empty = w[u].x == kOnes && w[u].y == kOnes;
                if (LOOKUP ? same : (same && slot_class(w[u].x, w[u].y) == 2)) {
                    found[u] = true;
                    more[u] = false;
                } else if (LOOKUP ? empty : slot_class(w[u].x, w[u].y) == 1) {
                    cand[u] = true;
                    at[u] = a;
                    more[u] = false;
                }
            }
        }
        if (ovf_used) {
#pragma unroll
            for (int u = 0; u < kWU; ++u)
                if (ok[u] && !found[u]) found[u] = wide_ovf_find(t, k[u].x, k[u].y);
        }
        if constexpr (LOOKUP) {
#pragma unroll
            for (int u = 0; u < kWU; ++u) {
                const uint64_t i = (r * kWU + u) * stride + tid;
                if (act[u] && out) out[i] = uint8_t(found[u]);
            }
        } else {
        // Stores: a CAS from EMPTY at the candidate slot, on in slot order
        // while the CAS returns another complete key (with t.chain_h1 only
        // at h_1, Section 4.1's start).  The rest claim.
        bool placed[kWU], claim[kWU], pend[kWU];
#pragma unroll
        for (int u = 0; u < kWU; ++u) {
            const bool miss = ok[u] && !found[u];
            pend[u] = miss && cand[u] && (!t.chain_h1 || at[u] == 0);
            claim[u] = miss && !pend[u];
            placed[u] = false;
        }
        for (uint32_t pass = 0; pass < t.k; ++pass) {
            bool any = false;
#pragma unroll
            for (int u = 0; u < kWU; ++u) any |= pend[u];
            if (!__any_sync(kFull, any)) break;
            ulonglong2 cw[kWU];
#pragma unroll
            for (int u = 0; u < kWU; ++u)
                if (pend[u]) {
                    uint64_t ol, oh;
                    cas128(t.slots + 2 * hidx(fold[u], t.seed[at[u]], t.nslots), k[u].x, k[u].y, ol, oh);
                    cw[u] = make_ulonglong2(ol, oh);
                    ++cas_count;
                }
#pragma unroll
            for (int u = 0; u < kWU; ++u) {
                if (!pend[u]) continue;
                if (cw[u].x == kOnes && cw[u].y == kOnes) {
                    placed[u] = true;
                    pend[u] = false;
                } else if (cw[u].x == k[u].x && cw[u].y == k[u].y) {
                    found[u] = true;                     // another copy stored it
                    pend[u] = false;
                } else if (t.chain_h1 || at[u] + 1 >= t.k) {
                    claim[u] = true;                     // every slot holds another key now
                    pend[u] = false;
                } else {
                    ++at[u];
                }
            }
        }
        // In-batch dedup of the keys with all k slots full: one winner per
        // distinct key; every such miss's first claim together, collisions
        // probe on.
        bool winner[kWU];
        uint64_t spos[kWU];
        ulonglong2 old[kWU];
#pragma unroll
        for (int u = 0; u < kWU; ++u) {
            winner[u] = placed[u];
            spos[u] = mix64(fold[u] ^ dseed) & sc.mask;
            old[u] = make_ulonglong2(0, 0);
            if (claim[u]) {
                uint64_t ol, oh;
                cas128(sc.set + 2 * spos[u], k[u].x, k[u].y, ol, oh);
                old[u] = make_ulonglong2(ol, oh);
            }
        }
#pragma unroll
        for (int u = 0; u < kWU; ++u) {
            if (!claim[u]) continue;
            bool settled = false;
            for (uint64_t probe = 0; probe <= sc.mask; ++probe) {
                if (probe) {
                    uint64_t ol, oh;
                    cas128(sc.set + 2 * spos[u], k[u].x, k[u].y, ol, oh);
                    old[u] = make_ulonglong2(ol, oh);
                }
                if (old[u].x == kOnes && old[u].y == kOnes) {
                    winner[u] = settled = true;
                    break;
                }
                if (old[u].x == k[u].x && old[u].y == k[u].y) {
                    settled = true;                      // another copy of the key won
                    break;
                }
                spos[u] = (spos[u] + 1) & sc.mask;
            }
            if (!settled) {                              // more distinct misses than the table holds
                set_flag(t.ctr, kFlagDropped);
                atomicAdd(&t.ctr->dropped, 1ull);
            }
        }
        // List the round's claim winners (and the stored keys, for a caller
        // that collects the new keys): one atomic per warp.
        bool listed[kWU];
        unsigned wm[kWU];
        unsigned total = 0;
#pragma unroll
        for (int u = 0; u < kWU; ++u) {
            listed[u] = winner[u] && (!placed[u] || list_stored);
            stored_here += (placed[u] && !list_stored) ? 1u : 0u;
            wm[u] = __ballot_sync(kFull, listed[u]);
            total += __popc(wm[u]);
        }
        unsigned int b = 0;
        if (total) {
            if (lane == 0) b = atomicAdd(&t.ctr->winners[parity], total);
            b = __shfl_sync(kFull, b, 0);
        }
#pragma unroll
        for (int u = 0; u < kWU; ++u) {
            const uint64_t i = (r * kWU + u) * stride + tid;
            bool is_new = winner[u];
            if (listed[u]) {
                const uint64_t p = uint64_t(b) + __popc(wm[u] & ((1u << lane) - 1));
                if (p < sc.win_cap) {
                    WideWinner wn;
                    wn.lo = k[u].x;
                    wn.hi = k[u].y;
                    wn.spos = spos[u];
                    wn.start = placed[u] ? kWidePlaced : 0u;
                    win[p] = wn;
                } else if (placed[u]) {
                    atomicAdd(&t.ctr->size, 1ull);       // stored already; it holds no claim
                } else {                                 // more winners than the table holds
                    is_new = false;
                    sc.set[2 * spos[u]] = kOnes;
                    sc.set[2 * spos[u] + 1] = kOnes;
                    set_flag(t.ctr, kFlagDropped);
                    atomicAdd(&t.ctr->dropped, 1ull);
                }
            }
            if (act[u] && out) out[i] = uint8_t(is_new);
            b += __popc(wm[u]);
        }
        }
    }
    if (!LOOKUP) {
        for (int o = 16; o; o >>= 1) {
            stored_here += __shfl_down_sync(kFull, stored_here, o);
            cas_count += __shfl_down_sync(kFull, cas_count, o);
        }
        if (lane == 0 && stored_here) atomicAdd(&t.ctr->size, stored_here);
        if (lane == 0 && cas_count) atomicAdd(&t.ctr->probe_cas, cas_count);
    }
}

// Eviction chains of the claim winners: each thread keeps kWU chains in
// flight and replaces a chain that ends (an empty slot, or the overflow set)
// with its next winner at once.  Records of keys the probe stored are only
// counted (they are listed for a caller that collects the new keys, which
// takes every record).
template <bool APPEND>
__global__ void __launch_bounds__(kBlock)
wide_cuckoo_insert_kernel(const DevTable t, const DevScratch sc, uint32_t parity, uint64_t max_winners,
                          ulonglong2* __restrict__ new_out, unsigned long long* __restrict__ new_count,
                          uint64_t new_cap) {
    const uint64_t count = min(uint64_t(__ldcg(&t.ctr->winners[parity])), max_winners);
    if (blockIdx.x == 0 && threadIdx.x == 0) t.ctr->winners[parity ^ 1u] = 0;
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t tid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    const WideWinner* win = reinterpret_cast<const WideWinner*>(sc.win);
    if (APPEND) {
        __shared__ ulonglong2 s_new[kBlock / 32][kStageCap];
        WarpStage<ulonglong2, kStageCap> stage(s_new[threadIdx.x >> 5]);
        const uint64_t rounds = (count + stride - 1) / stride;
        for (uint64_t r = 0; r < rounds; ++r) {
            const uint64_t i = r * stride + tid;
            ulonglong2 v = make_ulonglong2(0, 0);
            if (i < count) v = make_ulonglong2(win[i].lo, win[i].hi);
            stage.push(i < count, v, new_out, new_count, new_cap);
        }
        stage.flush(new_out, new_count, new_cap);
    }
    unsigned long long placed = 0, exchanges = 0;
    uint64_t next = tid;                         // this thread's next winner: tid, tid + stride, ...
    uint64_t lo[kWU], hi[kWU], pos[kWU];
    uint32_t evictions[kWU];
    bool live[kWU];
#pragma unroll
    for (int u = 0; u < kWU; ++u) {
        live[u] = false;
        lo[u] = hi[u] = pos[u] = 0;
        evictions[u] = 0;
    }
    // Bounded: each winner is taken once and its chain ends after at most
    // max_evictions + 1 exchanges.
    for (;;) {
        bool any = false;
#pragma unroll
        for (int u = 0; u < kWU; ++u) {
            while (!live[u] && next < count) {
                const WideWinner wn = win[next];
                next += stride;
                if (wn.start == kWidePlaced) {           // stored by the probe: only counted
                    ++placed;
                    continue;
                }
                sc.set[2 * wn.spos] = kOnes;             // leave the claim set empty for the next batch
                sc.set[2 * wn.spos + 1] = kOnes;
                lo[u] = wn.lo;
                hi[u] = wn.hi;
                pos[u] = hidx(wide_fold(wn.lo, wn.hi), t.seed[wn.start < t.k ? wn.start : 0], t.nslots);
                evictions[u] = 0;
                live[u] = true;
            }
            any |= live[u];
        }
        if (!any) break;
        ulonglong2 old[kWU];
#pragma unroll
        for (int u = 0; u < kWU; ++u)
            if (live[u]) {
                uint64_t ol, oh;
                exch128(t.slots + 2 * pos[u], lo[u], hi[u], ol, oh);
                old[u] = make_ulonglong2(ol, oh);
            }
#pragma unroll
        for (int u = 0; u < kWU; ++u) {
            if (!live[u]) continue;
            ++exchanges;
            if (old[u].x == kOnes && old[u].y == kOnes) {
                live[u] = false;
                ++placed;
                continue;
            }
            lo[u] = old[u].x;
            hi[u] = old[u].y;
            if (++evictions[u] > t.max_evict) {
                // The chain hit the eviction bound: the held key goes to the overflow set.
                const int rr = wide_ovf_insert(t, lo[u], hi[u]);
                if (rr == 1) {
                    ++placed;
                    atomicAdd(&t.ctr->ovf_used, 1u);
                } else if (rr < 0) {
                    set_flag(t.ctr, kFlagDropped);
                    atomicAdd(&t.ctr->dropped, 1ull);
                }
                live[u] = false;
                continue;
            }
            // Section 4.1: the evicted key sat at h_a(key) = pos; it moves on
            // to h_{a+1} (cyclically after h_k), a the smallest such index.
            const uint64_t fold = wide_fold(lo[u], hi[u]);
            uint32_t a = 0;
            for (; a + 1 < t.k; ++a)
                if (hidx(fold, t.seed[a], t.nslots) == pos[u]) break;
            const uint32_t nxt = (a + 1 == t.k) ? 0u : a + 1;
            pos[u] = hidx(fold, t.seed[nxt], t.nslots);
        }
    }
    for (int o = 16; o; o >>= 1) {
        placed += __shfl_down_sync(kFull, placed, o);
        exchanges += __shfl_down_sync(kFull, exchanges, o);
    }
    if (lane == 0 && placed) atomicAdd(&t.ctr->size, placed);
    if (lane == 0 && exchanges) atomicAdd(&t.ctr->exchanges, exchanges);
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

cudaError_t wide_cuckoo_probe(const DevTable& t, const DevScratch& sc, uint32_t parity, const void* keys, uint64_t n,
                              const unsigned long long* d_n, uint64_t off, uint8_t* is_new, cudaStream_t s,
                              bool list_stored) {
    ProfScope ps(kKCuckooProbe, s);
    auto k = wide_cuckoo_probe_kernel<false>;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, sc, parity, static_cast<const ulonglong2*>(keys),
                                                              n, d_n, off, is_new, list_stored);
    return cudaGetLastError();
}

cudaError_t wide_cuckoo_insert(const DevTable& t, const DevScratch& sc, uint32_t parity, void* new_out,
                               unsigned long long* new_count, uint64_t new_cap, uint64_t max_winners,
                               cudaStream_t s) {
    ProfScope ps(kKCuckooInsert, s);
    if (new_out) {
        auto k = wide_cuckoo_insert_kernel<true>;
        k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, sc, parity, max_winners,
                                                                  static_cast<ulonglong2*>(new_out), new_count, new_cap);
    } else {
        auto k = wide_cuckoo_insert_kernel<false>;
        k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, sc, parity, max_winners, nullptr, nullptr, 0);
    }
    return cudaGetLastError();
}

cudaError_t wide_cuckoo_lookup(const DevTable& t, const void* keys, uint64_t n, uint8_t* found, cudaStream_t s) {
    if (!n) return cudaSuccess;
    ProfScope ps(kKCuckooLookup, s);
    DevScratch none{};
    auto k = wide_cuckoo_probe_kernel<true>;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, none, 0u, static_cast<const ulonglong2*>(keys), n,
                                                              nullptr, 0, found, false);
    return cudaGetLastError();
}

cudaError_t wide_export(const DevTable& t, void* keys, unsigned long long* count, uint64_t cap, cudaStream_t s) {
    ProfScope ps(kKExport, s);
    auto k = wide_export_kernel;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(t, static_cast<uint64_t*>(keys), count, cap);
    return cudaGetLastError();
}

}  // namespace ht
