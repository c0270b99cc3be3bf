// The batched exploration as ONE persistent launch per group of
// explorations: every BFS level of every exploration runs inside a single
// cooperative kernel, with bounded grid-wide barriers between the phases of
// a step instead of one kernel launch (and one host round trip) per phase.
//
// A step of the group (ht_multi_dev.cuh): block 0 advances every
// exploration's cursor and shares the successor buffer; all blocks generate
// the expanded states' successors; all blocks find-or-put them, each 32-key
// tile against its own exploration's table, appending new states to that
// exploration's states array.  Bucket tables use the warp-cooperative tile
// of ht_bucket_tile.cuh.  Cuckoo tables (Section 4.1) need two phases, as in
// the single-table path: a probe that reads h_1 (then h_2..h_k when h_1 is
// occupied), elects one winner per distinct absent key in the table's own
// claim set and lists the winners, then -- after a barrier, so no table is
// written while any probe reads it -- the eviction-chain insert of every
// listed winner.
//
// Co-residency: the kernel is launched cooperatively with at most as many
// blocks as fit on the device at once, so every block runs while the others
// wait at a barrier.  Every barrier wait is bounded in time (barrier_ns,
// 2 s by default, far above any phase of a step): a block that waits too
// long sets kMultiTimeout in the run's status word and returns, and every
// other block then leaves at its next barrier; the host reports
// HT_ERR_TIMEOUT.  A test makes one block leave before its first barrier,
// as a block that died would, and checks that status.
#include "ht_bucket_tile.cuh"

namespace ht {
namespace {

constexpr uint32_t kBarrierPolls = 1u << 24;      // a second bound, in polls (~16 s at most)

__device__ __forceinline__ uint64_t globaltimer_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}

__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// Grid-wide barrier over all blocks of the launch (bar[0]: arrivals,
// bar[1]: generation).  Thread 0 of each block reads the generation, then
// arrives; the last arrival resets the count and publishes the next
// generation; the others poll it with back-off, bounded.  Returns false on
// every thread of the block when the run has timed out.
__device__ bool grid_sync(const MultiDev& m, int* s_ok) {
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        unsigned* cnt = m.bar;
        unsigned* gen = m.bar + 1;
        const unsigned g = ld_acquire_u32(gen);
        __threadfence();                                  // this block's writes before its arrival
        if (atomicAdd(cnt, 1u) + 1u == gridDim.x) {
            atomicExch(cnt, 0u);
            __threadfence();
            st_release_u32(gen, g + 1u);
        } else {
            const uint64_t t0 = globaltimer_ns();
            unsigned ns = 32;
            for (uint32_t polls = 0; ld_acquire_u32(gen) == g; ++polls) {
                if ((ld_acquire_u32(m.status) & kMultiTimeout) || polls > kBarrierPolls ||
                    globaltimer_ns() - t0 > m.barrier_ns) {
                    atomicOr(m.status, kMultiTimeout);
                    ok = 0;
                    break;
                }
                __nanosleep(ns);
                if (ns < 1024) ns *= 2;
            }
        }
        __threadfence();
        *s_ok = ok && !(ld_acquire_u32(m.status) & kMultiTimeout);
    }
    __syncthreads();
    return *s_ok != 0;
}

// Level 0 of every exploration: its initial state placed in its (empty)
// table -- bucket scheme: the first slot of bucket h_1, the lowest free slot
// of the claim order; Cuckoo: slot h_1 -- and stored as the first state.
// Tables are addressed as 64-bit key tables (a 32-bit set table's words are
// the same), states are written in their exploration's width.
template <bool CUCKOO, int BS>
__device__ void place_initial_states(const MultiDev& m, uint64_t gtid, uint64_t nthreads) {
    for (uint64_t e = gtid; e < m.count; e += nthreads) {
        const uint64_t key = m.s0[e];
        const DevTable& t = m.tables[e];
        const uint64_t pos = CUCKOO ? hidx(key, t.seed[0], t.nslots) : hidx(key, t.seed[0], t.nbuckets) * BS;
        const uint64_t old = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + pos), kEmpty, key);
        if (old != kEmpty) atomicOr(m.status, kMultiBadInit);
        if (m.narrow[e]) static_cast<unsigned int*>(m.states[e])[0] = static_cast<unsigned int>(key);
        else static_cast<unsigned long long*>(m.states[e])[0] = key;
        atomicAdd(&t.ctr->size, 1ull);
        m.total[e] = 1;
        m.lo[e] = 0;
        m.hi[e] = 1;
        m.cur[e] = 0;
        m.take[e] = 0;
        m.gen[e] = 0;
        m.level[e] = 0;
        m.done[e] = old == kEmpty ? 0u : 2u;
        m.level_sizes[e * m.max_levels] = 1;
    }
}

// Cuckoo probe of one step over warps [gw] of [nwarps]: each warp takes a
// contiguous range of the step's 32-key tiles (the TileMap numbering), one
// key per lane, against the tile's exploration e.  A key is looked up at h_1, then (h_1 occupied by another
// key) at h_2..h_k, then in the stash / overflow set when those are in use;
// a key stored at h_j has h_1..h_(j-1) occupied, so an empty h_1 proves it
// absent.  An absent key that saw an EMPTY slot stores itself there (a CAS
// in slot order); one whose k slots are all full claims its key in e's
// claim set, and the one claimant per distinct key joins the group's
// winner list with its exploration, for a chain from h_1.  Every new key is
// appended to e's states.
constexpr int kWinStage = 64;            // staged winner records per warp

__device__ void cuckoo_probe_tiles(const MultiDev& m, const multi::TileMap& tm, uint64_t gw, uint64_t nwarps,
                                   uint64_t* stage_buf, MultiWinner* wstage) {
    constexpr int KW = 64;
    using K = Keys<KW>;
    uint32_t wpend = 0;
    // Lists the staged winners with one atomic on the group's count.  The
    // list holds a whole step's successors, so it cannot run out; if it did,
    // the record's claim is given back and its table reports a dropped key.
    auto flush_winners = [&]() {
        __syncwarp();
        if (wpend) {
            const int ln = threadIdx.x & 31;
            unsigned long long b = 0;
            if (ln == 0) b = atomicAdd(m.win_count, (unsigned long long)wpend);
            b = __shfl_sync(0xFFFFFFFFu, b, 0);
            for (uint32_t j = ln; j < wpend; j += 32) {
                const MultiWinner wn = wstage[j];
                if (b + j < m.win_cap) {
                    m.win[b + j] = wn;
                } else {
                    const uint32_t we = wn.tag >> 8;
                    m.scratch[we].set[wn.spos] = kEmpty;
                    set_flag(m.tables[we].ctr, kFlagDropped);
                    atomicAdd(&m.tables[we].ctr->dropped, 1ull);
                }
            }
        }
        __syncwarp();
        wpend = 0;
    };
    const uint64_t tiles = tm.total(m);
    const int lane = threadIdx.x & 31;
    const uint64_t per = (tiles + nwarps - 1) / nwarps;
    const uint64_t t_begin = min(tiles, gw * per), t_end = min(tiles, t_begin + per);
    if (t_begin >= t_end) return;
    multi::StateStage<kStageCap> stage(stage_buf);
    multi::TileCursor cur;
    cur.start(m, tm, t_begin);
    uint32_t e = cur.e;
    uint64_t cnt = 0;
    uint32_t stash_used = 0, ovf_used = 0;
    auto load_desc = [&]() {
        cnt = multi::step_count(m, e);
        stash_used = __ldcg(&m.tables[e].ctr->stash_used);
        ovf_used = __ldcg(&m.tables[e].ctr->ovf_used);
    };
    load_desc();
    uint32_t run_e = e;                        // keys stored by this warp's CASes, per run of e
    unsigned long long run_n = 0;
    uint64_t next_key = __ldcg(reinterpret_cast<const unsigned long long*>(m.succ + cur.key_index(m, t_begin, lane)));
    for (uint64_t tile = t_begin; tile < t_end; ++tile) {
        const uint64_t cur_key = next_key;
        if (tile >= cur.b1) {                          // into a later exploration's tiles
            stage.flush(m, e);
            cur.seek(m, tm, tile);
            e = cur.e;
            load_desc();
        }
        const uint64_t i = 32 * (tile - cur.b0) + lane;
        if (tile + 1 < t_end) {
            multi::TileCursor nx = cur;
            nx.seek(m, tm, tile + 1);
            next_key = __ldcg(reinterpret_cast<const unsigned long long*>(m.succ + nx.key_index(m, tile + 1, lane)));
        }
        const bool mine = i < cnt;
        if (!__any_sync(0xFFFFFFFFu, mine)) continue;
        const DevTable& t = m.tables[e];
        const uint64_t key = mine ? K::keyof(cur_key) : 0;
        const bool ok = mine && !K::reserved(key);
        if (mine && !ok) set_flag(t.ctr, kFlagInvalidKey);
        uint64_t w = kEmpty;
        if (ok) w = __ldcg(reinterpret_cast<const unsigned long long*>(t.slots + hidx(key, t.seed[0], t.nslots)));
        bool found = ok && K::keyof(w) == key;
        const bool more = ok && !found && !K::empty(w);
        uint32_t start = 0;
        // h_2..h_k one slot at a time, stopping at the key or at the first
        // EMPTY slot (the key is not past it; a new key's chain starts
        // there): the probe is bound by the random lines it reads.
        bool go = more;
        for (uint32_t a = 1; a < t.k && __any_sync(0xFFFFFFFFu, go); ++a) {
            if (go) {
                const uint64_t v = __ldcg(reinterpret_cast<const unsigned long long*>(t.slots + hidx(key, t.seed[a], t.nslots)));
                if (K::keyof(v) == key) found = true;
                else if (K::empty(v)) start = a;
                go = !found && start == 0;
            }
        }
        if ((stash_used | ovf_used) && ok && !found) {
            uint64_t sw;
            found = find_spill<KW>(t, key, stash_used, ovf_used, &sw);
        }
        // An absent key that saw an EMPTY slot (h_1, or the first of
        // h_2..h_k; with t.chain_h1 only h_1) stores itself there with a CAS
        // from EMPTY, going on in slot order while the CAS returns another
        // key; a CAS that returns the key means another copy stored it.  Only
        // keys whose k slots are all full claim and run a chain.  (The
        // argument is the single-table kernel's: nothing moves a key during
        // the probe phase, the grid barrier ends it before any chain runs.)
        bool placed = false;
        bool pend = ok && !found && (!more || (start != 0 && !t.chain_h1));
        bool claim = ok && !found && !pend;
        uint32_t at = more ? start : 0u;
        for (uint32_t pass = 0; pass < t.k && __any_sync(0xFFFFFFFFu, pend); ++pass) {
            if (pend) {
                const uint64_t cw = atomicCAS(reinterpret_cast<unsigned long long*>(t.slots + hidx(key, t.seed[at], t.nslots)),
                                              kEmpty, K::word(key, 0u));
                if (cw == kEmpty) {
                    placed = true;
                    pend = false;
                } else if (K::keyof(cw) == key) {
                    found = true;                      // another copy stored it
                    pend = false;
                } else if (t.chain_h1 || at + 1 >= t.k) {
                    claim = true;                      // every slot holds another key now
                    pend = false;
                } else {
                    ++at;
                }
            }
        }
        // The stored keys count toward e's size, per run of tiles of e.
        {
            const unsigned pm = __ballot_sync(0xFFFFFFFFu, placed);
            if (e != run_e) {
                if (lane == 0 && run_n) atomicAdd(&m.tables[run_e].ctr->size, run_n);
                run_e = e;
                run_n = 0;
            }
            run_n += __popc(pm);
        }
        // In-batch dedup in e's claim set of the keys with every slot full:
        // the one claimant of each such key wins.
        const bool need = claim;
        bool winner = placed;
        uint32_t spos = 0;
        if (need) {
            const DevScratch& sc = m.scratch[e];
            spos = uint32_t(mix64(key ^ (t.aux_seed * 3 + 1)) & sc.mask);
            const uint64_t sw = atomicCAS(reinterpret_cast<unsigned long long*>(sc.set + spos), kEmpty, key);
            if (sw == kEmpty) {
                winner = true;
            } else if (K::keyof(sw) != key) {
                uint32_t at = 0;
                const uint32_t n = uint32_t(sc.mask + 1);
                const int rc = lp_insert<KW>(sc.set, n, spos + 1 == n ? 0u : spos + 1, key, key, &at);
                winner = rc == 1;
                spos = at;
                if (rc < 0) {                          // more distinct misses than the claim set holds
                    set_flag(t.ctr, kFlagDropped);
                    atomicAdd(&t.ctr->dropped, 1ull);
                }
            }
        }
        // Claim winners to the warp's stage of winner records (listed with
        // one atomic per flush; their chains start at h_1); every new key to
        // e's states.
        const bool listed = winner && !placed;
        const unsigned wm = __ballot_sync(0xFFFFFFFFu, listed);
        if (wm) {
            if (wpend + __popc(wm) > uint32_t(kWinStage)) flush_winners();
            if (listed) {
                MultiWinner& wn = wstage[wpend + __popc(wm & ((1u << lane) - 1))];
                wn.word = K::word(key, 0u);
                wn.spos = spos;
                wn.tag = e << 8;
            }
            wpend += __popc(wm);
        }
        stage.push(winner, key, m, e);
    }
    if (lane == 0 && run_n) atomicAdd(&m.tables[run_e].ctr->size, run_n);
    stage.flush(m, e);
    flush_winners();
}

// Cuckoo insert of the step's claim winners over threads [gtid] of
// [nthreads]: each thread keeps four eviction chains in flight (Section
// 4.1, Fig. 2) and refills a chain as soon as it ends.  A chain starts at
// h_1, exchanges its word in, and moves an evicted key k' from h_a(k') (the
// smallest a naming the slot) to h_(a+1); after max_evictions the held word
// goes to the stash.  Each winner's claim
// is cleared from its table's claim set when the winner is taken.
__device__ void cuckoo_insert_winners(const MultiDev& m, uint64_t gtid, uint64_t nthreads) {
    constexpr int KW = 64;
    using K = Keys<KW>;
    constexpr int U = 4;
    const uint64_t count = min(uint64_t(__ldcg(m.win_count)), m.win_cap);
    uint64_t next = gtid;
    uint64_t word[U], pos[U];
    uint32_t ev[U], ex[U];
    bool live[U];
#pragma unroll
    for (int u = 0; u < U; ++u) {
        live[u] = false;
        word[u] = pos[u] = 0;
        ev[u] = ex[u] = 0;
    }
    // Placements are counted per run of one exploration and added to its
    // size counter when the run ends.
    uint32_t run_e = 0;
    unsigned long long run_n = 0;
    auto placed = [&](uint32_t e) {
        if (run_n && e != run_e) {
            atomicAdd(&m.tables[run_e].ctr->size, run_n);
            run_n = 0;
        }
        run_e = e;
        ++run_n;
    };
    // Bounded: each winner is taken once and its chain ends after at most
    // max_evictions + 1 exchanges.
    for (;;) {
        bool any = false;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!live[u] && next < count) {
                const ulonglong2 r = __ldcg(reinterpret_cast<const ulonglong2*>(m.win + next));
                next += nthreads;
                const uint32_t spos = uint32_t(r.y), tag = uint32_t(r.y >> 32);
                const uint32_t e = tag >> 8, st = tag & 0xFFu;
                m.scratch[e].set[spos] = kEmpty;           // leave the claim set empty for the next step
                const DevTable& t = m.tables[e];
                word[u] = r.x;
                pos[u] = hidx(K::keyof(r.x), t.seed[st < t.k ? st : 0u], t.nslots);
                ex[u] = e;
                ev[u] = 0;
                live[u] = true;
            }
            any |= live[u];
        }
        if (!any) break;
        uint64_t old[U];
#pragma unroll
        for (int u = 0; u < U; ++u)
            if (live[u]) old[u] = atomicExch(reinterpret_cast<unsigned long long*>(m.tables[ex[u]].slots + pos[u]), word[u]);
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (!live[u]) continue;
            const DevTable& t = m.tables[ex[u]];
            if (K::empty(old[u])) {
                live[u] = false;
                placed(ex[u]);
                continue;
            }
            word[u] = old[u];
            if (++ev[u] > t.max_evict) {
                if (place_spill<KW>(t, K::keyof(word[u]), word[u]) == 1) placed(ex[u]);
                live[u] = false;
                continue;
            }
            const uint64_t key = K::keyof(old[u]);
            uint32_t a = 0;
            for (; a + 1 < t.k; ++a)
                if (hidx(key, t.seed[a], t.nslots) == pos[u]) break;
            const uint32_t nxt = (a + 1 == t.k) ? 0u : a + 1;
            pos[u] = hidx(key, t.seed[nxt], t.nslots);
        }
    }
    if (run_n) atomicAdd(&m.tables[run_e].ctr->size, run_n);
}

// Resident blocks per SM the kernel is compiled for (registers): measured
// on config 4, the bucket kernel is fastest at 2 (no spills), the Cuckoo
// kernel at 3.
#ifndef HT_PERSIST_MIN_BLOCKS_BUCKET
#define HT_PERSIST_MIN_BLOCKS_BUCKET 2
#endif
#ifndef HT_PERSIST_MIN_BLOCKS_CUCKOO
#define HT_PERSIST_MIN_BLOCKS_CUCKOO 3
#endif

template <bool CUCKOO, int BS, int G>
__global__ void __launch_bounds__(kBlock, CUCKOO ? HT_PERSIST_MIN_BLOCKS_CUCKOO : HT_PERSIST_MIN_BLOCKS_BUCKET)
multi_persistent_kernel(const __grid_constant__ MultiDev m, uint64_t budget, uint64_t max_steps, uint64_t max_work,
                        uint64_t max_tiles) {
    __shared__ uint64_t s_new[kBlock / 32][kStageCap];
    __shared__ unsigned long long sh[multi::kAdvShared];
    __shared__ unsigned int s_first[multi::kExactTileExpl + 1];
    __shared__ MultiWinner s_win[kBlock / 32][CUCKOO ? kWinStage : 1];
    __shared__ int s_ok;
    const uint64_t gtid = uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
    const uint64_t nthreads = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t gw = gtid >> 5, nwarps = nthreads >> 5;
    uint64_t* stage = s_new[threadIdx.x >> 5];
    place_initial_states<CUCKOO, BS>(m, gtid, nthreads);
    if (int(blockIdx.x) == m.absent_block) return;     // failure test: a block that never arrives
    if (!grid_sync(m, &s_ok)) return;
    uint64_t step = 0;
    for (; step < max_steps; ++step) {
        if (blockIdx.x == 0) multi::advance<kBlock>(m, budget, sh);
        if (!grid_sync(m, &s_ok)) return;
        if (__ldcg(m.active) == 0) break;
        multi::successors(m, max_work, gtid, nthreads);
        if (!grid_sync(m, &s_ok)) return;
        // Every block numbers the step's tiles over the successors made.
        const multi::TileMap tm = multi::tile_map<kBlock>(m, s_first, sh);
        if constexpr (CUCKOO) {
            cuckoo_probe_tiles(m, tm, gw, nwarps, stage, s_win[threadIdx.x >> 5]);
            if (!grid_sync(m, &s_ok)) return;
            cuckoo_insert_winners(m, gtid, nthreads);
        } else {
            bucket::multi_find_or_put<BS, G>(m, tm, gw, nwarps, stage);
        }
        if (!grid_sync(m, &s_ok)) return;
    }
    if (gtid == 0) *m.steps = step;
}

template <bool CUCKOO, int BS, int G>
cudaError_t launch_persistent(const MultiDev& m, uint64_t budget, uint64_t max_steps, uint64_t max_work,
                              uint64_t max_tiles, cudaStream_t s) {
    auto k = multi_persistent_kernel<CUCKOO, BS, G>;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k, kBlock, 0);
    if (e != cudaSuccess) return e;
    if (per_sm < 1) return cudaErrorInvalidConfiguration;
    // Every block resident at once (a cooperative launch refuses a grid that
    // does not fit), so the grid barriers cannot wait on an unscheduled block.
    const dim3 grid(unsigned(per_sm * sms)), block(kBlock);
    MultiDev mm = m;
    void* args[] = {&mm, &budget, &max_steps, &max_work, &max_tiles};
    ProfScope ps(kKMultiPersistent, s);
    return cudaLaunchCooperativeKernel(reinterpret_cast<const void*>(k), grid, block, args, 0, s);
}

}  // namespace

cudaError_t multi_persistent(ht_scheme scheme, const BucketCfg& c, const MultiDev& m, uint64_t budget,
                             uint64_t max_steps, uint64_t max_work, uint64_t max_tiles, cudaStream_t s) {
    if (scheme == HT_CUCKOO) return launch_persistent<true, 16, 2>(m, budget, max_steps, max_work, max_tiles, s);
#define P(BS, G)                                                                                           \
    if (c.bucket_slots == BS && c.lanes == G)                                                              \
        return launch_persistent<false, BS, G>(m, budget, max_steps, max_work, max_tiles, s);
    P(16, 2) P(16, 4) P(16, 8) P(16, 16) P(8, 2) P(8, 4) P(8, 8) P(32, 4) P(32, 8) P(32, 16) P(32, 32)
#undef P
    return cudaErrorInvalidValue;
}

}  // namespace ht
