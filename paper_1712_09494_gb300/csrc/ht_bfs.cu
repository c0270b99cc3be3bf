// Successor generation for state-space exploration (Section 3.2 of the
// paper: successor state vectors are built by combining the enabled
// transitions of the processes).  The model's transition tables live in
// shared memory, read-only, as the paper keeps them in texture memory.
#include <cstring>
#include <type_traits>

#include "ht_multi_dev.cuh"

namespace ht {
namespace {

// Successors of a frontier: lane l expands state l of the warp's 32.  The
// lanes count their successors, reserve one range for the warp, then emit
// them into the warp's buffer in shared memory (in chunks of kSuccStage when
// the warp has more), from where the warp writes them out with coalesced
// stores: each lane's successors are contiguous in the output, so writing
// them straight from the lanes would scatter every store instruction over
// 32 places.
constexpr int kSuccBlock = 128;
constexpr int kSuccStage = 1024;

template <typename T>
__global__ void __launch_bounds__(kSuccBlock)
successors_kernel(const PreparedModel* __restrict__ model, const T* __restrict__ states, uint64_t n,
                  const unsigned long long* __restrict__ d_n, uint64_t off, T* __restrict__ succ,
                  uint64_t cap, unsigned long long* __restrict__ count,
                  unsigned long long* __restrict__ total) {
    // 16-byte states (models wider than 63 bits) use a half-size stage.
    constexpr int kStage = sizeof(T) > 8 ? kSuccStage / 2 : kSuccStage;
    using S = typename std::conditional<(sizeof(T) > 8), unsigned __int128, uint64_t>::type;
    __shared__ PreparedModel sm;
    __shared__ T s_out[kSuccBlock / 32][kStage];
    {
        const uint32_t* src = reinterpret_cast<const uint32_t*>(model);
        uint32_t* dst = reinterpret_cast<uint32_t*>(&sm);
        for (int i = threadIdx.x; i < int(sizeof(PreparedModel) / 4); i += blockDim.x) dst[i] = src[i];
    }
    __syncthreads();
    if (d_n) {
        const uint64_t all = __ldcg(d_n);
        n = all > off ? min(n, all - off) : 0;
    }
    const int lane = threadIdx.x & 31;
    T* buf = s_out[threadIdx.x >> 5];
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    const uint64_t rounds = (n + stride - 1) / stride;       // warp-uniform trip count
    unsigned long long made = 0;
    for (uint64_t r = 0; r < rounds; ++r) {
        const uint64_t i = r * stride + uint64_t(blockIdx.x) * blockDim.x + threadIdx.x;
        const bool act = i < n;
        const S s = act ? S(states[i]) : S(0);
        uint32_t cnt = 0;
        if (act) cnt = count_successors(sm, s);
        // Warp-wide exclusive scan of the counts, one reservation per warp.
        uint32_t incl = cnt;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t v = __shfl_up_sync(0xFFFFFFFFu, incl, o);
            if (lane >= o) incl += v;
        }
        const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
        unsigned long long base = 0;
        if (lane == 0 && tot) base = atomicAdd(count, (unsigned long long)tot);
        base = __shfl_sync(0xFFFFFFFFu, base, 0);
        const uint32_t excl = incl - cnt;
        for (uint32_t chunk = 0; chunk < tot; chunk += kStage) {
            if (act && excl < chunk + kStage && incl > chunk) {
                uint32_t k = excl;
                for_each_successor(sm, s, [&](S v) {
                    if (k >= chunk && k < chunk + kStage) buf[k - chunk] = T(v);
                    ++k;
                });
            }
            __syncwarp();
            const uint32_t m = min(uint32_t(kStage), tot - chunk);
            for (uint32_t j = lane; j < m; j += 32)
                if (base + chunk + j < cap) succ[base + chunk + j] = buf[j];
            __syncwarp();
        }
        made += cnt;
    }
    if (total) {
        for (int o = 16; o; o >>= 1) made += __shfl_down_sync(0xFFFFFFFFu, made, o);
        if (lane == 0 && made) atomicAdd(total, made);
    }
}

// Multi-table successors: the expanded states of every exploration form one
// index space; each thread finds its exploration by binary search and
// appends to that exploration's segment of the successor buffer.
__global__ void __launch_bounds__(kBlock) multi_successors_kernel(const MultiDev m, uint64_t max_work) {
    const uint64_t stride = uint64_t(gridDim.x) * blockDim.x;
    multi::successors(m, max_work, uint64_t(blockIdx.x) * blockDim.x + threadIdx.x, stride);
}

}  // namespace

PreparedModel prepare_model(const ht_model& h) {
    PreparedModel p;
    memset(&p, 0, sizeof(p));
    // Transition j of component c in local state u: label 0 is a local
    // action; label q+1 belongs to synchronising pair q (whose members are
    // pair_c1[q] and pair_c2[q]).  The model was validated (deg <= 4, labels
    // <= num_pairs, members distinct).
    for (int c = 0; c < h.num_components && c < 16; ++c)
        for (int u = 0; u < 32; ++u)
            for (int j = 0; j < h.deg[c][u] && j < 4; ++j) {
                const int lab = h.lab[c][u][j];
                if (lab == 0) {
                    p.loc[c][u][p.nloc[c][u]++] = h.tgt[c][u][j];
                } else if (lab <= h.num_pairs && lab <= 8) {
                    const int q = lab - 1;
                    for (int side = 0; side < 2; ++side)
                        if ((side == 0 ? h.pair_c1[q] : h.pair_c2[q]) == c)
                            p.syn[q][side][u][p.nsyn[q][side][u]++] = h.tgt[c][u][j];
                }
            }
    int o = 0;
    for (int c = 0; c < 16; ++c) {
        p.bits[c] = h.bits[c];
        p.off[c] = uint8_t(o);
        if (c < h.num_components) o += h.bits[c];
    }
    memcpy(p.pc1, h.pair_c1, 8);
    memcpy(p.pc2, h.pair_c2, 8);
    p.C = h.num_components;
    p.P = h.num_pairs;
    return p;
}

cudaError_t multi_successors(int, const MultiDev& m, uint64_t max_work, cudaStream_t s) {
    ProfScope ps(kKSuccessors, s);
    auto k = multi_successors_kernel;
    k<<<launch_blocks((const void*)k, kBlock), kBlock, 0, s>>>(m, max_work);
    return cudaGetLastError();
}

cudaError_t successors(int kw, const PreparedModel* model, const void* states, uint64_t n,
                       const unsigned long long* d_n, uint64_t off, void* succ, uint64_t cap,
                       unsigned long long* count, unsigned long long* total, cudaStream_t s) {
    ProfScope ps(kKSuccessors, s);
    if (kw == 32) {
        auto k = successors_kernel<uint32_t>;
        k<<<launch_blocks((const void*)k, kSuccBlock), kSuccBlock, 0, s>>>(
            model, static_cast<const uint32_t*>(states), n, d_n, off, static_cast<uint32_t*>(succ), cap, count, total);
    } else if (kw == 128) {
        using U = unsigned __int128;
        auto k = successors_kernel<U>;
        k<<<launch_blocks((const void*)k, kSuccBlock), kSuccBlock, 0, s>>>(
            model, static_cast<const U*>(states), n, d_n, off, static_cast<U*>(succ), cap, count, total);
    } else {
        auto k = successors_kernel<uint64_t>;
        k<<<launch_blocks((const void*)k, kSuccBlock), kSuccBlock, 0, s>>>(
            model, static_cast<const uint64_t*>(states), n, d_n, off, static_cast<uint64_t*>(succ), cap, count, total);
    }
    return cudaGetLastError();
}

}  // namespace ht
