// LRU-based caching of remote copies under a budget (Section III-B2), run on
// the device at every superstep boundary for all partitions at once.
//
// Each partition p caches at most C copies of the remote vertices its
// in-edges read. The boundary before superstep t+1 (after superstep t's
// exchange) takes, per copy g of p (vertex u = ghost_gid[g]):
//   used  = u is in the frontier of superstep t+1 (u changed in superstep t;
//           before superstep 1: every vertex, or the SSSP source)
//   cand  = cached or used
//   W     = min(kLruWMax, floor(W / 2) * cached + reads_p(u) * used)
//           (decays by half per superstep, rises with use; 0 on entry)
//   a used copy that is not cached is downloaded: its slot takes the owner's
//   value and it counts in the superstep's `downloads`
// then keeps the C candidates of highest W, ties to the lower vertex id
// (copies are sorted by vertex id within a partition), and forgets the
// weights of the rest. Cached copies whose vertex changes are refreshed by
// the lazy upload (k_sync_pull, before this), so every copy a superstep uses
// holds its owner's current value, cached or not: the cache changes which
// values are moved, never a value.
//
// Kernels: k_lru_weigh (the update, a histogram of W per partition, the
// downloads), k_lru_threshold (per partition: the weight W* at which the
// top C end and how many ties at W* still fit), an exclusive scan of the tie
// flags (ghost order = (partition, vertex id)), k_lru_select (the new cached
// flags).
#include <algorithm>

#include "gxp_internal.hpp"

namespace gxp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kLruBlock = 256;
constexpr uint32_t kSmemBins = 1024;   // low weights are counted in shared memory first

// flags[g]: bit 0 cached, bit 1 candidate at this boundary
constexpr uint8_t kCached = 1u, kCand = 2u;

__device__ __forceinline__ bool quiet_superstep(const LruArgs& a) {
    if (!a.quiet_check) return false;
    unsigned long long c = 0;
    for (int i = 0; i < kStatLanes; ++i) c += a.quiet_check->changed[i];
    return c == 0ull;
}

__global__ void __launch_bounds__(kLruBlock) k_lru_weigh(const LruArgs a) {
    __shared__ uint32_t s_hist[kSmemBins];
    __shared__ uint32_t s_cand, s_dl;
    const uint32_t p = blockIdx.y;
    for (uint32_t i = threadIdx.x; i < kSmemBins; i += kLruBlock) s_hist[i] = 0u;
    __shared__ bool s_skip;
    if (threadIdx.x == 0) {
        s_cand = s_dl = 0u;
        s_skip = quiet_superstep(a);   // a superstep after a quiet one did nothing
    }
    __syncthreads();
    const bool skip = s_skip;
    const uint32_t g0 = a.ghost_base[p], g1 = a.ghost_base[p + 1];
    const int lane = threadIdx.x & 31;
    uint32_t cand_n = 0, dl_n = 0;
    for (uint32_t base = g0 + blockIdx.x * kLruBlock; !skip && base < g1; base += gridDim.x * kLruBlock) {
        const uint32_t g = base + threadIdx.x;
        bool cand = false;
        uint32_t w = 0;
        if (g < g1) {
            const uint32_t u = a.ghost_gid[g];
            const bool used = a.frontier_all ? true
                              : a.frontier_bits ? ((a.frontier_bits[u >> 5] >> (u & 31u)) & 1u) != 0u
                                                : u == a.frontier_one;
            const uint8_t f = a.flags[g];
            const bool cached = (f & kCached) != 0;
            cand = cached || used;
            if (cand) {
                const uint64_t x = (uint64_t)(cached ? a.weight[g] >> 1 : 0u) + (used ? a.reads[g] : 0u);
                w = x < (uint64_t)kLruWMax ? (uint32_t)x : kLruWMax;
                a.weight[g] = w;
                a.flags[g] = (uint8_t)(f | kCand);
                ++cand_n;
                if (used && !cached) {
                    a.ghost[g] = a.own_val[u];   // the download
                    ++dl_n;
                }
            } else if (f != 0u) {
                a.flags[g] = 0u;
            }
        }
        // histogram of W over the candidates: lanes with equal low weights add once
        const unsigned cm = __ballot_sync(kFull, cand);
        if (cand) {
            if (w < kSmemBins) {
                const unsigned grp = __match_any_sync(cm, w);
                if (lane == __ffs(grp) - 1) atomicAdd(&s_hist[w], (uint32_t)__popc(grp));
            } else {
                atomicAdd(&a.hist[(size_t)p * kLruBins + w], 1u);
            }
        }
    }
    cand_n = __reduce_add_sync(kFull, cand_n);
    dl_n = __reduce_add_sync(kFull, dl_n);
    if (lane == 0) {
        if (cand_n) atomicAdd(&s_cand, cand_n);
        if (dl_n) atomicAdd(&s_dl, dl_n);
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kSmemBins; i += kLruBlock)
        if (s_hist[i]) atomicAdd(&a.hist[(size_t)p * kLruBins + i], s_hist[i]);
    if (threadIdx.x == 0) {
        if (s_cand) atomicAdd(&a.part_state[p].cand, s_cand);
        if (s_dl) atomicAdd(&a.stats_out->downloads, (unsigned long long)s_dl);
    }
}

// One block per partition: W* and the ties at W* that still fit, from the
// histogram (which it clears for the next boundary).
__global__ void __launch_bounds__(1024) k_lru_threshold(const LruArgs a) {
    constexpr int kT = 1024;
    constexpr uint32_t kPer = kLruBins / kT;   // bins per thread, descending weights
    __shared__ uint32_t s_sum[kT];
    const uint32_t p = blockIdx.x;
    uint32_t* h = a.hist + (size_t)p * kLruBins;
    LruPart& st = a.part_state[p];
    const uint32_t cap = a.capacity;
    const uint32_t cand = st.cand;
    // thread t owns bins [kLruBins - kPer (t + 1), kLruBins - kPer t): the highest first
    const uint32_t hi = kLruBins - kPer * threadIdx.x;
    uint32_t mine = 0;
    for (uint32_t b = hi - kPer; b < hi; ++b) mine += h[b];
    s_sum[threadIdx.x] = mine;
    __syncthreads();
    // inclusive scan over threads (counts of higher bins first)
    for (uint32_t o = 1; o < kT; o <<= 1) {
        const uint32_t x = threadIdx.x >= o ? s_sum[threadIdx.x - o] : 0u;
        __syncthreads();
        s_sum[threadIdx.x] += x;
        __syncthreads();
    }
    const uint32_t incl = s_sum[threadIdx.x], excl = incl - mine;
    if (cand <= cap) {
        if (threadIdx.x == 0) {
            st.w_star = 0u;
            st.ties = kInf;   // every candidate stays
        }
    } else if (cap == 0u) {
        if (threadIdx.x == 0) {
            st.w_star = kLruWMax + 1u;   // nothing stays
            st.ties = 0u;
        }
    } else if (excl < cap && incl >= cap) {
        // the bin where the running count (highest weights first) reaches cap
        uint32_t run = excl;
        for (uint32_t b = hi; b-- > hi - kPer;) {
            const uint32_t c = h[b];
            if (run + c >= cap) {
                st.w_star = b;
                st.ties = cap - run;
                break;
            }
            run += c;
        }
    }
    __syncthreads();
    for (uint32_t b = hi - kPer; b < hi; ++b) h[b] = 0u;
    if (threadIdx.x == 0) st.cand = 0u;
}

__global__ void __launch_bounds__(kLruBlock) k_lru_ties(const LruArgs a) {
    const uint32_t p = blockIdx.y;
    const uint32_t g0 = a.ghost_base[p], g1 = a.ghost_base[p + 1];
    const uint32_t ws = a.part_state[p].w_star;
    for (uint32_t g = g0 + blockIdx.x * kLruBlock + threadIdx.x; g < g1; g += gridDim.x * kLruBlock)
        a.tie[g] = ((a.flags[g] & kCand) != 0u && a.weight[g] == ws) ? 1u : 0u;
}

__global__ void __launch_bounds__(kLruBlock) k_lru_select(const LruArgs a) {
    const uint32_t p = blockIdx.y;
    const uint32_t g0 = a.ghost_base[p], g1 = a.ghost_base[p + 1];
    const uint32_t ws = a.part_state[p].w_star, ties = a.part_state[p].ties;
    const uint32_t tie0 = a.tie_scan[g0];
    for (uint32_t g = g0 + blockIdx.x * kLruBlock + threadIdx.x; g < g1; g += gridDim.x * kLruBlock) {
        const uint8_t f = a.flags[g];
        if (!(f & kCand)) continue;
        const uint32_t w = a.weight[g];
        const bool keep = ties == kInf || w > ws || (w == ws && a.tie_scan[g] - tie0 < ties);
        a.flags[g] = keep ? kCached : 0u;
        if (!keep) a.weight[g] = 0u;
    }
}

}  // namespace

cudaError_t launch_lru_boundary(const LruArgs& a, uint32_t max_ghosts_per_part, cudaStream_t s) {
    if (a.n_ghost == 0) return cudaSuccess;
    const uint32_t bx = std::max<uint32_t>(1, std::min<uint32_t>((max_ghosts_per_part + kLruBlock - 1) / kLruBlock,
                                                                 (152u * 8u + a.n_parts - 1) / a.n_parts));
    const dim3 grid(bx, a.n_parts);
    k_lru_weigh<<<grid, kLruBlock, 0, s>>>(a);
    k_lru_threshold<<<a.n_parts, 1024, 0, s>>>(a);
    k_lru_ties<<<grid, kLruBlock, 0, s>>>(a);
    cudaError_t e = launch_exclusive_scan_u32(a.tie, a.n_ghost, a.tie_scan, a.scan_scratch, s);
    if (e != cudaSuccess) return e;
    k_lru_select<<<grid, kLruBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gxp
