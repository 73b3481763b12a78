// Mode-label propagation superstep: the paper's LP workload (Section V-A)
// as the three template functions of Section IV-A1 with MSGGen = l[u],
// MSGMerge = the mode of a vertex's incoming labels (ties to the smallest
// label) and MSGApply = take it. Jacobi order: labels are read from the
// previous superstep's buffer and written to the other one.
//
//  * rows with 1..32 in-edges: packed (in input order, edges adjacent) into
//    windows of at most 32 edges, one per warp step: each lane loads one
//    edge's label (coalesced), __match_any_sync on (row, label) gives every
//    label's count in its row, and two reductions over the row's lanes
//    (largest count, then smallest label with it) give the row's mode. No
//    sort (sorting each row in its lane cost about 2,000 instructions per 32
//    rows, every lane waiting on the longest row);
//  * rows with 33..4096 in-edges: a CTA per row gathers the labels into
//    shared memory, sorts them (bitonic), finds each run's start with a
//    block max-scan of run starts, and reduces (count, -label) at run ends;
//  * hub rows (more in-edges): each chunk of 4096 is sorted the same way and
//    its runs are added into the hub's hash table (open addressing, at most
//    half full); a CTA per hub then reduces its table and empties it.
#include "frontier.cuh"

#include <algorithm>

namespace gxp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kLpBlock = 256;
constexpr int kLpWarps = kLpBlock / 32;
constexpr int kGatherUnroll = 4;

// the label of in-edge source s of partition P (previous superstep)
__device__ __forceinline__ uint32_t lp_label(const LpArgs& a, const LpPart& P, uint32_t s) {
    if (P.src_map) return __ldg(a.own_cur + __ldg(P.src_map + s));
    return s < P.n_own ? __ldg(a.own_cur + P.v_begin + s) : __ldg(a.ghost + P.ghost_base + (s - P.n_own));
}

// MSGApply: returns whether the label changed
__device__ __forceinline__ bool lp_apply(const LpArgs& a, uint32_t g, uint32_t label) {
    const uint32_t old = a.own_cur[g];
    a.own_nxt[g] = label;
    if (label == old) return false;
    if (a.changed_bits) atomicOr(a.changed_bits + (g >> 5), 1u << (g & 31u));
    return true;
}

// a min-label superstep after a quiet one changes nothing: the same holds
// here (same labels in, same labels out), so such a superstep returns at once
__device__ __forceinline__ bool lp_quiet(const LpArgs& a, int lane) {
    if (!a.skip_if_quiet) return false;
    unsigned long long c = a.stats_in->changed[lane] + a.stats_in->changed[lane + 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    return c == 0ull;
}

__device__ __forceinline__ void lp_count(const LpArgs& a, uint32_t n_changed, uint64_t slot) {
    if (n_changed) atomicAdd(&a.stats_out->changed[slot % kStatLanes], (unsigned long long)n_changed);
}

// (count, -label) as one key: the larger key is the more frequent label,
// and among equally frequent ones the smaller
__device__ __forceinline__ unsigned long long mode_key(uint32_t count, uint32_t label) {
    return ((unsigned long long)count << 32) | (unsigned long long)(~label);
}

constexpr int kWinUnroll = 4;   // windows a warp has in flight

__global__ void __launch_bounds__(kLpBlock) k_lp_windows(const LpArgs a) {
    const int lane = threadIdx.x & 31;
    if (blockIdx.x == 0 && a.stats_clear != nullptr) {
        // zero the ring slot two supersteps ahead (never read or written by this one)
        unsigned long long* z = reinterpret_cast<unsigned long long*>(a.stats_clear);
        for (uint32_t i = threadIdx.x; i < sizeof(StepStats) / 8; i += kLpBlock) z[i] = 0ull;
    }
    if (lp_quiet(a, lane)) return;
    const uint64_t w0 = ((uint64_t)blockIdx.x * kLpBlock + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * kLpBlock) >> 5;
    const uint32_t upto = lane == 31 ? 0xFFFFFFFFu : (2u << lane) - 1u;   // lanes 0..lane
    uint32_t n_changed = 0;
    for (uint64_t wb = w0 * kWinUnroll; wb < a.n_windows; wb += nw * kWinUnroll) {
        // loads of kWinUnroll windows issued together: descriptor, then the
        // edge's source and the row's value index, then the label and the
        // row's old label
        LpWindow W[kWinUnroll];
        const LpPart* P[kWinUnroll];
        uint32_t src[kWinUnroll], g[kWinUnroll], label[kWinUnroll], old[kWinUnroll];
        bool has[kWinUnroll], lead[kWinUnroll];
#pragma unroll
        for (int q = 0; q < kWinUnroll; ++q) {
            const bool live = wb + q < a.n_windows;
            W[q] = live ? a.windows[wb + q] : LpWindow{0u, 0u, 0u, 0u};
            P[q] = a.parts + (W[q].n_part >> 6);
            has[q] = (uint32_t)lane < (W[q].n_part & 63u);
            lead[q] = has[q] && ((W[q].starts >> lane) & 1u);
        }
#pragma unroll
        for (int q = 0; q < kWinUnroll; ++q) {
            src[q] = has[q] ? __ldg(P[q]->src + W[q].e0 + lane) : 0u;
            g[q] = lead[q] ? __ldg(a.row_g + W[q].first + (uint32_t)__popc(W[q].starts & upto) - 1u) : 0u;
        }
#pragma unroll
        for (int q = 0; q < kWinUnroll; ++q) {
            label[q] = has[q] ? lp_label(a, *P[q], src[q]) : 0u;
            old[q] = lead[q] ? a.own_cur[g[q]] : 0u;
        }
#pragma unroll
        for (int q = 0; q < kWinUnroll; ++q) {
            // the lanes of this lane's row: [first, end) of the window
            const uint32_t total = W[q].n_part & 63u;
            const uint32_t mine = W[q].starts & upto;
            const uint32_t first = mine ? 31u - (uint32_t)__clz(mine) : 0u;
            const uint32_t above = W[q].starts & ~upto;
            const uint32_t end = above ? (uint32_t)(__ffs(above) - 1) : total;
            const uint32_t row_lanes = (end >= 32u ? 0xFFFFFFFFu : (1u << end) - 1u) & ~((1u << first) - 1u);
            const unsigned act = __ballot_sync(kFull, has[q]);
            if (has[q]) {
                // lanes of the row carrying the same label: the label's count in the row
                unsigned grp;
                if (a.narrow_labels)
                    grp = __match_any_sync(act, (first << 27) | label[q]);
                else
                    grp = __match_any_sync(act, ((unsigned long long)first << 32) | label[q]);
                const uint32_t c = (uint32_t)__popc(grp);
                // the row's largest count, then the smallest label with it
                const uint32_t cmax = __reduce_max_sync(row_lanes, c);
                const uint32_t mode = __reduce_min_sync(row_lanes, c == cmax ? label[q] : kInf);
                if (lead[q]) {
                    a.own_nxt[g[q]] = mode;
                    if (mode != old[q]) {
                        ++n_changed;
                        if (a.changed_bits) atomicOr(a.changed_bits + (g[q] >> 5), 1u << (g[q] & 31u));
                    }
                }
            }
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_changed += __shfl_xor_sync(kFull, n_changed, o);
    if (lane == 0) lp_count(a, n_changed, w0);
}

// add `count` occurrences of `label` to a hub's table (open addressing with
// linear probing; the table is at most half full, so a slot is always found)
__device__ __forceinline__ void lp_table_add(uint32_t* keys, uint32_t* counts, uint32_t log2_size, uint32_t label,
                                             uint32_t count) {
    const uint32_t mask = (1u << log2_size) - 1u;
    uint32_t slot = (label * 0x9E3779B1u) >> (32u - log2_size);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t k = atomicCAS(keys + slot, kInf, label);
        if (k == kInf || k == label) {
            atomicAdd(counts + slot, count);
            return;
        }
        slot = (slot + 1u) & mask;
    }
}

__global__ void __launch_bounds__(kLpBlock) k_lp_chunks(const LpArgs a) {
    __shared__ uint32_t lab[kLpChunk];
    __shared__ uint32_t s_warp[kLpWarps];
    __shared__ unsigned long long s_best[kLpWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (lp_quiet(a, lane)) return;
    uint32_t n_changed = 0;
    for (uint64_t c = blockIdx.x; c < a.n_chunks; c += gridDim.x) {
        const LpRow r = a.chunks[c];
        const LpPart P = a.parts[r.part];
        const uint32_t n = r.n;
        uint32_t np2 = 2;
        while (np2 < n) np2 <<= 1;
        for (uint32_t i0 = 0; i0 < np2; i0 += (uint32_t)kLpBlock * kGatherUnroll) {
            uint32_t s[kGatherUnroll];
#pragma unroll
            for (int q = 0; q < kGatherUnroll; ++q) {
                const uint32_t i = i0 + (uint32_t)q * kLpBlock + (uint32_t)tid;
                s[q] = i < n ? __ldg(P.src + r.e0 + i) : 0u;
            }
#pragma unroll
            for (int q = 0; q < kGatherUnroll; ++q) {
                const uint32_t i = i0 + (uint32_t)q * kLpBlock + (uint32_t)tid;
                if (i < np2) lab[i] = i < n ? lp_label(a, P, s[q]) : kInf;   // padding sorts last
            }
        }
        __syncthreads();
        for (uint32_t k = 2; k <= np2; k <<= 1) {   // bitonic sort, ascending
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = (uint32_t)tid; i < np2; i += kLpBlock) {
                    const uint32_t l = i ^ j;
                    if (l > i) {
                        const uint32_t x = lab[i], y = lab[l];
                        if ((x > y) == ((i & k) == 0u)) {
                            lab[i] = y;
                            lab[l] = x;
                        }
                    }
                }
                __syncthreads();
            }
        }
        // thread t owns lab[lo, hi); a run starts where the label changes
        const uint32_t per = (n + kLpBlock - 1) / kLpBlock;
        const uint32_t lo = min(n, (uint32_t)tid * per), hi = min(n, lo + per);
        uint32_t last_start = 0;   // 0 is always a start: the identity of the max-scan
        for (uint32_t i = lo; i < hi; ++i)
            if (i == 0 || lab[i] != lab[i - 1]) last_start = i;
        // exclusive max-scan of the segments' last starts over the block
        uint32_t incl = last_start;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl = max(incl, y);
        }
        if (lane == 31) s_warp[warp] = incl;
        __syncthreads();
        uint32_t before = __shfl_up_sync(kFull, incl, 1);
        if (lane == 0) before = 0;
        for (int w = 0; w < warp; ++w) before = max(before, s_warp[w]);
        // walk the segment: at each run end, its length from the run's start
        uint32_t start = before;
        unsigned long long best = 0ull;
        for (uint32_t i = lo; i < hi; ++i) {
            if (i == 0 || lab[i] != lab[i - 1]) start = i;
            if (i + 1 == n || lab[i + 1] != lab[i]) {
                const uint32_t len = i - start + 1;
                if (r.hub != kInf) {
                    const LpHub H = a.hubs[r.hub];
                    lp_table_add(a.keys + H.table, a.counts + H.table, H.log2_size, lab[i], len);
                } else {
                    best = max(best, mode_key(len, lab[i]));
                }
            }
        }
        if (r.hub == kInf) {
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(kFull, best, o));
            if (lane == 0) s_best[warp] = best;
            __syncthreads();
            if (tid == 0) {
                unsigned long long b = 0ull;
                for (int w = 0; w < kLpWarps; ++w) b = max(b, s_best[w]);
                if (lp_apply(a, r.g, ~(uint32_t)b)) ++n_changed;
            }
        }
        __syncthreads();   // lab[] and the shared arrays are reused by the next row
    }
    if (tid == 0) lp_count(a, n_changed, blockIdx.x);
}

__global__ void __launch_bounds__(kLpBlock) k_lp_hubs(const LpArgs a) {
    __shared__ unsigned long long s_best[kLpWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    if (lp_quiet(a, lane)) return;
    uint32_t n_changed = 0;
    for (uint32_t h = blockIdx.x; h < a.n_hubs; h += gridDim.x) {
        const LpHub H = a.hubs[h];
        const uint64_t size = 1ull << H.log2_size;
        uint32_t* keys = a.keys + H.table;
        uint32_t* counts = a.counts + H.table;
        unsigned long long best = 0ull;
        for (uint64_t i = (uint64_t)tid; i < size; i += kLpBlock) {
            const uint32_t k = keys[i];
            if (k != kInf) {
                best = max(best, mode_key(counts[i], k));
                keys[i] = kInf;   // empty again for the next superstep
                counts[i] = 0u;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(kFull, best, o));
        if (lane == 0) s_best[warp] = best;
        __syncthreads();
        if (tid == 0) {
            unsigned long long b = 0ull;
            for (int w = 0; w < kLpWarps; ++w) b = max(b, s_best[w]);
            if (lp_apply(a, H.g, ~(uint32_t)b)) ++n_changed;
        }
        __syncthreads();
    }
    if (tid == 0) lp_count(a, n_changed, blockIdx.x + 17u);
}

}  // namespace

cudaError_t launch_lp_superstep(const LpArgs& a, cudaStream_t s) {
    const uint32_t g_win =
        (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((a.n_windows + 8 * kWinUnroll - 1) / (8 * kWinUnroll),
                                                           152ull * 16));
    k_lp_windows<<<g_win, kLpBlock, 0, s>>>(a);   // also clears the stat slot two supersteps ahead
    if (a.n_chunks)
        k_lp_chunks<<<(uint32_t)std::min<uint64_t>(a.n_chunks, 152ull * 8), kLpBlock, 0, s>>>(a);
    if (a.n_hubs) k_lp_hubs<<<(uint32_t)std::min<uint64_t>(a.n_hubs, 152ull * 8), kLpBlock, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gxp
