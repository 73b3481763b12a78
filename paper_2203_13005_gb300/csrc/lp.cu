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
//  * rows with 33..256 in-edges: a warp per row, 257..2048: a CTA per row;
//    both count the labels in a shared-memory hash table (2^k >= 2 in-degree
//    slots, open addressing; equal labels of a warp added once) and reduce
//    (count, -label) over it (sorting each row with a bitonic network in a
//    CTA, up to 78 barriers a row, ran 3x slower on R-MAT);
//  * hub rows (more in-edges): each chunk of 2048 is counted the same way
//    and its counts are added into the hub's global hash table; segments of
//    4096 slots that a label entered this superstep, spread over all CTAs,
//    reduce the tables into a 64-bit maximum per hub and empty them (once
//    labels settle, most segments stay empty and are skipped), and a thread
//    per hub applies.
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

// kOnePart: one partition (no cached copies): every source is a local
// index into the label array, read without the partition descriptor
template <bool kOnePart>
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
        const uint32_t* src0 = kOnePart ? a.parts[0].src : nullptr;
#pragma unroll
        for (int q = 0; q < kWinUnroll; ++q) {
            src[q] = has[q] ? __ldg((kOnePart ? src0 : P[q]->src) + W[q].e0 + lane) : 0u;
            g[q] = lead[q] ? __ldg(a.row_g + W[q].first + (uint32_t)__popc(W[q].starts & upto) - 1u) : 0u;
        }
#pragma unroll
        for (int q = 0; q < kWinUnroll; ++q) {
            if constexpr (kOnePart) label[q] = has[q] ? __ldg(a.own_cur + src[q]) : 0u;
            else label[q] = has[q] ? lp_label(a, *P[q], src[q]) : 0u;
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

// add `count` occurrences of `label` to a hash table of 2^log2_size slots
// (open addressing with linear probing; a table of 2^k >= 2 n slots, or 2^32,
// has a free slot for every distinct label, so one is always found). Works
// on global and on shared memory tables.
__device__ __forceinline__ uint32_t lp_table_add(uint32_t* keys, uint32_t* counts, uint32_t log2_size,
                                                 uint32_t label, uint32_t count) {
    const uint32_t mask = log2_size >= 32u ? 0xFFFFFFFFu : (1u << log2_size) - 1u;
    uint32_t slot = (label * 0x9E3779B1u) >> (32u - log2_size);
    for (uint64_t probe = 0; probe <= mask; ++probe) {
        const uint32_t k = atomicCAS(keys + slot, kInf, label);
        if (k == kInf || k == label) {
            atomicAdd(counts + slot, count);
            return slot;
        }
        slot = (slot + 1u) & mask;
    }
    return 0u;
}

__device__ __forceinline__ unsigned long long block_max(unsigned long long v, unsigned long long* s_red) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = max(v, __shfl_xor_sync(kFull, v, o));
    if (lane == 0) s_red[warp] = v;
    __syncthreads();
    unsigned long long b = 0ull;
    for (int w = 0; w < kLpWarps; ++w) b = max(b, s_red[w]);
    return b;
}

// Rows of 33..256 in-edges, a warp each (8 rows in flight per CTA): the
// warp counts the row's labels in its own shared-memory hash table (2^k >=
// 2n slots, at most 512), takes the largest (count, -label) over the table
// with a warp reduction and empties it.
__global__ void __launch_bounds__(kLpBlock) k_lp_warp_rows(const LpArgs a) {
    __shared__ uint32_t t_key[kLpWarps][2 * kLpWarpRow], t_cnt[kLpWarps][2 * kLpWarpRow];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lp_quiet(a, lane)) return;
    uint32_t* keys = t_key[warp];
    uint32_t* cnts = t_cnt[warp];
    for (uint32_t i = (uint32_t)lane; i < 2 * kLpWarpRow; i += 32u) {
        keys[i] = kInf;
        cnts[i] = 0u;
    }
    __syncwarp();
    const uint64_t w0 = ((uint64_t)blockIdx.x * kLpBlock + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * kLpBlock) >> 5;
    uint32_t n_changed = 0;
    for (uint64_t ri = w0; ri < a.n_warp_rows; ri += nw) {
        const LpRow r = a.warp_rows[ri];
        const LpPart P = a.parts[r.part];
        const uint32_t n = r.n;
        uint32_t lg = 1;
        while ((1u << lg) < 2u * n) ++lg;
        for (uint32_t i0 = 0; i0 < n; i0 += 32u * kGatherUnroll) {
            uint32_t sv[kGatherUnroll], lab[kGatherUnroll];
#pragma unroll
            for (int q = 0; q < kGatherUnroll; ++q) {
                const uint32_t i = i0 + 32u * q + (uint32_t)lane;
                sv[q] = i < n ? __ldg(P.src + r.e0 + i) : 0u;
            }
#pragma unroll
            for (int q = 0; q < kGatherUnroll; ++q) {
                const uint32_t i = i0 + 32u * q + (uint32_t)lane;
                lab[q] = i < n ? lp_label(a, P, sv[q]) : 0u;
            }
#pragma unroll
            for (int q = 0; q < kGatherUnroll; ++q) {
                const bool has = i0 + 32u * q + (uint32_t)lane < n;
                const unsigned act = __ballot_sync(kFull, has);
                if (has) {
                    const unsigned grp = __match_any_sync(act, lab[q]);
                    if (lane == __ffs(grp) - 1) lp_table_add(keys, cnts, lg, lab[q], (uint32_t)__popc(grp));
                }
            }
        }
        __syncwarp();
        unsigned long long best = 0ull;
        for (uint32_t i = (uint32_t)lane; i < (1u << lg); i += 32u) {
            const uint32_t k = keys[i];
            if (k != kInf) {
                best = max(best, mode_key(cnts[i], k));
                keys[i] = kInf;
                cnts[i] = 0u;
            }
        }
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) best = max(best, __shfl_xor_sync(kFull, best, o));
        if (lane == 0 && lp_apply(a, r.g, ~(uint32_t)best)) ++n_changed;
        __syncwarp();
    }
    if (lane == 0) lp_count(a, n_changed, w0);
}

// Rows of 257..2048 in-edges (hub = kInf) and chunks of 2048 of hub rows: the
// CTA counts the labels in a shared-memory hash table (2^k >= 2n slots),
// then takes the mode (a row) or adds its counts into the hub's table.
__global__ void __launch_bounds__(kLpBlock) k_lp_rows(const LpArgs a) {
    __shared__ uint32_t t_key[2 * kLpChunk], t_cnt[2 * kLpChunk];
    __shared__ unsigned long long s_red[kLpWarps];
    const int tid = threadIdx.x, lane = tid & 31;
    if (lp_quiet(a, lane)) return;
    for (uint32_t i = (uint32_t)tid; i < 2 * kLpChunk; i += kLpBlock) {
        t_key[i] = kInf;
        t_cnt[i] = 0u;
    }
    __syncthreads();
    uint32_t n_changed = 0;
    for (uint64_t c = blockIdx.x; c < a.n_chunks; c += gridDim.x) {
        const LpRow r = a.chunks[c];
        const LpPart P = a.parts[r.part];
        const uint32_t n = r.n;
        uint32_t lg = 1;
        while ((1u << lg) < 2u * n) ++lg;
        const uint32_t size = 1u << lg;
        for (uint32_t i0 = 0; i0 < n; i0 += (uint32_t)kLpBlock * kGatherUnroll) {
            uint32_t sv[kGatherUnroll], lab[kGatherUnroll];
#pragma unroll
            for (int q = 0; q < kGatherUnroll; ++q) {
                const uint32_t i = i0 + (uint32_t)q * kLpBlock + (uint32_t)tid;
                sv[q] = i < n ? __ldg(P.src + r.e0 + i) : 0u;
            }
#pragma unroll
            for (int q = 0; q < kGatherUnroll; ++q) {
                const uint32_t i = i0 + (uint32_t)q * kLpBlock + (uint32_t)tid;
                lab[q] = i < n ? lp_label(a, P, sv[q]) : 0u;
            }
            // lanes with the same label add once (labels repeat as they settle:
            // one slot's atomics would otherwise serialize)
#pragma unroll
            for (int q = 0; q < kGatherUnroll; ++q) {
                const bool has = i0 + (uint32_t)q * kLpBlock + (uint32_t)tid < n;
                const unsigned act = __ballot_sync(kFull, has);
                if (has) {
                    const unsigned grp = __match_any_sync(act, lab[q]);
                    if (lane == __ffs(grp) - 1) lp_table_add(t_key, t_cnt, lg, lab[q], (uint32_t)__popc(grp));
                }
            }
        }
        __syncthreads();
        // read the counts and empty the table for the next row
        unsigned long long best = 0ull;
        for (uint32_t i = (uint32_t)tid; i < size; i += kLpBlock) {
            const uint32_t k = t_key[i];
            if (k != kInf) {
                const uint32_t cnt = t_cnt[i];
                if (r.hub == kInf) {
                    best = max(best, mode_key(cnt, k));
                } else {
                    const LpHub H = a.hubs[r.hub];
                    const uint32_t slot = lp_table_add(a.keys + H.table, a.counts + H.table, H.log2_size, k, cnt);
                    a.seg_used[H.seg0 + slot / kLpSegment] = 1u;   // same value from every writer
                }
                t_key[i] = kInf;
                t_cnt[i] = 0u;
            }
        }
        if (r.hub == kInf) {
            best = block_max(best, s_red);
            if (tid == 0 && lp_apply(a, r.g, ~(uint32_t)best)) ++n_changed;
        }
        __syncthreads();   // the table and s_red are reused by the next row
    }
    if (tid == 0) lp_count(a, n_changed, blockIdx.x);
}

// hub tables, a segment per CTA: the best (count, -label) of the segment
// goes into the hub's 64-bit maximum, and the segment is emptied
__global__ void __launch_bounds__(kLpBlock) k_lp_segments(const LpArgs a) {
    __shared__ unsigned long long s_red[kLpWarps];
    const int tid = threadIdx.x, lane = tid & 31;
    if (lp_quiet(a, lane)) return;
    for (uint32_t sg = blockIdx.x; sg < a.n_segments; sg += gridDim.x) {
        if (!a.seg_used[sg]) continue;   // no label took a slot here this superstep (uniform in the CTA)
        const LpSegment S = a.segments[sg];
        uint32_t* keys = a.keys + S.slot0;
        uint32_t* counts = a.counts + S.slot0;
        unsigned long long best = 0ull;
        for (uint32_t i = (uint32_t)tid; i < S.n; i += kLpBlock) {
            const uint32_t k = keys[i];
            if (k != kInf) {
                best = max(best, mode_key(counts[i], k));
                keys[i] = kInf;   // empty again for the next superstep
                counts[i] = 0u;
            }
        }
        best = block_max(best, s_red);
        if (tid == 0) {
            if (best) atomicMax(a.hub_best + S.hub, best);
            a.seg_used[sg] = 0u;
        }
        __syncthreads();
    }
}

// a thread per hub: apply the mode its segments agreed on
__global__ void k_lp_hubs(const LpArgs a) {
    const int lane = threadIdx.x & 31;
    if (lp_quiet(a, lane)) return;
    uint32_t n_changed = 0;
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < a.n_hubs; h += gridDim.x * blockDim.x) {
        const unsigned long long best = a.hub_best[h];
        a.hub_best[h] = 0ull;
        if (lp_apply(a, a.hubs[h].g, ~(uint32_t)best)) ++n_changed;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) n_changed += __shfl_xor_sync(kFull, n_changed, o);
    if (lane == 0) lp_count(a, n_changed, blockIdx.x * 8u + (threadIdx.x >> 5) + 17u);
}

}  // namespace

cudaError_t launch_lp_superstep(const LpArgs& a, cudaStream_t s) {
    const uint32_t g_win =
        (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>((a.n_windows + 8 * kWinUnroll - 1) / (8 * kWinUnroll),
                                                           152ull * 16));
    if (a.n_parts == 1) k_lp_windows<true><<<g_win, kLpBlock, 0, s>>>(a);   // also clears the stat slot
    else k_lp_windows<false><<<g_win, kLpBlock, 0, s>>>(a);                 // two supersteps ahead
    if (a.n_warp_rows)
        k_lp_warp_rows<<<(uint32_t)std::min<uint64_t>((a.n_warp_rows + 7) / 8, 152ull * 8), kLpBlock, 0, s>>>(a);
    if (a.n_chunks) k_lp_rows<<<(uint32_t)std::min<uint64_t>(a.n_chunks, 152ull * 4), kLpBlock, 0, s>>>(a);
    if (a.n_segments)
        k_lp_segments<<<(uint32_t)std::min<uint64_t>(a.n_segments, 152ull * 8), kLpBlock, 0, s>>>(a);
    if (a.n_hubs) k_lp_hubs<<<(uint32_t)std::min<uint64_t>((a.n_hubs + 255) / 256, 152ull * 4), 256, 0, s>>>(a);
    return cudaGetLastError();
}

}  // namespace gxp
