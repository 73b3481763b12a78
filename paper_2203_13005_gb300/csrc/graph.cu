// Load-time and per-superstep helper kernels:
//  * edge-block (tile) construction over a partition's CSC — the paired edge
//    and vertex blocks of Section II-B, with hub vertices split;
//  * out-degrees (PageRank's MSGGen divides by them);
//  * initial vertex values and cache (ghost) fills;
//  * synchronization caching and skipping between partitions (Section
//    III-B, Algorithm 3): changed ∩ boundary -> global data queue (sorted by
//    id) -> the caches of the partitions that read those vertices; the
//    exchange is skipped on the device when the queue is empty everywhere.
#include "frontier.cuh"

#include <algorithm>

namespace gxp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;

// -------------------------------------------------------------- tiles

// Merge-path position of a cut (vertex ends consumed i, edges consumed j): a
// vertex end weighs kVertexCost items, an edge one.
__device__ __forceinline__ uint64_t cut_pos(uint64_t c) {
    return (c >> 32) * kVertexCost + (c & 0xFFFFFFFFull);
}

// Cut k of the merged sequence (vertex ends + edges) at weighted position k*T,
// clamped before the end of the vertex it falls in and snapped back to the
// start of that vertex unless it is a hub (in-degree > H). Packed as
// (vertex << 32 | edge).
__global__ void k_cuts(const uint32_t* __restrict__ col_ptr, uint32_t n, uint32_t n_edges,
                       uint32_t T, uint32_t H, uint32_t nt, uint64_t* __restrict__ cuts) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k > nt) return;
    const uint64_t total = (uint64_t)n * kVertexCost + n_edges;
    const uint64_t D = min((uint64_t)k * T, total);
    // largest i in [0, n] with i*cost + col_ptr[i] <= D
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo + 1u) / 2u;
        if ((uint64_t)mid * kVertexCost + col_ptr[mid] <= D) lo = mid;
        else hi = mid - 1u;
    }
    const uint32_t i = lo;
    uint64_t j = D - (uint64_t)i * kVertexCost;
    if (i < n) {
        if (j > col_ptr[i + 1]) j = col_ptr[i + 1];   // inside vertex i's end item: cut before it
        if (j > col_ptr[i] && col_ptr[i + 1] - col_ptr[i] <= H) j = col_ptr[i];
    }
    cuts[k] = ((uint64_t)i << 32) | j;
}

__device__ uint32_t upper_bound_cut(const uint64_t* cuts, uint32_t nt, uint64_t p) {
    // first k in [0, nt] with cut_pos(cuts[k]) > p (nt + 1 if none)
    uint32_t lo = 0, hi = nt + 1u;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (cut_pos(cuts[mid]) > p) hi = mid;
        else lo = mid + 1u;
    }
    return lo;
}

__global__ void k_tiles(const uint32_t* __restrict__ col_ptr, uint32_t n, const uint64_t* __restrict__ cuts,
                        uint32_t nt, uint32_t part, uint32_t tile_base, Tile* __restrict__ tiles) {
    const uint32_t k = blockIdx.x * blockDim.x + threadIdx.x;
    if (k >= nt) return;
    const uint32_t i0 = (uint32_t)(cuts[k] >> 32), j0 = (uint32_t)cuts[k];
    const uint32_t i1 = (uint32_t)(cuts[k + 1] >> 32), j1 = (uint32_t)cuts[k + 1];
    const bool head = i0 < n && j0 > col_ptr[i0];
    const bool tail = i1 < n && j1 > col_ptr[i1];
    Tile t;
    t.v0 = i0;
    t.nv = i1 - i0 + (tail ? 1u : 0u);
    t.e0 = j0;
    t.ne = j1 - j0;
    t.part = part;
    t.flags = (head ? kHeadOpen : 0u) | (tail ? kTailOpen : 0u);
    t.hub_t0 = kInf;
    t.nparts = 0;
    if (t.nv == 0u && t.ne == 0u) t.flags = 0u;
    if (head) {
        const uint64_t p_first = (uint64_t)i0 * kVertexCost + col_ptr[i0];
        t.hub_t0 = tile_base + upper_bound_cut(cuts, nt, p_first) - 1u;
    }
    if (tail && !(head && t.nv == 1u)) {
        const uint64_t p_end = (uint64_t)i1 * kVertexCost + col_ptr[i1 + 1];
        const uint32_t t1 = upper_bound_cut(cuts, nt, p_end) - 1u;
        t.nparts = t1 - k + 1u;
    }
    tiles[k] = t;
}

// ----------------------------------------------------------- out-degree

// Sources below kOutdegHot are counted in shared memory and flushed once per
// block: atomics on one address serialize, and power-law generators that do
// not permute ids (R-MAT) put their hubs at the lowest ids (the hottest
// R-MAT 22 source has ~160K out-edges, which took ~1 ms of global atomics).
constexpr uint32_t kOutdegHot = 8192;

__global__ void __launch_bounds__(256) k_outdeg(const uint32_t* __restrict__ src, uint64_t n_edges, uint32_t n_own,
                                                uint32_t v_begin, const uint32_t* __restrict__ ghost_gid,
                                                uint32_t* __restrict__ outdeg) {
    __shared__ uint32_t hot[kOutdegHot];
    for (uint32_t i = threadIdx.x; i < kOutdegHot; i += blockDim.x) hot[i] = 0u;
    __syncthreads();
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n_edges;
         e += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t u = src[e];
        const uint32_t g = u < n_own ? v_begin + u : ghost_gid[u - n_own];
        if (g < kOutdegHot) {
            atomicAdd(&hot[g], 1u);
        } else {
            // one atomic per distinct source among the active lanes
            const unsigned act = __activemask();
            const unsigned peers = __match_any_sync(act, g);
            if ((threadIdx.x & 31) == (unsigned)(__ffs(peers) - 1)) atomicAdd(&outdeg[g], (uint32_t)__popc(peers));
        }
    }
    __syncthreads();
    for (uint32_t i = threadIdx.x; i < kOutdegHot; i += blockDim.x)
        if (hot[i]) atomicAdd(&outdeg[i], hot[i]);
}

__global__ void k_validate(const uint32_t* __restrict__ col_ptr, uint32_t n_own,
                           const uint32_t* __restrict__ src, uint64_t n_edges, uint32_t n_local,
                           uint32_t* err) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n_edges; e += stride)
        if (src[e] >= n_local) atomicOr(err, kErrBounds);
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < n_own; v += stride)
        if (col_ptr[v] > col_ptr[v + 1]) atomicOr(err, kErrInput);
    if (blockIdx.x == 0 && threadIdx.x == 0 && (col_ptr[0] != 0u || (uint64_t)col_ptr[n_own] != n_edges))
        atomicOr(err, kErrInput);
}

// CSC imported as given: col_ptr (u64) -> u32 with its checks (bit 0 of
// err: not running from 0 to n_edges or decreasing), sources < n_local (bit 1)
__global__ void k_csc_import(const uint64_t* __restrict__ cp64, uint32_t n, uint64_t n_edges,
                             uint32_t* __restrict__ cp32, const uint32_t* __restrict__ src, uint32_t n_local,
                             uint32_t* err) {
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    for (uint64_t v = t0; v <= n; v += stride) {
        const uint64_t c = cp64[v];
        const bool bad = c > n_edges || (v == 0 && c != 0) || (v == n && c != n_edges) || (v < n && cp64[v + 1] < c);
        if (bad) atomicOr(err, 1u);
        cp32[v] = (uint32_t)c;
    }
    bool oob = false;
    for (uint64_t e = t0; e < n_edges; e += stride) oob |= src[e] >= n_local;
    if (__any_sync(0xFFFFFFFFu, oob) && (threadIdx.x & 31) == 0) atomicOr(err, 2u);
}

// ------------------------------------------------------- initial values


__global__ void k_init_values(int algo, uint32_t ppr_source, uint32_t n, uint32_t source, uint32_t* own,
                              float* rank, const uint32_t* outdeg, StepStats* st, const uint32_t* label_of) {
    unsigned long long dang = 0;
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) {
        if (algo == (int)Algo::SSSP) {
            own[v] = (v == source) ? 0u : kInf;
        } else if (algo == (int)Algo::CC || algo == (int)Algo::LP) {
            own[v] = label_of ? label_of[v] : v;   // CC / LP labels are input ids
        } else {
            // PageRank: r_0 = 1/N everywhere; personalized PageRank: r_0 = e_source
            const float r0 = ppr_source == kInf ? (float)(1.0 / (double)n) : (v == ppr_source ? 1.0f : 0.0f);
            rank[v] = r0;
            const uint32_t od = outdeg[v];
            own[v] = __float_as_uint(od ? __fdiv_rn(r0, (float)od) : 0.0f);
            if (od == 0u) dang += fx_of(r0);
        }
    }
    if (algo == (int)Algo::PR) {
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) dang += __shfl_xor_sync(kFull, dang, o);
        if ((threadIdx.x & 31) == 0 && dang)
            atomicAdd(&st->dangling_fx[(blockIdx.x * (blockDim.x / 32) + threadIdx.x / 32) % kStatLanes], dang);
    }
}

__global__ void k_identity_slots(uint32_t* a, uint32_t* b, uint32_t* c, uint32_t v) {
    *a = v;
    *b = v;
    *c = v;
}

__global__ void k_init_ghosts(uint32_t n_ghost, const uint32_t* __restrict__ gid,
                              const uint32_t* __restrict__ own, uint32_t* __restrict__ ghost) {
    for (uint32_t g = blockIdx.x * blockDim.x + threadIdx.x; g < n_ghost; g += gridDim.x * blockDim.x)
        ghost[g] = own[gid[g]];
}

// ----------------------------------------------------------------- sync

__device__ __forceinline__ uint32_t range_mask(uint32_t w, uint32_t v_lo, uint32_t v_hi) {
    const uint32_t base = w * 32u;
    const uint32_t lo = v_lo > base ? v_lo - base : 0u;
    const uint32_t hi = v_hi < base + 32u ? v_hi - base : 32u;
    if (hi <= lo) return 0u;
    const uint32_t upper = hi == 32u ? kFull : ((1u << hi) - 1u);
    return upper & ~((1u << lo) - 1u);
}

constexpr int kSyncBlock = 256;

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t x, uint32_t* s_warp, uint32_t& total) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t incl = x;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) s_warp[warp] = incl;
    __syncthreads();
    if (warp == 0) {
        uint32_t v = lane < kSyncBlock / 32 ? s_warp[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(kFull, v, o);
            if (lane >= o) v += y;
        }
        if (lane < kSyncBlock / 32) s_warp[lane] = v;
    }
    __syncthreads();
    const uint32_t warp_off = warp ? s_warp[warp - 1] : 0u;
    total = s_warp[kSyncBlock / 32 - 1];
    __syncthreads();
    return warp_off + incl - x;
}

// Count changed ∩ boundary per block; the last block to finish turns the
// counts into per-block offsets and decides whether the exchange is skipped.
__global__ void __launch_bounds__(kSyncBlock) k_sync_count(const SyncArgs a) {
    __shared__ uint32_t s_warp[kSyncBlock / 32];
    __shared__ bool s_last;
    const uint32_t p = blockIdx.y;
    const PartDev P = a.parts[p];
    const uint32_t v_lo = P.v_begin, v_hi = P.v_begin + P.n_own;
    const uint32_t w_lo = v_lo >> 5, w_hi = (v_hi + 31u) >> 5;
    const uint32_t w = w_lo + blockIdx.x * kSyncBlock + threadIdx.x;
    uint32_t c = 0;
    if (P.n_own && w < w_hi) c = __popc(a.changed_bits[w] & a.boundary_bits[w] & range_mask(w, v_lo, v_hi));
    uint32_t total;
    block_excl_scan(c, s_warp, total);
    if (threadIdx.x == 0) {
        a.block_counts[p * a.blocks_x + blockIdx.x] = total;
        __threadfence();
        const uint32_t ticket = atomicAdd(a.done_ctr, 1u);
        s_last = ticket == gridDim.x * gridDim.y - 1u;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    unsigned long long grand = 0;
    for (uint32_t q = 0; q < a.n_parts; ++q) {
        uint32_t run = 0;
        for (uint32_t b0 = 0; b0 < a.blocks_x; b0 += kSyncBlock) {
            const uint32_t b = b0 + threadIdx.x;
            const uint32_t x = b < a.blocks_x ? __ldcg(&a.block_counts[q * a.blocks_x + b]) : 0u;
            uint32_t tot;
            const uint32_t ex = block_excl_scan(x, s_warp, tot);
            if (b < a.blocks_x) a.block_offsets[q * a.blocks_x + b] = run + ex;
            run += tot;
        }
        if (threadIdx.x == 0) a.part_counts[q] = run;
        grand += run;
    }
    if (threadIdx.x == 0) {
        a.stats_out->boundary_changed = grand;
        a.stats_out->skipped = grand == 0 ? 1ull : 0ull;
        a.stats_out->exchanged = 1ull;
        // the next superstep pulls anyway when its frontier would be too much
        // work to push: its own vertices' items and out-edges, plus at least
        // one item per changed boundary vertex for the copies that would join
        // (each has a copy somewhere); then the copies are not listed. Nor
        // are they when the superstep did not list its own vertices.
        bool list = a.fc.list_out != nullptr && __ldcg(&a.stats_out->unlisted) == 0ull;
        if (list && a.fc.direction == GXP_DIR_AUTO) {
            const unsigned long long ne = __ldcg(&a.stats_out->list_ne);
            list = ((ne >> 32) + (ne & 0xFFFFFFFFull) + grand) * (unsigned long long)a.fc.push_div <=
                   a.fc.total_edges;
        }
        a.stats_out->list_copies = list ? 1ull : 0ull;
        *a.done_ctr = 0u;
    }
}

// Write each partition's global data queue (ascending ids): the changed
// boundary vertices with their new values.
__global__ void __launch_bounds__(kSyncBlock) k_sync_write(const SyncArgs a) {
    __shared__ uint32_t s_warp[kSyncBlock / 32];
    if (a.stats_out->skipped) return;   // uniform: Section III-B3 skip
    const uint32_t p = blockIdx.y;
    const PartDev P = a.parts[p];
    const uint32_t v_lo = P.v_begin, v_hi = P.v_begin + P.n_own;
    const uint32_t w_lo = v_lo >> 5, w_hi = (v_hi + 31u) >> 5;
    const uint32_t w = w_lo + blockIdx.x * kSyncBlock + threadIdx.x;
    uint32_t bits = 0;
    if (P.n_own && w < w_hi) bits = a.changed_bits[w] & a.boundary_bits[w] & range_mask(w, v_lo, v_hi);
    uint32_t total;
    uint32_t pos = block_excl_scan(__popc(bits), s_warp, total);
    if (P.n_own == 0 || blockIdx.x * kSyncBlock >= w_hi - w_lo) return;
    pos += a.block_offsets[p * a.blocks_x + blockIdx.x] + (uint32_t)a.gdq_base[p];
    // A warp writes its 32 words' pairs one word at a time, lane l taking the
    // word's bit l: the word's vertices are 32 consecutive ids, so the value
    // load is one 128-byte line and the pairs land at consecutive positions
    // (a thread walking its own word wrote 32 scattered runs per store).
    const uint32_t lane = threadIdx.x & 31u;
    unsigned todo = __ballot_sync(kFull, bits != 0u);
    while (todo) {
        const int j = __ffs(todo) - 1;
        todo &= todo - 1u;
        const uint32_t bj = __shfl_sync(kFull, bits, j);
        const uint32_t pj = __shfl_sync(kFull, pos, j);
        const uint32_t wj = __shfl_sync(kFull, w, j);
        if ((bj >> lane) & 1u) {
            const uint32_t gid = wj * 32u + lane;
            const uint32_t at = pj + __popc(bj & ((1u << lane) - 1u));
            a.gdq_ids[at] = gid;
            a.gdq_vals[at] = a.own_val[gid];
        }
    }
}

// Caching (Section III-B): every cached copy of an uploaded vertex takes its
// new value. Each partition's cache list is sorted by global id, so a thread
// per cached copy reads the changed bits and the owners' values in
// ascending order and writes the cache sequentially.
// With a cache budget only the kept copies (pull_list) are refreshed here.
// With frontier lists on, every copy whose vertex changed (cached or not)
// also joins the next frontier as slot n_vertices + g: the partition that
// holds it relaxes its in-edges from that vertex if the next superstep pushes.
__global__ void k_sync_pull(const SyncArgs a) {
    if (a.stats_out->skipped) return;   // uniform: Section III-B3 skip
    const bool list = a.stats_out->list_copies != 0ull;   // decided by k_sync_count for every CTA
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    auto pull = [&](uint32_t g) -> bool {   // copy g takes its owner's new value if it changed
        const uint32_t gid = a.ghost_gid[g];
        const bool ch = ((a.changed_bits[gid >> 5] >> (gid & 31u)) & 1u) != 0u;
        // not cached: downloaded when used (lru.cu)
        if (ch && (!a.cached || (a.cached[g] & 1u))) a.ghost[g] = a.own_val[gid];
        return ch;
    };
    if (!list) {
        // four copies per thread and round, their loads issued together: a
        // thread keeps four independent chains (id -> changed bit -> value)
        // in flight instead of one
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x, n = a.n_pull;
        for (uint64_t g0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; g0 < n; g0 += 4u * stride) {
            uint32_t gid[4], word[4], val[4];
            bool wr[4];
#pragma unroll
            for (int k = 0; k < 4; ++k) gid[k] = g0 + k * stride < n ? a.ghost_gid[g0 + k * stride] : 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) word[k] = g0 + k * stride < n ? a.changed_bits[gid[k] >> 5] : 0u;
#pragma unroll
            for (int k = 0; k < 4; ++k) {
                const uint64_t g = g0 + k * stride;
                // not cached: downloaded when used (lru.cu)
                wr[k] = g < n && ((word[k] >> (gid[k] & 31u)) & 1u) != 0u && (!a.cached || (a.cached[g] & 1u));
                val[k] = wr[k] ? a.own_val[gid[k]] : 0u;
            }
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (wr[k]) a.ghost[g0 + k * stride] = val[k];
        }
        return;
    }
    // The changed copies join the next frontier. A CTA takes a contiguous
    // chunk: pass 1 pulls and counts their items, one atomic reserves the
    // CTA's range of the list (one per warp made the list counter a
    // same-address bottleneck), pass 2 writes the items 256 copies at a time
    // at block-scanned offsets.
    __shared__ uint32_t s_items[8], s_edges[8];
    __shared__ unsigned long long s_base;
    const uint64_t per = ((((uint64_t)a.n_pull + gridDim.x - 1) / gridDim.x) + 255) & ~255ull;
    const uint64_t lo = min((uint64_t)a.n_pull, (uint64_t)blockIdx.x * per), hi = min((uint64_t)a.n_pull, lo + per);
    if (lo >= hi) return;   // uniform over the CTA
    auto degree = [&](uint32_t g) { return __ldg(a.out_ptr + a.n_vertices + g + 1) - __ldg(a.out_ptr + a.n_vertices + g); };
    uint32_t items = 0, edges = 0;
    for (uint64_t g = lo + threadIdx.x; g < hi; g += blockDim.x) {
        if (pull((uint32_t)g)) {
            const uint32_t d = degree((uint32_t)g);
            items += frontier_items(d);
            edges += d;
        }
    }
    items = __reduce_add_sync(0xFFFFFFFFu, items);
    edges = __reduce_add_sync(0xFFFFFFFFu, edges);
    if (lane == 0) {
        s_items[warp] = items;
        s_edges[warp] = edges;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t ti = 0, te = 0;
        for (int w = 0; w < 8; ++w) {
            ti += s_items[w];
            te += s_edges[w];
        }
        s_base = ti ? atomicAdd(&a.stats_out->list_ne, list_pack(ti, te)) >> 32 : 0ull;
    }
    __syncthreads();
    unsigned long long run = s_base;
    for (uint64_t r0 = lo; r0 < hi; r0 += blockDim.x) {
        const uint64_t g = r0 + threadIdx.x;
        bool ch = false;
        if (g < hi) {
            const uint32_t gid = a.ghost_gid[g];
            ch = ((a.changed_bits[gid >> 5] >> (gid & 31u)) & 1u) != 0u;
        }
        const uint32_t nit = ch ? frontier_items(degree((uint32_t)g)) : 0u;
        const uint32_t incl = warp_inclusive_scan(nit, lane);
        __syncthreads();   // the previous round's totals are read
        if (lane == 31) s_items[warp] = incl;
        __syncthreads();
        uint32_t before = 0, round = 0;
        for (int w = 0; w < 8; ++w) {
            if (w < warp) before += s_items[w];
            round += s_items[w];
        }
        if (round) frontier_write(a.fc, run + before, incl, nit, a.n_vertices + (uint32_t)g, lane);
        run += round;
    }
}

}  // namespace

uint32_t tile_count(uint32_t n_own, uint64_t n_edges, uint32_t tile_items) {
    const uint64_t items = (uint64_t)n_own * kVertexCost + n_edges;
    return (uint32_t)((items + tile_items - 1) / tile_items);
}

cudaError_t launch_build_tiles(const uint32_t* col_ptr, uint32_t n_own, uint32_t n_edges,
                               uint32_t tile_items, uint32_t hub_items, uint32_t part,
                               uint32_t tile_base, uint32_t nt, Tile* tiles, uint64_t* cuts,
                               cudaStream_t s) {
    if (nt == 0) return cudaSuccess;
    k_cuts<<<(nt + 1 + 255) / 256, 256, 0, s>>>(col_ptr, n_own, n_edges, tile_items, hub_items, nt, cuts);
    k_tiles<<<(nt + 255) / 256, 256, 0, s>>>(col_ptr, n_own, cuts, nt, part, tile_base, tiles);
    return cudaGetLastError();
}

cudaError_t launch_outdeg(const PartDev& p, const uint32_t* src, const uint32_t* ghost_gid,
                          uint32_t* outdeg, cudaStream_t s) {
    if (p.n_edges == 0) return cudaSuccess;
    // a few blocks per SM: each flushes its shared counters once
    const uint64_t blocks = std::min<uint64_t>((p.n_edges + 255) / 256, 152ull * 4);
    k_outdeg<<<(unsigned)blocks, 256, 0, s>>>(src, p.n_edges, p.n_own, p.v_begin, ghost_gid, outdeg);
    return cudaGetLastError();
}

cudaError_t launch_validate_csc(const uint32_t* col_ptr, uint32_t n_own, const uint32_t* src,
                                uint64_t n_edges, uint32_t n_local, uint32_t* err, cudaStream_t s) {
    const uint64_t work = std::max<uint64_t>(std::max<uint64_t>(n_edges, n_own), 1);
    const uint64_t blocks = std::min<uint64_t>((work + 255) / 256, 152ull * 16);
    k_validate<<<(unsigned)blocks, 256, 0, s>>>(col_ptr, n_own, src, n_edges, n_local, err);
    return cudaGetLastError();
}

cudaError_t launch_csc_import(const uint64_t* cp64, uint32_t n, uint64_t n_edges, uint32_t* cp32,
                              const uint32_t* src, uint32_t n_local, uint32_t* err, cudaStream_t s) {
    const uint64_t work = std::max<uint64_t>((uint64_t)n + 1, n_edges);
    const uint64_t blocks = std::min<uint64_t>((work + 255) / 256, 152ull * 16);
    k_csc_import<<<(unsigned)blocks, 256, 0, s>>>(cp64, n, n_edges, cp32, src, n_local, err);
    return cudaGetLastError();
}

cudaError_t launch_init_values(Algo a, uint32_t ppr_source, uint32_t n, uint32_t source, uint32_t* own, float* rank,
                               const uint32_t* outdeg, StepStats* st, const uint32_t* label_of, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t blocks = std::min<uint32_t>((n + 255) / 256, 152u * 8);
    k_init_values<<<blocks, 256, 0, s>>>((int)a, ppr_source, n, source, own, rank, outdeg, st, label_of);
    return cudaGetLastError();
}

cudaError_t launch_identity_slots(uint32_t* a, uint32_t* b, uint32_t* c, uint32_t v, cudaStream_t s) {
    k_identity_slots<<<1, 1, 0, s>>>(a, b, c, v);
    return cudaGetLastError();
}

cudaError_t launch_init_ghosts(Algo, uint32_t n_ghost, const uint32_t* gid, const uint32_t* own,
                               uint32_t* ghost, cudaStream_t s) {
    if (n_ghost == 0) return cudaSuccess;
    const uint32_t blocks = std::min<uint32_t>((n_ghost + 255) / 256, 152u * 8);
    k_init_ghosts<<<blocks, 256, 0, s>>>(n_ghost, gid, own, ghost);
    return cudaGetLastError();
}

cudaError_t launch_sync(const SyncArgs& a, uint32_t, cudaStream_t s) {
    if (a.n_parts == 0 || a.blocks_x == 0) return cudaSuccess;
    dim3 grid(a.blocks_x, a.n_parts);
    k_sync_count<<<grid, kSyncBlock, 0, s>>>(a);
    k_sync_write<<<grid, kSyncBlock, 0, s>>>(a);
    if (a.n_pull)
        k_sync_pull<<<std::min<uint32_t>((a.n_pull + 255) / 256, 152u * 16), 256, 0, s>>>(a);
    return cudaGetLastError();
}


}  // namespace gxp
