// Host-called kernels of the push direction: the out-edge copy of the graph
// (sources' out-edges grouped by source, renumbered like the pull layout)
// and the seeding of a frontier list. The push superstep itself runs inside
// the superstep kernel (frontier.cuh, sell.cu).
#include "frontier.cuh"

#include <algorithm>

namespace gxp {
namespace {

// The out-edge fill takes each edge's slot with an atomic on its source's
// cursor. Atomics on one 128-byte line serialize in L2 (tens of ns each),
// and the sources renumbered first have the most out-edges (in- and
// out-degrees go together in the power-law graphs served here: the hottest
// R-MAT 22 source has ~160K). So:
//  * each of the first kHot sources has kSub sub-ranges, one per destination
//    class r mod kSub, sized by a counting pass; every (source, class)
//    cursor has a line of its own;
//  * the next sources up to kWarm have one cursor on a line of its own;
//  * the rest are packed.
constexpr uint32_t kHot = 4096;
constexpr uint32_t kSub = 64;
constexpr uint32_t kWarm = 65536;
constexpr uint32_t kLine = 32;   // words per 128-byte line

struct Cursors {
    uint32_t* hot;    // [kHot * kSub] lines
    uint32_t* warm;   // [kWarm - kHot] lines
    uint32_t* cold;   // [n - kWarm]

    __device__ __forceinline__ uint32_t* of(uint32_t u, uint32_t r) const {
        if (u < kHot) return hot + ((uint64_t)u * kSub + (r % kSub)) * kLine;
        if (u < kWarm) return warm + (uint64_t)(u - kHot) * kLine;
        return cold + (u - kWarm);
    }
};

static size_t cursor_words(uint32_t n) {
    return (size_t)kHot * kSub * kLine + (size_t)(kWarm - kHot) * kLine + (n > kWarm ? (size_t)(n - kWarm) : 0u);
}

// The two passes (count, fill) walk the CSC in its input row order: a warp
// takes 32 consecutive rows and walks their edges flattened 32 at a time
// (coalesced loads, each lane finding its row by binary search over the
// warp's scan of the row lengths). Rows of more than kHeavyEdges in-edges are
// left out of that walk and cut into chunks of kHeavyEdges, which the count
// pass lists and separate warps walk (a single warp on a hub row would hold
// the whole pass up).
constexpr uint32_t kHeavyEdges = 2048;

// Per lane, kEdgeUnroll edges are in flight at once: their source loads,
// then their renumbering loads, then their atomics are issued together
// before any result is used (one such chain per edge would leave the walk
// bound by memory latency).
constexpr int kEdgeUnroll = 4;

template <bool kFill>
struct EdgeOp {
    const RowSource in;
    Cursors cur;
    uint32_t* out_dst;
    uint32_t* out_w;

    // edges e[q] (input CSC indices) into renumbered rows r[q], for the lanes
    // with has[q]; called by all 32 lanes
    __device__ __forceinline__ void operator()(const bool (&has)[kEdgeUnroll], const uint32_t (&e)[kEdgeUnroll],
                                               const uint32_t (&r)[kEdgeUnroll], int lane) const {
        uint32_t u[kEdgeUnroll], w[kEdgeUnroll];
#pragma unroll
        for (int q = 0; q < kEdgeUnroll; ++q) {
            u[q] = has[q] ? in.src[e[q]] : 0u;
            w[q] = (kFill && out_w && has[q]) ? in.w[e[q]] : 0u;
        }
        if (in.src_map) {
#pragma unroll
            for (int q = 0; q < kEdgeUnroll; ++q) u[q] = has[q] ? in.src_map[u[q]] : 0u;
        }
        uint32_t* c[kEdgeUnroll];
        unsigned grp[kEdgeUnroll];
        uint32_t base[kEdgeUnroll];
#pragma unroll
        for (int q = 0; q < kEdgeUnroll; ++q) {
            const bool want = has[q] && (kFill || u[q] < kHot);   // the count pass counts hot sources only
            const unsigned act = __ballot_sync(0xFFFFFFFFu, want);
            c[q] = cur.of(u[q], r[q]);
            grp[q] = 0u;
            base[q] = 0u;
            if (want) {
                grp[q] = __match_any_sync(act, (unsigned long long)(uintptr_t)c[q]);
                if (lane == __ffs(grp[q]) - 1) base[q] = atomicAdd(c[q], (uint32_t)__popc(grp[q]));
            }
        }
        if (!kFill) return;
#pragma unroll
        for (int q = 0; q < kEdgeUnroll; ++q) {
            if (!has[q]) continue;
            const uint32_t b = __shfl_sync(grp[q], base[q], __ffs(grp[q]) - 1);
            const uint32_t pos = b + (uint32_t)__popc(grp[q] & ((1u << lane) - 1u));
            out_dst[pos] = r[q];
            if (out_w) out_w[pos] = w[q];
        }
    }
};

// light rows; the count pass also lists the heavy rows' chunks {row, chunk}
template <bool kFill>
__global__ void __launch_bounds__(256) k_edges_light(const EdgeOp<kFill> op, uint32_t n, uint2* heavy,
                                                     uint32_t* n_heavy) {
    const int lane = threadIdx.x & 31;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const RowSource& in = op.in;
    for (uint64_t r0 = w0 * 32u; r0 < n; r0 += nw * 32u) {
        const uint64_t ro = r0 + (uint64_t)lane;   // input row of this lane
        uint32_t beg = 0, len = 0, rn = 0;
        if (ro < n) {
            beg = in.col_ptr[ro];
            len = in.col_ptr[ro + 1] - beg;
            rn = in.src_map ? in.src_map[ro] : (uint32_t)ro;   // its renumbered id
        }
        const bool heavy_row = len > kHeavyEdges;
        if (!kFill) {   // list the heavy row's chunks
            const uint32_t nc = heavy_row ? (len + kHeavyEdges - 1) / kHeavyEdges : 0u;
            const uint32_t incl = warp_inclusive_scan(nc, lane);
            const uint32_t tot = __shfl_sync(0xFFFFFFFFu, incl, 31);
            uint32_t base = 0;
            if (tot && lane == 0) base = atomicAdd(n_heavy, tot);
            base = __shfl_sync(0xFFFFFFFFu, base, 0);
            for (uint32_t c = 0; c < nc; ++c) heavy[base + incl - nc + c] = make_uint2((uint32_t)ro, c);
        }
        if (heavy_row) len = 0;
        const uint32_t incl = warp_inclusive_scan(len, lane);
        const uint32_t excl = incl - len;
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        for (uint32_t k0 = 0; k0 < total; k0 += 32u * kEdgeUnroll) {
            bool has[kEdgeUnroll];
            uint32_t e[kEdgeUnroll], r[kEdgeUnroll];
#pragma unroll
            for (int q = 0; q < kEdgeUnroll; ++q) {
                const uint32_t k = k0 + 32u * q + (uint32_t)lane;
                const int j = warp_owner(incl, k);
                e[q] = __shfl_sync(0xFFFFFFFFu, beg, j) + (k - __shfl_sync(0xFFFFFFFFu, excl, j));
                r[q] = __shfl_sync(0xFFFFFFFFu, rn, j);
                has[q] = k < total;
            }
            op(has, e, r, lane);
        }
    }
}

// heavy rows' chunks, one warp each
template <bool kFill>
__global__ void __launch_bounds__(256) k_edges_heavy(const EdgeOp<kFill> op, const uint2* heavy,
                                                     const uint32_t* n_heavy) {
    const int lane = threadIdx.x & 31;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t nh = *n_heavy;
    const RowSource& in = op.in;
    for (uint64_t i = w0; i < nh; i += nw) {
        const uint2 h = heavy[i];
        const uint32_t e0 = in.col_ptr[h.x] + h.y * kHeavyEdges;
        const uint32_t e1 = min(in.col_ptr[h.x + 1], e0 + kHeavyEdges);
        const uint32_t rn = in.src_map ? in.src_map[h.x] : h.x;
        for (uint32_t eb = e0; eb < e1; eb += 32u * kEdgeUnroll) {
            bool has[kEdgeUnroll];
            uint32_t e[kEdgeUnroll], r[kEdgeUnroll];
#pragma unroll
            for (int q = 0; q < kEdgeUnroll; ++q) {
                e[q] = eb + 32u * q + (uint32_t)lane;
                has[q] = e[q] < e1;
                r[q] = rn;
            }
            op(has, e, r, lane);
        }
    }
}

// sub-range starts of the hot sources (warp per source: 2 classes a lane),
// and the cursors of the others
__global__ void __launch_bounds__(256) k_cursor_init(const uint32_t* out_ptr, uint32_t n, const Cursors cur) {
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    const uint32_t n_hot = min(n, kHot);
    for (uint64_t w = tid >> 5; w < n_hot; w += nt >> 5) {
        uint32_t* ca = cur.of((uint32_t)w, 2u * lane);
        uint32_t* cb = cur.of((uint32_t)w, 2u * lane + 1u);
        const uint32_t a = *ca, b = *cb;
        const uint32_t incl = warp_inclusive_scan(a + b, lane);
        const uint32_t base = out_ptr[w] + incl - (a + b);
        *ca = base;
        *cb = base + a;
    }
    for (uint64_t u = (uint64_t)kHot + tid; u < n; u += nt) *cur.of((uint32_t)u, 0u) = out_ptr[u];
}

// items of one vertex, or of all vertices (source == kInf). All vertices:
// CTA c takes a contiguous chunk of them, sums its items and out-edges,
// reserves its range of the list with one atomic (one per warp made the list
// counter the bottleneck: a million same-address atomics at 2^22 slots), then
// writes the items 256 vertices at a time at block-scanned offsets. Under
// GXP_DIR_AUTO a superstep whose frontier is every vertex always pulls
// ((items + edges) * push_div exceeds the edges), so only the counts are
// recorded and the items are not written.
__global__ void __launch_bounds__(256) k_seed_frontier(uint32_t n, uint32_t source, const uint32_t* out_ptr,
                                                       const FrontierCfg f, StepStats* st) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (source != kInf) {
        if (blockIdx.x == 0 && threadIdx.x < 32) {
            const uint32_t deg = out_ptr[source + 1] - out_ptr[source];
            frontier_append(lane == 0, source, deg, f, st, lane);
        }
        return;
    }
    __shared__ uint32_t s_items[8], s_edges[8];
    __shared__ unsigned long long s_base;
    const uint64_t per = ((((uint64_t)n + gridDim.x - 1) / gridDim.x) + 255) & ~255ull;
    const uint64_t lo = std::min<uint64_t>(n, (uint64_t)blockIdx.x * per), hi = std::min<uint64_t>(n, lo + per);
    if (lo >= hi) return;   // uniform over the CTA
    uint32_t items = 0, edges = 0;
    for (uint64_t v = lo + threadIdx.x; v < hi; v += blockDim.x) {
        const uint32_t deg = out_ptr[v + 1] - out_ptr[v];
        items += frontier_items(deg);
        edges += deg;
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
        s_base = atomicAdd(&st->list_ne, list_pack(ti, te)) >> 32;
    }
    __syncthreads();
    if (f.direction != GXP_DIR_PUSH) return;   // the first superstep pulls: its list is never read
    unsigned long long run = s_base;
    for (uint64_t r0 = lo; r0 < hi; r0 += blockDim.x) {
        const uint64_t v = r0 + threadIdx.x;
        const bool has = v < hi;
        const uint32_t nit = has ? frontier_items(out_ptr[v + 1] - out_ptr[v]) : 0u;
        const uint32_t incl = warp_inclusive_scan(nit, lane);
        __syncthreads();   // the previous round's totals are read
        if (lane == 31) s_items[warp] = incl;
        __syncthreads();
        uint32_t before = 0, round = 0;
        for (int w = 0; w < 8; ++w) {
            if (w < warp) before += s_items[w];
            round += s_items[w];
        }
        frontier_write(f, run + before, incl, nit, (uint32_t)v, lane);
        run += round;
    }
}

// one partition's rows and edges into the CSC over global rows with slot sources
__global__ void __launch_bounds__(256) k_unify_csc(const PartDev p, uint32_t V, uint64_t edge_base, uint32_t* ucol,
                                                   uint32_t* usrc, bool last) {
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x, nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = t0; r < p.n_own + (last ? 1u : 0u); r += nt)
        ucol[p.v_begin + r] = (uint32_t)(edge_base + p.col_ptr[r]);
    const uint32_t copy0 = V + p.ghost_base;
    for (uint64_t e = t0; e < p.n_edges; e += nt) {
        const uint32_t u = p.src[e];
        usrc[edge_base + e] = u < p.n_own ? p.v_begin + u : copy0 + (u - p.n_own);
    }
}

// out-degree of every slot; lanes with equal slots add once
__global__ void __launch_bounds__(256) k_slot_degrees(const uint32_t* usrc, uint64_t n_edges, uint32_t* outdeg) {
    const int lane = threadIdx.x & 31;
    const uint64_t nt = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < n_edges; b += nt) {
        const uint64_t e = b + (uint64_t)lane;
        const bool has = e < n_edges;
        const uint32_t u = has ? usrc[e] : 0u;
        const unsigned act = __ballot_sync(0xFFFFFFFFu, has);
        if (has) {
            const unsigned grp = __match_any_sync(act, u);
            if (lane == __ffs(grp) - 1) atomicAdd(outdeg + u, (uint32_t)__popc(grp));
        }
    }
}

// every slot (vertices, then cached copies) whose value is below INF
__global__ void __launch_bounds__(256) k_seed_finite(uint32_t V, uint32_t n_ghost, const uint32_t* own,
                                                     const uint32_t* ghost, const uint32_t* out_ptr,
                                                     const FrontierCfg f, StepStats* st) {
    const int lane = threadIdx.x & 31;
    const uint64_t n = (uint64_t)V + n_ghost;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
        const uint64_t u = b + (uint64_t)lane;
        bool has = false;
        uint32_t deg = 0;
        if (u < n) {
            const uint32_t x = u < V ? own[u] : ghost[u - V];
            has = x != kInf;
            deg = has ? out_ptr[u + 1] - out_ptr[u] : 0u;
        }
        frontier_append(has, (uint32_t)u, deg, f, st, lane);
    }
}

}  // namespace

cudaError_t launch_unify_csc(const PartDev& p, uint32_t n_vertices, uint64_t edge_base, uint32_t* ucol,
                             uint32_t* usrc, bool last, cudaStream_t s) {
    const uint64_t work = std::max<uint64_t>((uint64_t)p.n_own + 1, p.n_edges);
    const uint32_t g = (uint32_t)std::min<uint64_t>((work + 255) / 256, 152ull * 16);
    k_unify_csc<<<g, 256, 0, s>>>(p, n_vertices, edge_base, ucol, usrc, last);
    return cudaGetLastError();
}

cudaError_t launch_slot_degrees(const uint32_t* usrc, uint64_t n_edges, uint32_t n_slots, uint32_t* outdeg,
                                cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(outdeg, 0, 4ull * n_slots, s);
    if (e != cudaSuccess || n_edges == 0) return e;
    const uint32_t g = (uint32_t)std::min<uint64_t>((n_edges + 255) / 256, 152ull * 16);
    k_slot_degrees<<<g, 256, 0, s>>>(usrc, n_edges, outdeg);
    return cudaGetLastError();
}

cudaError_t launch_seed_finite(uint32_t n_vertices, uint32_t n_ghost, const uint32_t* own, const uint32_t* ghost,
                               const uint32_t* out_ptr, const FrontierCfg& f, StepStats* stats, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&stats->list_ne, 0, sizeof(unsigned long long), s);
    const uint64_t n = (uint64_t)n_vertices + n_ghost;
    if (e != cudaSuccess || n == 0) return e;
    const uint32_t grid = (uint32_t)std::min<uint64_t>((n + 255) / 256, 152ull * 16);
    k_seed_finite<<<grid, 256, 0, s>>>(n_vertices, n_ghost, own, ghost, out_ptr, f, stats);
    return cudaGetLastError();
}

// scratch words: cursors, scan sums, heavy chunk count, then the heavy
// chunks (uint2, from a 16-byte aligned word)
static size_t heavy_offset_words(uint32_t n) {
    const size_t w = cursor_words(n) + ((size_t)n + 2047) / 2048 + 1 + 1;
    return (w + 3) & ~(size_t)3;
}

size_t out_edges_scratch_words(uint32_t n_src, uint64_t n_edges) {
    const size_t heavy = 2 * (n_edges / kHeavyEdges + 1);   // chunk entries: at most 2 E / kHeavyEdges
    return heavy_offset_words(n_src) + 2 * heavy;
}

cudaError_t launch_out_edges(const RowSource& in, uint32_t n, uint32_t n_src, uint64_t n_edges,
                             const uint32_t* outdeg, uint32_t* out_ptr, uint32_t* scratch, uint32_t* out_dst,
                             uint32_t* out_w, cudaStream_t s) {
    Cursors cur;
    cur.hot = scratch;
    cur.warm = cur.hot + (size_t)kHot * kSub * kLine;
    cur.cold = cur.warm + (size_t)(kWarm - kHot) * kLine;
    uint32_t* scan = scratch + cursor_words(n_src);                  // scan scratch
    uint32_t* n_heavy = scan + ((size_t)n_src + 2047) / 2048 + 1;    // heavy chunk count
    uint2* heavy = reinterpret_cast<uint2*>(scratch + heavy_offset_words(n_src));   // heavy chunks
    cudaError_t e = launch_exclusive_scan_u32(outdeg, n_src, out_ptr, scan, s);
    if (e != cudaSuccess || n == 0) return e;
    if ((e = cudaMemsetAsync(cur.hot, 0, 4ull * kHot * kSub * kLine, s)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(n_heavy, 0, 4, s)) != cudaSuccess) return e;
    const uint32_t gl = (uint32_t)std::min<uint64_t>(((uint64_t)n + 255) / 256, 152ull * 16);
    const uint32_t gs = (uint32_t)std::min<uint64_t>(((uint64_t)n_src + 255) / 256, 152ull * 16);
    const uint32_t gh = (uint32_t)std::min<uint64_t>((n_edges / kHeavyEdges + 8) / 8 + 1, 152ull * 16);
    const EdgeOp<false> count{in, cur, nullptr, nullptr};
    k_edges_light<false><<<gl, 256, 0, s>>>(count, n, heavy, n_heavy);
    k_edges_heavy<false><<<gh, 256, 0, s>>>(count, heavy, n_heavy);
    k_cursor_init<<<gs, 256, 0, s>>>(out_ptr, n_src, cur);
    const EdgeOp<true> fill{in, cur, out_dst, out_w};
    k_edges_light<true><<<gl, 256, 0, s>>>(fill, n, heavy, n_heavy);
    k_edges_heavy<true><<<gh, 256, 0, s>>>(fill, heavy, n_heavy);
    return cudaGetLastError();
}

cudaError_t launch_seed_frontier(uint32_t n, uint32_t source, const uint32_t* out_ptr, const FrontierCfg& f,
                                 StepStats* stats, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&stats->list_ne, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    const uint32_t grid = source != kInf ? 1u : (uint32_t)std::min<uint64_t>(((uint64_t)n + 255) / 256, 152ull * 8);
    k_seed_frontier<<<grid, 256, 0, s>>>(n, source, out_ptr, f, stats);
    return cudaGetLastError();
}

}  // namespace gxp
