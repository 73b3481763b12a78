// Kernels of the query server: 64 query slots share every pass over the
// edges (continuous batching). A slot's arithmetic reads only its own column,
// in an order fixed by the edge order, so a query's result is bit-identical
// whether it runs alone or among others.
//
//  * SSSP slots use the batched Bellman-Ford superstep of msssp.cu (its
//    per-slot improvement flags tell the server when a query has converged).
//  * Personalized PageRank slots iterate
//        r_{t+1} = d * A^T D^-1 r_t + ((1 - d) + d * D_t) e_s
//    (Jacobi; D_t = rank mass on dangling vertices, returned to the source s
//    together with the teleport), with fp32 messages c = r * (1 / outdeg)
//    and exact fixed-point dangling sums per slot. Lane l of a warp holds
//    slots 2l and 2l+1; lanes whose slots are both idle skip every load and
//    store.
//      k_ppr_units   one warp per work unit (<= 256 in-edges of one vertex):
//                    sums the sources' message rows in edge order; a vertex
//                    held by one unit is applied at once, a vertex split
//                    over several units leaves one partial row per unit;
//      k_ppr_split   adds a split vertex's partials in unit order, applies.
//    Apply adds the source term, writes the next messages, and writes the
//    ranks only in a slot's last superstep (the result).
//  * Slot management: batched column initialisation and a row-tile transpose
//    that copies finished columns out as contiguous result vectors.
#include <algorithm>

#include "gxp_internal.hpp"

namespace gxp {
namespace {

constexpr int kSvBlock = 256;
constexpr int kSvWarps = kSvBlock / 32;
constexpr int kSvUnroll = 8;
constexpr int kTileRows = 64;   // rows per transpose tile

uint32_t grid_for(uint64_t items, uint64_t per_block) {
    const uint64_t b = (items + per_block - 1) / per_block;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 8));
}

}  // namespace

// Grid of a serving superstep kernel: one warp per item up to 16 waves of
// 8 blocks per SM, so each block lives a fraction of the kernel and the
// block scheduler can interleave lanes of other graphs (higher-priority
// streams) at block boundaries instead of after the whole superstep.
uint32_t serve_grid(uint64_t items) {
    const uint64_t b = (items + kSvWarps - 1) / kSvWarps;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 8 * 16));
}

namespace {

// Per-slot constants of a PPR superstep, kept in shared memory so the
// gather loop keeps its registers for rows in flight: damping, source
// (kInf for an idle slot) and (1 - d) + d * D_t, D_t from the exact
// fixed-point sum of the slot's dangling mass.
struct PprSlots {
    float2 d[32], add[32];
    uint2 src[32];
    unsigned long long dang[64];   // this block's dangling mass of r_{t+1}
    uint32_t warps_done;

    __device__ void init(const PprArgs& a) {
        const int s = threadIdx.x;
        if (s < 64) {
            const bool busy = (a.active_mask >> s) & 1ull;
            const float d_s = a.slot_damping[s];
            reinterpret_cast<float*>(d)[s] = d_s;
            reinterpret_cast<float*>(add)[s] =
                busy ? (float)((1.0 - (double)d_s) + (double)d_s * fx_to_double(a.dang_cur[s])) : 0.0f;
            reinterpret_cast<uint32_t*>(src)[s] = busy ? a.slot_source[s] : kInf;
            dang[s] = 0ull;
        }
        if (threadIdx.x == 0) warps_done = 0u;
        __syncthreads();
    }

    // MSGApply of vertex v (1 / out-degree inv, 0 if dangling) for lane l's
    // slots with merged sum: r = d * sum, plus the source term at the slot's
    // source; message r * inv; ranks only in a slot's last superstep
    __device__ void apply(const PprArgs& a, uint32_t v, float inv, float2 sum, int l) {
        const float2 dl = d[l], al = add[l];
        const uint2 sl = src[l];
        float2 r = make_float2(dl.x * sum.x, dl.y * sum.y);
        if (v == sl.x) r.x += al.x;
        if (v == sl.y) r.y += al.y;
        reinterpret_cast<float2*>(a.msg_nxt)[(uint64_t)v * 32u + l] = make_float2(r.x * inv, r.y * inv);
        if ((a.finish_mask >> (2 * l)) & 3ull) reinterpret_cast<float2*>(a.rank)[(uint64_t)v * 32u + l] = r;
        if (inv == 0.0f) {
            atomicAdd(&dang[2 * l], fx_of(r.x));
            atomicAdd(&dang[2 * l + 1], fx_of(r.y));
        }
    }

    // the block's dangling sums -> one global atomic per slot, issued by the
    // block's last warp to finish (no barrier: early warps leave at once)
    __device__ void flush(unsigned long long* out) {
        __syncwarp();
        const int lane = threadIdx.x & 31;
        uint32_t last = 0u;
        if (lane == 0) {
            __threadfence_block();
            last = atomicAdd(&warps_done, 1u) == (blockDim.x >> 5) - 1u ? 1u : 0u;
        }
        if (!__shfl_sync(0xFFFFFFFFu, last, 0)) return;
        __threadfence_block();
        for (int i = lane; i < 64; i += 32) {
            const unsigned long long v = atomicAdd(&dang[i], 0ull);
            if (v) atomicAdd(&out[i], v);
        }
    }
};

// One warp per work unit, lane l holding slots 2l and 2l+1 (idle pairs skip
// every load and store). kSvUnroll source ids are read at a time (each a
// broadcast load), then their kSvUnroll message rows (256 bytes each) are in
// flight together; the sum runs in edge order. Per-slot constants live in
// shared memory so that 32 registers suffice and 64 warps fit on an SM.
__global__ void __launch_bounds__(kSvBlock, 8) k_ppr_units(const PprArgs a) {
    __shared__ PprSlots sl;
    sl.init(a);
    const int lane = threadIdx.x & 31;
    const bool live = (a.active_mask >> (2 * lane)) & 3ull;
    const float2* msg = reinterpret_cast<const float2*>(a.msg_cur);
    const uint64_t warp0 = ((uint64_t)blockIdx.x * kSvBlock + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * kSvBlock) >> 5;
    for (uint64_t k = warp0; k < a.n_units; k += n_warps) {
        const uint4 un = a.units[k];   // dst, first edge, edges, partial + 1 | 0
        const float inv = __ldg(a.inv_outdeg + un.x);
        const uint32_t* e = a.src + un.y;
        float2 acc = make_float2(0.0f, 0.0f);
        for (uint32_t i = 0; i < un.z; i += kSvUnroll) {
            uint32_t u[kSvUnroll];
#pragma unroll
            for (int q = 0; q < kSvUnroll; ++q) u[q] = i + q < un.z ? __ldg(e + i + q) : kInf;
            float2 m[kSvUnroll];
#pragma unroll
            for (int q = 0; q < kSvUnroll; ++q)
                m[q] = (u[q] != kInf && live) ? msg[(uint64_t)u[q] * 32u + lane] : make_float2(0.0f, 0.0f);
#pragma unroll
            for (int q = 0; q < kSvUnroll; ++q)
                if (u[q] != kInf) {
                    acc.x += m[q].x;
                    acc.y += m[q].y;
                }
        }
        if (!live) continue;
        if (un.w) reinterpret_cast<float2*>(a.partial)[(uint64_t)(un.w - 1u) * 32u + lane] = acc;
        else sl.apply(a, un.x, inv, acc, lane);
    }
    sl.flush(a.dang_next);
}

// One warp per vertex split over several units: adds its partial rows in
// unit order and applies.
__global__ void __launch_bounds__(kSvBlock, 8) k_ppr_split(const PprArgs a) {
    __shared__ PprSlots sl;
    sl.init(a);
    const int lane = threadIdx.x & 31;
    const bool live = (a.active_mask >> (2 * lane)) & 3ull;
    const float2* part = reinterpret_cast<const float2*>(a.partial);
    const uint32_t warp0 = (blockIdx.x * kSvBlock + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * kSvBlock) >> 5;
    for (uint32_t r = warp0; r < a.n_split_rows && live; r += n_warps) {
        const uint2 sr = a.split_rows[r];   // {vertex, first partial}
        const uint32_t end = a.split_rows[r + 1].y;
        float2 acc = make_float2(0.0f, 0.0f);
        for (uint32_t p = sr.y; p < end; ++p) {   // unit order
            const float2 x = part[(uint64_t)p * 32u + lane];
            acc.x += x.x;
            acc.y += x.y;
        }
        sl.apply(a, sr.x, __ldg(a.inv_outdeg + sr.x), acc, lane);
    }
    sl.flush(a.dang_next);
}

// thread (v, l): slots 2l and 2l+1 of row v, where they are in `mask`:
// messages of r_0 = e_src (the ranks are written by the slot's last superstep)
__global__ void k_ppr_slots_init(float* msg_cur, const float* inv_outdeg, uint64_t n, uint64_t mask,
                                 const uint32_t* slot_source, unsigned long long* dang_cur) {
    const uint64_t total = n * 32u;
    if (blockIdx.x == 0 && threadIdx.x < 64 && ((mask >> threadIdx.x) & 1ull)) {
        const uint32_t src = slot_source[threadIdx.x];
        dang_cur[threadIdx.x] = inv_outdeg[src] == 0.0f ? fx_of(1.0f) : 0ull;
    }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = i >> 5;
        const uint32_t l = (uint32_t)(i & 31u);
        const uint32_t pair = (uint32_t)(mask >> (2u * l)) & 3u;
        if (!pair) continue;
        const float inv = __ldg(inv_outdeg + v);
#pragma unroll
        for (uint32_t b = 0; b < 2; ++b)
            if ((pair >> b) & 1u) msg_cur[v * 64u + 2u * l + b] = v == slot_source[2u * l + b] ? inv : 0.0f;
    }
}

__global__ void k_sssp_slots_init(uint32_t* dist, uint64_t n, uint64_t mask, const uint32_t* slot_source,
                                  uint32_t* frontier) {
    const uint64_t total = n * 32u;
    if (blockIdx.x == 0 && threadIdx.x < 64 && ((mask >> threadIdx.x) & 1ull)) {
        const uint32_t src = slot_source[threadIdx.x];
        atomicOr(&frontier[src >> 5], 1u << (src & 31u));
    }
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < total;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t v = i >> 5;
        const uint32_t l = (uint32_t)(i & 31u);
        const uint32_t pair = (uint32_t)(mask >> (2u * l)) & 3u;
        if (!pair) continue;
#pragma unroll
        for (uint32_t b = 0; b < 2; ++b)
            if ((pair >> b) & 1u) dist[v * 64u + 2u * l + b] = v == slot_source[2u * l + b] ? 0u : kInf;
    }
}

// 64-row tiles of mat[V][64] through shared memory: coalesced row reads,
// then one coalesced 256-byte run per listed column
__global__ void __launch_bounds__(kSvBlock) k_gather_columns(const uint32_t* mat, uint64_t n, GatherList list) {
    __shared__ uint32_t tile[kTileRows][65];
    __shared__ uint32_t s_slot[64];
    __shared__ uint32_t* s_out[64];
    if (threadIdx.x < list.n) {
        s_slot[threadIdx.x] = list.slot[threadIdx.x];
        s_out[threadIdx.x] = list.out[threadIdx.x];
    }
    const uint64_t n_tiles = (n + kTileRows - 1) / kTileRows;
    for (uint64_t t = blockIdx.x; t < n_tiles; t += gridDim.x) {
        const uint64_t v0 = t * kTileRows;
        const uint32_t rows = n - v0 < (uint64_t)kTileRows ? (uint32_t)(n - v0) : (uint32_t)kTileRows;
        __syncthreads();   // previous tile fully written out
        for (uint32_t i = threadIdx.x; i < rows * 64u; i += kSvBlock) tile[i >> 6][i & 63u] = mat[v0 * 64u + i];
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < list.n * (uint32_t)kTileRows; i += kSvBlock) {
            const uint32_t j = i / kTileRows, r = i % kTileRows;
            if (r < rows) s_out[j][v0 + r] = tile[r][s_slot[j]];
        }
    }
}

}  // namespace

cudaError_t launch_ppr_superstep(const PprArgs& a, cudaStream_t s) {
    k_ppr_units<<<serve_grid(a.n_units), kSvBlock, 0, s>>>(a);
    if (a.n_split_rows) k_ppr_split<<<serve_grid(a.n_split_rows), kSvBlock, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t launch_ppr_slots_init(float* msg_cur, const float* inv_outdeg, uint64_t n, uint64_t mask,
                                  const uint32_t* slot_source, unsigned long long* dang_cur, cudaStream_t s) {
    if (!mask) return cudaSuccess;
    k_ppr_slots_init<<<grid_for(n * 32u, kSvBlock), kSvBlock, 0, s>>>(msg_cur, inv_outdeg, n, mask, slot_source,
                                                                      dang_cur);
    return cudaGetLastError();
}

cudaError_t launch_sssp_slots_init(uint32_t* dist, uint64_t n, uint64_t mask, const uint32_t* slot_source,
                                   uint32_t* frontier, cudaStream_t s) {
    if (!mask) return cudaSuccess;
    k_sssp_slots_init<<<grid_for(n * 32u, kSvBlock), kSvBlock, 0, s>>>(dist, n, mask, slot_source, frontier);
    return cudaGetLastError();
}

cudaError_t launch_gather_columns(const uint32_t* mat, uint64_t n, const GatherList& list, cudaStream_t s) {
    if (list.n == 0 || n == 0) return cudaSuccess;
    k_gather_columns<<<grid_for((n + kTileRows - 1) / kTileRows, 1), kSvBlock, 0, s>>>(mat, n, list);
    return cudaGetLastError();
}

}  // namespace gxp
