// Batched multi-source SSSP superstep: up to 64 Bellman-Ford instances (one
// per source, Section V-A's multi-source SSSP-BF) advance together in one
// pass over the edges, so every edge block read from memory (or streamed by
// the pipeline shuffle of Section III-A) serves all sources.
//
// Layout: dist[v][64] uint32 (one 256-byte row per vertex); an edge is a
// (source, weight) uint2 in destination order, or one uint32 (weight << 24 |
// source) when sources and weights fit, halving the bytes every superstep
// reads (and streams). Work unit = up to
// kUnitEdges in-edges of one destination; a warp owns a unit and each lane
// two source slots:
//   MSGGen   the warp reads 32 in-edges at once (one per lane, coalesced)
//            and tests each source against the frontier (changed in the
//            previous superstep); for the active ones only, taken from the
//            ballot mask and broadcast by shuffle, it reads u's 256-byte row
//            (coalesced, 8 rows in flight) and adds w, saturating below INF.
//            A unit with no active in-edge ends there (no row traffic);
//   MSGMerge per-slot minimum in registers;
//   MSGApply new = min(old, merged) is stored in place (rows split over
//            several units use atomicMin), and a destination with any
//            improved slot sets its frontier bit for the next superstep.
// Slots in idle_mask (no query) are skipped. In-place updates only ever
// lower distances, so the fixed point equals the per-source Bellman-Ford
// result; superstep counts may be below Jacobi's.
#include <algorithm>

#include "grid_sync.cuh"
#include "gxp_internal.hpp"

namespace gxp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kMsBlock = 256;
constexpr int kRowsInFlight = 8;   // source rows gathered at once per warp

__device__ __forceinline__ uint32_t sat_add(uint32_t d, uint32_t w) {
    if (d == kInf) return kInf;
    uint32_t s = d + w;
    if (s < d || s == kInf) s = kInf - 1u;
    return s;
}

template <bool kPacked>
__device__ __forceinline__ uint2 load_edge(const void* base, uint64_t i) {
    if (kPacked) {
        const uint32_t p = __ldg(static_cast<const uint32_t*>(base) + i);
        return make_uint2(p & ((1u << kPackSrcBits) - 1u), p >> kPackSrcBits);
    }
    return __ldg(static_cast<const uint2*>(base) + i);
}

// One block's share of a superstep (the units u_begin + warp, + n_warps, ...
// of the grid). kLoop: called by the persistent loop, which reads frontier
// bits written earlier in the same launch, so through coherent loads.
template <bool kDry, bool kPacked, bool kLoop>
__device__ __forceinline__ void msssp_block(const MsArgs& a) {
    __shared__ uint32_t s_imp[2], s_done;
    __shared__ unsigned long long s_changed, s_active;
    const int lane = threadIdx.x & 31;
    if (threadIdx.x < 2) s_imp[threadIdx.x] = 0u;
    if (threadIdx.x == 0) {
        s_changed = 0ull;
        s_active = 0ull;
        s_done = 0u;
    }
    __syncthreads();
    const bool live = ((~a.idle_mask >> (2 * lane)) & 3ull) != 0ull;   // either of my 2 slots busy
    uint32_t imp_lo = 0u, imp_hi = 0u;   // improved slots 0..31 / 32..63 (bit = slot)
    const uint32_t warp0 = (blockIdx.x * kMsBlock + threadIdx.x) >> 5;
    const uint32_t n_warps = (gridDim.x * kMsBlock) >> 5;
    uint32_t changed_units = 0;
    unsigned long long n_active = 0;   // active in-edges this warp walked (the same in every lane)
    for (uint64_t k = a.u_begin + warp0; k < a.u_end; k += n_warps) {
        const uint4 un = a.units[k];   // v, first edge (global), edges, split flag
        const uint32_t v = un.x, len = un.z;
        const uint64_t e = un.y - a.edge_base;   // first edge of the unit in this block
        uint2 acc = make_uint2(kInf, kInf);
        bool any = false;
        for (uint32_t base = 0; base < len; base += 32u) {
            // 32 edges at once, one per lane (coalesced), each tested against the frontier
            uint2 my = make_uint2(0u, 0u);
            bool act = false;
            if (base + lane < len) {
                my = load_edge<kPacked>(a.edges, e + base + lane);
                const uint32_t fw = kLoop ? __ldca(a.frontier_cur + (my.x >> 5)) : __ldg(a.frontier_cur + (my.x >> 5));
                act = (fw >> (my.x & 31u)) & 1u;
            }
            uint32_t mask = __ballot_sync(kFull, act);
            any |= mask != 0u;
            n_active += (unsigned)__popc(mask);
            while (mask) {
                // the active edges, kRowsInFlight source rows loaded at a time
                int idx[kRowsInFlight];
#pragma unroll
                for (int q = 0; q < kRowsInFlight; ++q) {
                    idx[q] = mask ? __ffs(mask) - 1 : -1;
                    mask &= mask - 1u;
                }
                uint2 ed[kRowsInFlight], row[kRowsInFlight];
#pragma unroll
                for (int q = 0; q < kRowsInFlight; ++q) {
                    ed[q].x = __shfl_sync(kFull, my.x, idx[q] & 31);
                    ed[q].y = __shfl_sync(kFull, my.y, idx[q] & 31);
                }
#pragma unroll
                for (int q = 0; q < kRowsInFlight; ++q)
                    row[q] = (idx[q] >= 0 && live)
                                 ? reinterpret_cast<const uint2*>(a.dist)[(uint64_t)ed[q].x * 32u + lane]
                                 : make_uint2(kInf, kInf);
#pragma unroll
                for (int q = 0; q < kRowsInFlight; ++q) {
                    acc.x = min(acc.x, sat_add(row[q].x, ed[q].y));
                    acc.y = min(acc.y, sat_add(row[q].y, ed[q].y));
                }
            }
        }
        if (!any) continue;   // no in-edge from the frontier: nothing to merge or apply
        if (kDry) {
            changed_units += (acc.x == 0u && acc.y == 0u);   // keeps the loads live
            continue;
        }
        uint32_t pair = 0u;   // my 2 slots that improved
        if (live) {
            uint2* mine = reinterpret_cast<uint2*>(a.dist) + (uint64_t)v * 32u + lane;
            const uint2 old = *mine;
            pair = (acc.x < old.x ? 1u : 0u) | (acc.y < old.y ? 2u : 0u);
            if (un.w) {   // row split across units: combine with atomics
                if (pair & 1u) atomicMin(&a.dist[(uint64_t)v * 64u + 2u * lane], acc.x);
                if (pair & 2u) atomicMin(&a.dist[(uint64_t)v * 64u + 2u * lane + 1u], acc.y);
            } else if (pair) {
                *mine = make_uint2(min(old.x, acc.x), min(old.y, acc.y));
            }
        }
        const uint32_t lo = __reduce_or_sync(kFull, lane < 16 ? pair << (2 * lane) : 0u);
        const uint32_t hi = __reduce_or_sync(kFull, lane >= 16 ? pair << (2 * lane - 32) : 0u);
        if (lo | hi) {
            if (lane == 0) atomicOr(&a.frontier_next[v >> 5], 1u << (v & 31u));
            ++changed_units;
            imp_lo |= lo;
            imp_hi |= hi;
        }
    }
    // block totals in shared memory; the block's last warp to finish issues
    // one global atomic per word (no barrier: early warps leave at once)
    if (lane == 0) {
        if (changed_units) atomicAdd(&s_changed, (unsigned long long)changed_units);
        if (n_active && a.active) atomicAdd(&s_active, n_active);
        if (imp_lo) atomicOr(&s_imp[0], imp_lo);
        if (imp_hi) atomicOr(&s_imp[1], imp_hi);
        __threadfence_block();
        const bool last = atomicAdd(&s_done, 1u) == (uint32_t)(kMsBlock / 32) - 1u;
        if (last) {
            __threadfence_block();
            const unsigned long long c = atomicAdd(&s_changed, 0ull);
            if (c) atomicAdd(a.changed, c);
            if (a.active) {
                const unsigned long long na = atomicAdd(&s_active, 0ull);
                if (na) atomicAdd(a.active, na);
            }
            const uint32_t i0 = atomicOr(&s_imp[0], 0u), i1 = atomicOr(&s_imp[1], 0u);
            if (!kDry && a.slot_improved != nullptr) {
                if (i0) atomicOr(&a.slot_improved[0], i0);
                if (i1) atomicOr(&a.slot_improved[1], i1);
            }
        }
    }
}

template <bool kDry, bool kPacked>
__global__ void __launch_bounds__(kMsBlock, 4) k_msssp(const MsArgs a) {
    msssp_block<kDry, kPacked, false>(a);
}

// Persistent form of a resident batched run: one cooperative launch runs
// supersteps until one improves nothing (or max_steps). Superstep t reads
// frontier F[t % 3], sets bits in F[(t + 1) % 3] and counts its changed
// units in changed[t % 4]; meanwhile every CTA clears its share of F[(t + 2)
// % 3], which superstep t - 1 read and superstep t + 1 writes, and block 0
// clears changed[(t + 2) % 4] (every CTA read the counter of superstep t - 2
// before it arrived at the barrier that ended superstep t - 1), so one grid
// barrier per superstep orders everything. The distances are updated in
// place, as in the launch-per-superstep form.
template <bool kPacked>
__global__ void __launch_bounds__(kMsBlock, 4)
    k_msssp_loop(MsArgs a, uint32_t* f0, uint32_t* f1, uint32_t* f2, unsigned long long* changed, uint64_t words,
                 uint32_t max_steps, GridBar* bar, uint64_t timeout_ns, uint32_t force, uint32_t* err,
                 uint32_t* steps_out) {
    uint32_t* const F[3] = {f0, f1, f2};
    __shared__ uint32_t s_more;
    for (uint32_t t = 0; t < max_steps; ++t) {
        a.frontier_cur = F[t % 3];
        a.frontier_next = F[(t + 1) % 3];
        a.changed = changed + t % 4;
        uint32_t* const clear = F[(t + 2) % 3];
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
            clear[i] = 0u;
        if (blockIdx.x == 0 && threadIdx.x == 0) changed[(t + 2) % 4] = 0ull;
        msssp_block<false, kPacked, true>(a);
        if (!grid_barrier(bar, gridDim.x, timeout_ns, force != 0u, err)) return;
        if (threadIdx.x == 0) s_more = __ldcg(changed + t % 4) != 0ull ? 1u : 0u;
        __syncthreads();
        if (!s_more || t + 1 == max_steps) {
            if (blockIdx.x == 0 && threadIdx.x == 0) *steps_out = t + 1;
            return;
        }
    }
}

__global__ void k_msssp_init(uint32_t* dist, uint64_t n_vertices) {
    const uint64_t total = n_vertices * 64u;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += (uint64_t)gridDim.x * blockDim.x)
        dist[i] = kInf;
}

// slot s of vertex sources[s] starts at 0 and the source is on the frontier
__global__ void k_msssp_sources(uint32_t* dist, const uint32_t* sources, uint32_t n_sources, uint32_t* frontier) {
    for (uint32_t s = threadIdx.x; s < n_sources; s += blockDim.x) {
        dist[(uint64_t)sources[s] * 64u + s] = 0u;
        atomicOr(&frontier[sources[s] >> 5], 1u << (sources[s] & 31u));
    }
}

__global__ void k_popc(const uint32_t* bits, uint64_t words, unsigned long long* out) {
    unsigned long long c = 0;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words; i += (uint64_t)gridDim.x * blockDim.x)
        c += __popc(bits[i]);
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}

}  // namespace

cudaError_t launch_msssp(const MsArgs& a, bool dry, uint32_t grid, cudaStream_t s) {
    if (a.u_end <= a.u_begin) return cudaSuccess;
    if (a.packed) {
        if (dry) k_msssp<true, true><<<grid, kMsBlock, 0, s>>>(a);
        else k_msssp<false, true><<<grid, kMsBlock, 0, s>>>(a);
    } else {
        if (dry) k_msssp<true, false><<<grid, kMsBlock, 0, s>>>(a);
        else k_msssp<false, false><<<grid, kMsBlock, 0, s>>>(a);
    }
    return cudaGetLastError();
}

cudaError_t launch_msssp_init(uint32_t* dist, uint64_t n_vertices, const uint32_t* sources, uint32_t n_sources,
                              uint32_t* frontier, cudaStream_t s) {
    k_msssp_init<<<1216, 256, 0, s>>>(dist, n_vertices);
    k_msssp_sources<<<1, 64, 0, s>>>(dist, sources, n_sources, frontier);
    return cudaGetLastError();
}

cudaError_t launch_popc(const uint32_t* bits, uint64_t words, unsigned long long* out, cudaStream_t s) {
    k_popc<<<608, 256, 0, s>>>(bits, words, out);
    return cudaGetLastError();
}

cudaError_t launch_msssp_loop(const MsArgs& a, uint32_t* const frontier[3], unsigned long long* changed,
                              uint64_t words, uint32_t max_steps, GridBar* bar, uint64_t timeout_ns, bool force,
                              uint32_t* err, uint32_t* steps_out, cudaStream_t s) {
    if (a.u_end <= a.u_begin || max_steps == 0) return cudaErrorInvalidValue;
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess)
        e = a.packed ? cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_msssp_loop<true>, kMsBlock, 0)
                     : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_msssp_loop<false>, kMsBlock, 0);
    if (e != cudaSuccess) return e;
    const uint64_t resident = (uint64_t)sms * (uint64_t)per_sm;
    if (resident == 0) return cudaErrorNotSupported;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(msssp_grid(a.u_end - a.u_begin), resident);
    MsArgs args = a;
    uint32_t* f0 = frontier[0];
    uint32_t* f1 = frontier[1];
    uint32_t* f2 = frontier[2];
    uint32_t fo = force ? 1u : 0u;
    void* params[] = {&args, &f0, &f1, &f2, &changed, &words, &max_steps, &bar, &timeout_ns, &fo, &err, &steps_out};
    return a.packed ? cudaLaunchCooperativeKernel((const void*)k_msssp_loop<true>, dim3(grid), dim3(kMsBlock), params,
                                                  0, s)
                    : cudaLaunchCooperativeKernel((const void*)k_msssp_loop<false>, dim3(grid), dim3(kMsBlock), params,
                                                  0, s);
}

uint32_t msssp_grid(uint64_t units) {
    const uint64_t warps = std::max<uint64_t>(1, units);
    const uint64_t blocks = (warps + (kMsBlock / 32) - 1) / (kMsBlock / 32);
    return (uint32_t)std::min<uint64_t>(blocks, 152ull * 8);
}

}  // namespace gxp
