// Host-called kernels of the push direction: the out-edge copy of the graph
// (sources' out-edges grouped by source, renumbered like the pull layout)
// and the seeding of a frontier list. The push superstep itself runs inside
// the superstep kernel (frontier.cuh, sell.cu).
#include "frontier.cuh"

#include <algorithm>

namespace gxp {
namespace {

// out-edge copy: one warp per (renumbered) row, each in-edge (u -> row)
// placed at its source's next free slot
__global__ void __launch_bounds__(256) k_out_fill(const RowSource in, uint32_t n, uint32_t* cursor,
                                                  uint32_t* out_dst, uint32_t* out_w) {
    const int lane = threadIdx.x & 31;
    const uint64_t w0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t r = w0; r < n; r += nw) {
        const uint32_t old = in.row_map ? in.row_map[r] : (uint32_t)r;
        const uint32_t e0 = in.col_ptr[old], e1 = in.col_ptr[old + 1];
        for (uint32_t e = e0 + (uint32_t)lane; e < e1; e += 32u) {
            const uint32_t s0 = in.src[e];
            const uint32_t u = in.src_map ? in.src_map[s0] : s0;
            const uint32_t pos = atomicAdd(cursor + u, 1u);
            out_dst[pos] = (uint32_t)r;
            if (out_w) out_w[pos] = in.w[e];
        }
    }
}

// items of one vertex, or of all vertices (source == kInf)
__global__ void __launch_bounds__(256) k_seed_frontier(uint32_t n, uint32_t source, const uint32_t* out_ptr,
                                                       const FrontierCfg f, StepStats* st) {
    const int lane = threadIdx.x & 31;
    if (source != kInf) {
        if (blockIdx.x == 0 && threadIdx.x < 32) {
            const uint32_t deg = out_ptr[source + 1] - out_ptr[source];
            frontier_append(lane == 0, source, deg, f, st, lane);
        }
        return;
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t b = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); b < n; b += stride) {
        const uint64_t v = b + (uint64_t)lane;
        const bool has = v < n;
        const uint32_t deg = has ? out_ptr[v + 1] - out_ptr[v] : 0u;
        frontier_append(has, (uint32_t)v, deg, f, st, lane);
    }
}

}  // namespace

size_t out_edges_scratch_words(uint32_t n) { return (size_t)n + 1 + ((size_t)n + 2047) / 2048 + 1; }

cudaError_t launch_out_edges(const RowSource& in, uint32_t n, const uint32_t* outdeg, uint32_t* out_ptr,
                             uint32_t* cursor, uint32_t* scan_scratch, uint32_t* out_dst, uint32_t* out_w,
                             cudaStream_t s) {
    cudaError_t e = launch_exclusive_scan_u32(outdeg, n, out_ptr, scan_scratch, s);
    if (e != cudaSuccess || n == 0) return e;
    e = cudaMemcpyAsync(cursor, out_ptr, 4ull * n, cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) return e;
    const uint64_t blocks = ((uint64_t)n * 32 + 255) / 256;
    k_out_fill<<<(uint32_t)std::min<uint64_t>(blocks, 152ull * 64), 256, 0, s>>>(in, n, cursor, out_dst, out_w);
    return cudaGetLastError();
}

cudaError_t launch_seed_frontier(uint32_t n, uint32_t source, const uint32_t* out_ptr, const FrontierCfg& f,
                                 StepStats* stats, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(&stats->list_ne, 0, sizeof(unsigned long long), s);
    if (e != cudaSuccess || n == 0) return e;
    const uint32_t grid = source != kInf ? 1u : (uint32_t)std::min<uint64_t>(((uint64_t)n + 255) / 256, 152ull * 16);
    k_seed_frontier<<<grid, 256, 0, s>>>(n, source, out_ptr, f, stats);
    return cudaGetLastError();
}

}  // namespace gxp
