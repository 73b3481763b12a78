// Device-side build of the sliced-ELL layout of one partition (the edge
// blocks of Section II-B, in the form the superstep kernel reads):
//
//  1. k_sort_rows_warp / k_sort_rows_block: each row's in-edges sorted by
//     (source, weight), so the k-th sources of a slice's rows fall in
//     similar id ranges. Rows of up to 32 / 256 edges are bitonic-sorted in
//     a warp's registers, rows of up to kSortMax edges in shared memory;
//     longer (hub) rows are sorted in runs of kSortMax edges, so each run a
//     warp gathers is ordered.
//  2. k_sell_windows: per window of kSellWindow rows, a stable counting sort
//     of the rows with at most H in-edges by descending in-degree (one warp
//     per window, bins in shared memory; degrees above kExactBins share
//     power-of-two bins), and the list of hub rows (more than H in-edges).
//  3. k_sell_slices: slices of 32 consecutive sorted rows, their widths and
//     row slots; k_scan_widths: element offsets of the slices.
//  4. k_sell_fill: the column-major slice arrays (one warp per slice).
//  5. k_hub_rows / k_scan_parts / k_hub_parts: hub rows in id order, split
//     into parts of T edges.
//  6. k_order_slices: all partitions' slice descriptors stably ordered by
//     decreasing width class (heavy slices first).
#include <algorithm>

#include "gxp_internal.hpp"

namespace gxp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kSortMax = 2048;     // longest row sorted (shared-memory bitonic)
constexpr uint32_t kExactBins = 4096;   // in-degrees sorted exactly up to here
constexpr uint32_t kBins = kExactBins + 34;

__device__ __forceinline__ uint64_t umin64(uint64_t a, uint64_t b) { return a < b ? a : b; }
__device__ __forceinline__ uint64_t umax64(uint64_t a, uint64_t b) { return a < b ? b : a; }

// Bitonic sort of 32 * kSlots keys held as x[s] at index s * 32 + lane.
template <int kSlots>
__device__ __forceinline__ void warp_bitonic(uint64_t (&x)[kSlots], int lane) {
    constexpr int N = 32 * kSlots;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int s = 0; s < kSlots; ++s) {
                    const int ps = s ^ (j >> 5);
                    if (ps > s) {
                        const bool up = ((s * 32 + lane) & k) == 0;
                        const uint64_t a = x[s], b = x[ps];
                        if ((a > b) == up) {
                            x[s] = b;
                            x[ps] = a;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int s = 0; s < kSlots; ++s) {
                    const uint64_t o = __shfl_xor_sync(kFull, x[s], j);
                    const bool up = ((s * 32 + lane) & k) == 0;
                    const bool lower = (lane & j) == 0;
                    x[s] = (lower == up) ? umin64(x[s], o) : umax64(x[s], o);
                }
            }
        }
    }
}

template <int kSlots>
__device__ __forceinline__ void sort_row_in_warp(uint32_t b, uint32_t d, const uint32_t* src, const uint32_t* w,
                                                 uint32_t* ssrc, uint32_t* sw, int lane) {
    uint64_t x[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        const uint32_t i = s * 32 + lane;
        x[s] = i < d ? ((uint64_t)src[b + i] << 32) | (w ? w[b + i] : 0u) : ~0ull;
    }
    warp_bitonic<kSlots>(x, lane);
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        const uint32_t i = s * 32 + lane;
        if (i < d) {
            ssrc[b + i] = (uint32_t)(x[s] >> 32);
            if (sw) sw[b + i] = (uint32_t)x[s];
        }
    }
}

// one warp per row: sorts rows of up to 256 edges, lists the runs of
// kSortMax edges of longer rows ({row, first edge of the run}) for the block sort
__global__ void k_sort_rows_warp(const uint32_t* col_ptr, uint32_t n, const uint32_t* src, const uint32_t* w,
                                 uint32_t* ssrc, uint32_t* sw, uint2* big_runs, uint32_t* n_big) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v = warp0; v < n; v += n_warps) {
        const uint32_t b = col_ptr[v], d = col_ptr[v + 1] - b;
        if (d <= 32) {
            sort_row_in_warp<1>(b, d, src, w, ssrc, sw, lane);
        } else if (d <= 256) {
            sort_row_in_warp<8>(b, d, src, w, ssrc, sw, lane);
        } else {
            const uint32_t runs = (d + kSortMax - 1) / kSortMax;
            uint32_t at = 0;
            if (lane == 0) at = atomicAdd(n_big, runs);
            at = __shfl_sync(kFull, at, 0);
            for (uint32_t r = lane; r < runs; r += 32) big_runs[at + r] = make_uint2((uint32_t)v, r * kSortMax);
        }
    }
}

// one CTA per listed run (257 .. kSortMax edges): bitonic sort in shared memory
__global__ void __launch_bounds__(256) k_sort_rows_block(const uint32_t* col_ptr, const uint32_t* src,
                                                         const uint32_t* w, uint32_t* ssrc, uint32_t* sw,
                                                         const uint2* big_runs, const uint32_t* n_big) {
    __shared__ uint64_t x[kSortMax];
    const uint32_t cnt = *n_big;
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const uint2 run = big_runs[r];
        const uint32_t b = col_ptr[run.x] + run.y;
        const uint32_t d = min(kSortMax, col_ptr[run.x + 1] - b);
        uint32_t N = 32;
        while (N < d) N <<= 1;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < N; i += blockDim.x)
            x[i] = i < d ? ((uint64_t)src[b + i] << 32) | (w ? w[b + i] : 0u) : ~0ull;
        __syncthreads();
        for (uint32_t k = 2; k <= N; k <<= 1)
            for (uint32_t j = k >> 1; j > 0; j >>= 1) {
                for (uint32_t i = threadIdx.x; i < N; i += blockDim.x) {
                    const uint32_t p = i ^ j;
                    if (p > i) {
                        const bool up = (i & k) == 0;
                        const uint64_t a = x[i], c = x[p];
                        if ((a > c) == up) {
                            x[i] = c;
                            x[p] = a;
                        }
                    }
                }
                __syncthreads();
            }
        for (uint32_t i = threadIdx.x; i < d; i += blockDim.x) {
            ssrc[b + i] = (uint32_t)(x[i] >> 32);
            if (sw) sw[b + i] = (uint32_t)x[i];
        }
    }
}

__device__ __forceinline__ uint32_t deg_bin(uint32_t d) {
    return d <= kExactBins ? d : kExactBins + (31u - (uint32_t)__clz(d));
}

// bins[k] <- number of entries in bins above k (exclusive offsets in
// descending bin order); lane l of the warp handles a chunk of bins
__device__ void descending_offsets(uint32_t* bins, int lane) {
    constexpr uint32_t kChunk = (kBins + 31) / 32;
    const int hi = (int)kBins - 1 - lane * (int)kChunk;   // this lane's bins: hi, hi-1, ...
    uint32_t sum = 0;
    for (int i = 0; i < (int)kChunk; ++i)
        if (hi - i >= 0) sum += bins[hi - i];
    uint32_t incl = sum;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += t;
    }
    uint32_t run = incl - sum;
    for (int i = 0; i < (int)kChunk; ++i)
        if (hi - i >= 0) {
            const uint32_t c = bins[hi - i];
            bins[hi - i] = run;
            run += c;
        }
    __syncwarp();
}

// one warp (one CTA) per window: stable counting sort of the non-hub rows by
// descending in-degree, hub rows in id order; window-relative outputs
__global__ void __launch_bounds__(32) k_sell_windows(const uint32_t* col_ptr, uint32_t n, uint32_t H,
                                                     uint32_t* rows_out, uint32_t* hub_out, uint32_t* nonhub_cnt,
                                                     uint32_t* hub_cnt) {
    __shared__ uint32_t bins[kBins];
    const int lane = threadIdx.x;
    const uint32_t win = blockIdx.x;
    const uint32_t w0 = win * kSellWindow;
    const uint32_t w1 = (uint32_t)min((uint64_t)w0 + kSellWindow, (uint64_t)n);
    for (uint32_t i = lane; i < kBins; i += 32) bins[i] = 0u;
    __syncwarp();
    for (uint32_t v0 = w0; v0 < w1; v0 += 32) {
        const uint32_t v = v0 + lane;
        if (v < w1) {
            const uint32_t d = col_ptr[v + 1] - col_ptr[v];
            if (d <= H) atomicAdd(&bins[deg_bin(d)], 1u);
        }
    }
    __syncwarp();
    descending_offsets(bins, lane);
    const uint32_t lt = (1u << lane) - 1u;
    uint32_t hubs = 0;
    for (uint32_t v0 = w0; v0 < w1; v0 += 32) {
        const uint32_t v = v0 + lane;
        bool ok = false, hub = false;
        uint32_t key = 0x80000000u | (uint32_t)lane;   // groups alone
        if (v < w1) {
            const uint32_t d = col_ptr[v + 1] - col_ptr[v];
            hub = d > H;
            ok = !hub;
            if (ok) key = deg_bin(d);
        }
        const uint32_t grp = __match_any_sync(kFull, key);
        const uint32_t hb = __ballot_sync(kFull, hub);
        if (ok) rows_out[w0 + bins[key] + __popc(grp & lt)] = v;
        if (hub) hub_out[w0 + hubs + __popc(hb & lt)] = v;
        __syncwarp();
        if (ok && (grp & lt) == 0u) bins[key] += __popc(grp);
        hubs += __popc(hb);
        __syncwarp();
    }
    if (lane == 0) {
        nonhub_cnt[win] = (w1 - w0) - hubs;
        hub_cnt[win] = hubs;
    }
}

// one CTA per window, a warp per slice: row slots and width (largest in-degree)
__global__ void k_sell_slices(const uint32_t* col_ptr, const uint32_t* rows_out, const uint32_t* nonhub_cnt,
                              const uint32_t* slice_base, uint32_t* perm, uint32_t* width) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t win = blockIdx.x, w0 = win * kSellWindow, cnt = nonhub_cnt[win];
    const uint32_t ns = (cnt + 31) / 32;
    for (uint32_t j = warp; j < ns; j += blockDim.x >> 5) {
        const uint32_t i = j * 32 + lane;
        const uint32_t r = i < cnt ? rows_out[w0 + i] : kSellPad;
        uint32_t d = r != kSellPad ? col_ptr[r + 1] - col_ptr[r] : 0u;
        const uint32_t s = slice_base[win] + j;
        perm[(uint64_t)s * 32 + lane] = r;
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) d = max(d, __shfl_xor_sync(kFull, d, o));
        if (lane == 0) width[s] = d;
    }
}

// single CTA: exclusive prefix of 32 * width (u64) over n slices; out[n] = total
__global__ void __launch_bounds__(1024) k_scan_widths(const uint32_t* width, uint32_t n, uint64_t* out) {
    __shared__ unsigned long long part[1024];
    const uint32_t t = threadIdx.x;
    const uint32_t per = (n + 1023) / 1024;
    const uint32_t a = min(n, t * per), b = min(n, a + per);
    unsigned long long s = 0;
    for (uint32_t i = a; i < b; ++i) s += 32ull * width[i];
    part[t] = s;
    __syncthreads();
    for (uint32_t o = 1; o < 1024; o <<= 1) {
        const unsigned long long x = t >= o ? part[t - o] : 0ull;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    unsigned long long run = part[t] - s;
    for (uint32_t i = a; i < b; ++i) {
        out[i] = run;
        run += 32ull * width[i];
    }
    if (t == 1023) out[n] = part[1023];
}

// one warp per slice: column-major fill of sources (and weights), descriptors
__global__ void k_sell_fill(const uint32_t* col_ptr, const uint32_t* ssrc, const uint32_t* sw, const uint32_t* perm,
                            const uint32_t* width, const uint64_t* off, uint32_t n_slices, uint32_t part,
                            uint32_t* sell_src, uint32_t* sell_w, SellSlice* desc) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t s = warp0; s < n_slices; s += n_warps) {
        const uint32_t r = perm[s * 32 + lane];
        const uint32_t wd = width[s];
        const uint64_t o = off[s];
        const uint32_t b = r != kSellPad ? col_ptr[r] : 0u;
        const uint32_t d = r != kSellPad ? col_ptr[r + 1] - b : 0u;
        for (uint32_t k = 0; k < wd; ++k) {
            const bool has = k < d;
            sell_src[o + 32ull * k + lane] = has ? ssrc[b + k] : kSellPad;
            if (sell_w) sell_w[o + 32ull * k + lane] = has ? sw[b + k] : 0u;
        }
        if (lane == 0) desc[s] = SellSlice{part, (uint32_t)(s * 32), wd, 0u, o};
    }
}

// one warp per window: hub rows into one list in id order
__global__ void k_hub_rows(const uint32_t* hub_out, const uint32_t* hub_cnt, const uint32_t* hub_base,
                           uint32_t* hub_list) {
    const uint32_t win = blockIdx.x, w0 = win * kSellWindow, cnt = hub_cnt[win], base = hub_base[win];
    for (uint32_t i = threadIdx.x; i < cnt; i += blockDim.x) hub_list[base + i] = hub_out[w0 + i];
}

// single CTA: exclusive prefix of the parts of each hub row; out[n] = total
__global__ void __launch_bounds__(1024) k_scan_parts(const uint32_t* col_ptr, const uint32_t* hub_list, uint32_t n,
                                                     uint32_t T, uint32_t* out) {
    __shared__ uint32_t part[1024];
    const uint32_t t = threadIdx.x;
    const uint32_t per = (n + 1023) / 1024;
    const uint32_t a = min(n, t * per), b = min(n, a + per);
    auto parts = [&](uint32_t h) {
        const uint32_t v = hub_list[h];
        const uint32_t d = col_ptr[v + 1] - col_ptr[v];
        return (d + T - 1) / T;
    };
    uint32_t s = 0;
    for (uint32_t i = a; i < b; ++i) s += parts(i);
    part[t] = s;
    __syncthreads();
    for (uint32_t o = 1; o < 1024; o <<= 1) {
        const uint32_t x = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += x;
        __syncthreads();
    }
    uint32_t run = part[t] - s;
    for (uint32_t i = a; i < b; ++i) {
        out[i] = run;
        run += parts(i);
    }
    if (t == 1023) out[n] = part[1023];
}

__global__ void k_hub_parts(const uint32_t* col_ptr, const uint32_t* hub_list, const uint32_t* part_off, uint32_t n,
                            uint32_t T, uint32_t part, uint32_t part_base, HubPart* hubs) {
    for (uint32_t h = blockIdx.x * blockDim.x + threadIdx.x; h < n; h += gridDim.x * blockDim.x) {
        const uint32_t v = hub_list[h];
        const uint32_t b = col_ptr[v], d = col_ptr[v + 1] - b;
        const uint32_t np = (d + T - 1) / T, local = part_off[h], t0 = part_base + local;
        for (uint32_t k = 0; k < np; ++k)   // this partition's array; t0 indexes all partitions' parts
            hubs[local + k] = HubPart{v, part, b + k * T, min(T, d - k * T), t0, np, {0u, 0u}};
    }
}

// one warp: stable order of all slice descriptors by decreasing width (exact
// up to kExactBins, by power-of-two class above)
__global__ void __launch_bounds__(32) k_order_slices(const SellSlice* in, uint32_t n, SellSlice* out) {
    __shared__ uint32_t bins[kBins];
    const int lane = threadIdx.x;
    for (uint32_t i = lane; i < kBins; i += 32) bins[i] = 0u;
    __syncwarp();
    for (uint32_t i = lane; i < n; i += 32) atomicAdd(&bins[deg_bin(in[i].width)], 1u);
    __syncwarp();
    descending_offsets(bins, lane);
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t i0 = 0; i0 < n; i0 += 32) {
        const uint32_t i = i0 + lane;
        const bool ok = i < n;
        const uint32_t key = ok ? deg_bin(in[i].width) : 0x80000000u | (uint32_t)lane;
        const uint32_t grp = __match_any_sync(kFull, key);
        if (ok) out[bins[key] + __popc(grp & lt)] = in[i];
        __syncwarp();
        if (ok && (grp & lt) == 0u) bins[key] += __popc(grp);
        __syncwarp();
    }
}

uint32_t grid_warps(uint64_t warps, uint32_t block) {
    const uint64_t b = (warps * 32 + block - 1) / block;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 64));
}

}  // namespace

cudaError_t launch_sort_rows(const uint32_t* col_ptr, uint32_t n, const uint32_t* src, const uint32_t* w,
                             uint32_t* ssrc, uint32_t* sw, uint2* scratch_runs, uint32_t* scratch_cnt,
                             cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(scratch_cnt, 0, 4, s);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    k_sort_rows_warp<<<grid_warps(n, 256), 256, 0, s>>>(col_ptr, n, src, w, ssrc, sw, scratch_runs, scratch_cnt);
    k_sort_rows_block<<<152 * 4, 256, 0, s>>>(col_ptr, src, w, ssrc, sw, scratch_runs, scratch_cnt);
    return cudaGetLastError();
}

cudaError_t launch_sell_windows(const uint32_t* col_ptr, uint32_t n, uint32_t H, uint32_t* rows_out,
                                uint32_t* hub_out, uint32_t* nonhub_cnt, uint32_t* hub_cnt, cudaStream_t s) {
    const uint32_t nw = (n + kSellWindow - 1) / kSellWindow;
    if (nw == 0) return cudaSuccess;
    k_sell_windows<<<nw, 32, 0, s>>>(col_ptr, n, H, rows_out, hub_out, nonhub_cnt, hub_cnt);
    return cudaGetLastError();
}

cudaError_t launch_sell_slices(const uint32_t* col_ptr, uint32_t n, const uint32_t* rows_out,
                               const uint32_t* nonhub_cnt, const uint32_t* slice_base, uint32_t* perm,
                               uint32_t* width, uint64_t* off, uint32_t n_slices, cudaStream_t s) {
    const uint32_t nw = (n + kSellWindow - 1) / kSellWindow;
    if (nw) k_sell_slices<<<nw, 256, 0, s>>>(col_ptr, rows_out, nonhub_cnt, slice_base, perm, width);
    k_scan_widths<<<1, 1024, 0, s>>>(width, n_slices, off);
    return cudaGetLastError();
}

cudaError_t launch_sell_fill(const uint32_t* col_ptr, const uint32_t* ssrc, const uint32_t* sw, const uint32_t* perm,
                             const uint32_t* width, const uint64_t* off, uint32_t n_slices, uint32_t part,
                             uint32_t* sell_src, uint32_t* sell_w, SellSlice* desc, cudaStream_t s) {
    if (n_slices == 0) return cudaSuccess;
    k_sell_fill<<<grid_warps(n_slices, 256), 256, 0, s>>>(col_ptr, ssrc, sw, perm, width, off, n_slices, part,
                                                          sell_src, sell_w, desc);
    return cudaGetLastError();
}

cudaError_t launch_hub_rows(const uint32_t* col_ptr, uint32_t n, const uint32_t* hub_out, const uint32_t* hub_cnt,
                            const uint32_t* hub_base, uint32_t* hub_list, uint32_t n_hub_rows, uint32_t T,
                            uint32_t* part_off, cudaStream_t s) {
    const uint32_t nw = (n + kSellWindow - 1) / kSellWindow;
    if (nw) k_hub_rows<<<nw, 256, 0, s>>>(hub_out, hub_cnt, hub_base, hub_list);
    k_scan_parts<<<1, 1024, 0, s>>>(col_ptr, hub_list, n_hub_rows, T, part_off);
    return cudaGetLastError();
}

cudaError_t launch_hub_parts(const uint32_t* col_ptr, const uint32_t* hub_list, const uint32_t* part_off,
                             uint32_t n_hub_rows, uint32_t T, uint32_t part, uint32_t part_base, HubPart* hubs,
                             cudaStream_t s) {
    if (n_hub_rows == 0) return cudaSuccess;
    k_hub_parts<<<(n_hub_rows + 255) / 256, 256, 0, s>>>(col_ptr, hub_list, part_off, n_hub_rows, T, part, part_base,
                                                         hubs);
    return cudaGetLastError();
}

cudaError_t launch_order_slices(const SellSlice* in, uint32_t n, SellSlice* out, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    k_order_slices<<<1, 32, 0, s>>>(in, n, out);
    return cudaGetLastError();
}

}  // namespace gxp
