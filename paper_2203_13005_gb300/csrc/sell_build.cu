// Device-side build of the sliced-ELL layout of one partition (the edge
// blocks of Section II-B, in the form the superstep kernel reads):
//
//  1. k_sort_rows_warp / k_sort_rows_block: each row's in-edges sorted by
//     source, so the k-th sources of a slice's rows fall in similar id
//     ranges. Rows of up to 32 / 256 edges are bitonic-sorted in a warp's
//     registers (by (source, weight)), rows of up to kSortMax edges
//     radix-sorted in shared memory (stably by source); longer (hub) rows
//     are sorted in runs of kSortMax edges, so each run a warp gathers is
//     ordered.
//  2. k_sell_windows: per window of kSellWindow rows, a stable counting sort
//     of the rows with at most H in-edges by descending in-degree (one CTA
//     per window, per-warp bins in shared memory; degrees above kExactBins
//     share power-of-two bins), and the list of hub rows (more than H in-edges).
//  3. k_sell_slices: slices of 32 consecutive sorted rows, their widths and
//     row slots; k_scan_widths: element offsets of the slices.
//  4. k_sell_fill: the slice arrays (one warp per slice), columns in groups
//     of 4 so that a lane reads 4 of its row's sources with one 128-bit load;
//     the empty slots of rows shorter than their slice (and of the columns
//     rounding the width up to 4) hold the partition's padding id, whose
//     value slot always holds the merge's identity.
//  5. k_hub_rows / k_scan_parts / k_hub_parts: hub rows in id order, split
//     into parts of T edges.
//  6. k_order_count / k_order_offsets / k_order_scatter: all partitions'
//     slice descriptors stably ordered by decreasing width (heavy slices first:
//     the hardware then schedules light ones at the tail).
#include <algorithm>

#include "gxp_internal.hpp"

namespace gxp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr uint32_t kSortMax = 2048;     // longest row sorted (shared-memory bitonic)
constexpr uint32_t kExactBins = 1024;   // in-degrees / widths ordered exactly up to here
constexpr uint32_t kBins = kExactBins + 34;   // above: one bin per power of two
constexpr int kSortWarps = 8;             // warps of a counting-sort CTA
constexpr uint32_t kSortChunk = kSellWindow / kSortWarps;   // items per warp

// Sort keys: (source << 32 | weight) for weighted rows, the source alone
// otherwise (bitonic sorting is deterministic, so equal sources keep a fixed
// order either way).
template <bool kW> struct SortKey;
template <> struct SortKey<true> {
    using T = uint64_t;
    static constexpr T kMax = ~0ull;
    __device__ static T make(uint32_t s, const uint32_t* w, uint32_t i) { return ((uint64_t)s << 32) | w[i]; }
    __device__ static uint32_t src(T k) { return (uint32_t)(k >> 32); }
    __device__ static uint32_t wt(T k) { return (uint32_t)k; }
};
template <> struct SortKey<false> {
    using T = uint32_t;
    static constexpr T kMax = ~0u;
    __device__ static T make(uint32_t s, const uint32_t*, uint32_t) { return s; }
    __device__ static uint32_t src(T k) { return k; }
    __device__ static uint32_t wt(T) { return 0u; }
};

// Bitonic sort of 32 * kSlots keys held as x[s] at index s * 32 + lane;
// stopping after the stage of size n (a power of two) sorts keys [0, n).
template <int kSlots, class T>
__device__ __forceinline__ void warp_bitonic(T (&x)[kSlots], int lane, int n) {
    constexpr int N = 32 * kSlots;
#pragma unroll
    for (int k = 2; k <= N; k <<= 1) {
        if (k > n) break;
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
#pragma unroll
                for (int s = 0; s < kSlots; ++s) {
                    const int ps = s ^ (j >> 5);
                    if (ps > s) {
                        const bool up = ((s * 32 + lane) & k) == 0;
                        const T a = x[s], b = x[ps];
                        if ((a > b) == up) {
                            x[s] = b;
                            x[ps] = a;
                        }
                    }
                }
            } else {
#pragma unroll
                for (int s = 0; s < kSlots; ++s) {
                    const T o = __shfl_xor_sync(kFull, x[s], j);
                    const bool up = ((s * 32 + lane) & k) == 0;
                    const bool lower = (lane & j) == 0;
                    x[s] = (lower == up) ? (x[s] < o ? x[s] : o) : (x[s] < o ? o : x[s]);
                }
            }
        }
    }
}

template <int kSlots, bool kW>
__device__ __forceinline__ void sort_row_in_warp(uint32_t b, uint32_t ib, uint32_t d, const uint32_t* src,
                                                 const uint32_t* w, const uint32_t* src_map, uint32_t* ssrc,
                                                 uint32_t* sw, int lane) {
    using K = SortKey<kW>;
    typename K::T x[kSlots];
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        const uint32_t i = s * 32 + lane;
        if (i < d) {
            const uint32_t u = src[ib + i];
            x[s] = K::make(src_map ? src_map[u] : u, w, ib + i);
        } else {
            x[s] = K::kMax;
        }
    }
    int np2 = 2;
    while (np2 < (int)d) np2 <<= 1;
    warp_bitonic<kSlots>(x, lane, np2);
#pragma unroll
    for (int s = 0; s < kSlots; ++s) {
        const uint32_t i = s * 32 + lane;
        if (i < d) {
            ssrc[b + i] = K::src(x[s]);
            if (kW) sw[b + i] = K::wt(x[s]);
        }
    }
}

// A warp takes 32 consecutive rows at a time: their offsets (and, through
// the row map, where their edges come from) are read by one lane each, so
// the rows' headers cost one round of loads rather than a chain per row, and
// rows without edges cost nothing more. Then the warp sorts the rows of up to
// 256 edges one after another and lists the runs of kSortMax edges of longer
// rows ({row, first edge of the run}) for the block sort.
template <bool kW>
__global__ void k_sort_rows_warp(const uint32_t* col_ptr, uint32_t n, const RowSource in, uint32_t* ssrc,
                                 uint32_t* sw, uint2* big_runs, uint32_t* n_big) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t v0 = warp0 * 32; v0 < n; v0 += n_warps * 32) {
        const uint64_t v = v0 + (uint32_t)lane;
        uint32_t b = 0, d = 0, ib = 0;
        if (v < n) {
            b = col_ptr[v];
            d = col_ptr[v + 1] - b;
            if (d) ib = in.col_ptr[in.row_map ? in.row_map[v] : (uint32_t)v];
        }
        for (unsigned todo = __ballot_sync(kFull, d != 0u); todo; todo &= todo - 1u) {
            const int r = __ffs(todo) - 1;
            const uint32_t rb = __shfl_sync(kFull, b, r), rd = __shfl_sync(kFull, d, r), rib = __shfl_sync(kFull, ib, r);
            // the smallest register network that holds the row
            if (rd <= 32) {
                sort_row_in_warp<1, kW>(rb, rib, rd, in.src, in.w, in.src_map, ssrc, sw, lane);
            } else if (rd <= 64) {
                sort_row_in_warp<2, kW>(rb, rib, rd, in.src, in.w, in.src_map, ssrc, sw, lane);
            } else if (rd <= 128) {
                sort_row_in_warp<4, kW>(rb, rib, rd, in.src, in.w, in.src_map, ssrc, sw, lane);
            } else if (rd <= 256) {
                sort_row_in_warp<8, kW>(rb, rib, rd, in.src, in.w, in.src_map, ssrc, sw, lane);
            } else {
                const uint32_t runs = (rd + kSortMax - 1) / kSortMax;
                uint32_t at = 0;
                if (lane == 0) at = atomicAdd(n_big, runs);
                at = __shfl_sync(kFull, at, 0);
                for (uint32_t k = lane; k < runs; k += 32)
                    big_runs[at + k] = make_uint2((uint32_t)(v0 + (uint32_t)r), k * kSortMax);
            }
        }
    }
}

// One CTA per listed run (257 .. kSortMax edges): a stable LSD radix sort of
// the run's sources in shared memory, 8 bits per pass (ceil(key_bits / 8)
// passes), carrying each edge's position in the run so that weights follow.
// Equal sources keep their input order. Warp w owns positions [256 w, 256 w
// + 256) and walks them 32 at a time in order: per pass it counts the digits
// of its keys (match_any groups), a scan over (digit, warp) gives every
// warp's first slot per digit, and the second walk places each key at its
// slot plus its rank among the equal digits of its 32.
constexpr int kRadixWarps = 8;
constexpr uint32_t kRadixPerWarp = kSortMax / kRadixWarps;   // 256
static_assert(kRadixPerWarp % 32 == 0, "whole warp steps");

template <bool kW>
__global__ void __launch_bounds__(kRadixWarps * 32) k_sort_rows_block(const uint32_t* col_ptr, const RowSource in,
                                                                      uint32_t* ssrc, uint32_t* sw,
                                                                      const uint2* big_runs, const uint32_t* n_big,
                                                                      uint32_t key_bits) {
    __shared__ uint32_t key[2][kSortMax];
    __shared__ uint16_t pos[2][kSortMax];
    __shared__ uint32_t hist[kRadixWarps][256];
    __shared__ uint32_t warp_tot[kRadixWarps];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t cnt = *n_big;
    const uint32_t passes = (key_bits + 7) / 8;
    for (uint32_t r = blockIdx.x; r < cnt; r += gridDim.x) {
        const uint2 run = big_runs[r];
        const uint32_t b = col_ptr[run.x] + run.y;
        const uint32_t d = min(kSortMax, col_ptr[run.x + 1] - b);
        const uint32_t ib = in.col_ptr[in.row_map ? in.row_map[run.x] : run.x] + run.y;
        __syncthreads();   // the previous run's buffers are read out
        for (uint32_t i = tid; i < d; i += blockDim.x) {
            const uint32_t u = in.src[ib + i];
            key[0][i] = in.src_map ? in.src_map[u] : u;
            pos[0][i] = (uint16_t)i;
        }
        int cur = 0;
        // this warp's positions (runs shorter than kSortMax leave the last warps idle)
        const uint32_t w_end = min((uint32_t)(warp + 1) * kRadixPerWarp, (d + 31u) & ~31u);
        for (uint32_t p = 0; p < passes; ++p) {
            const uint32_t sh = 8u * p;
            for (uint32_t i = tid; i < kRadixWarps * 256; i += blockDim.x) (&hist[0][0])[i] = 0u;
            __syncthreads();
            // counts of each warp's digits
            for (uint32_t j0 = (uint32_t)warp * kRadixPerWarp; j0 < w_end; j0 += 32) {
                const uint32_t i = j0 + (uint32_t)lane;
                const bool has = i < d;
                const uint32_t dg = has ? (key[cur][i] >> sh) & 255u : 0u;
                const unsigned act = __ballot_sync(kFull, has);
                if (has) {
                    const unsigned grp = __match_any_sync(act, dg);
                    if (lane == __ffs(grp) - 1) hist[warp][dg] += (uint32_t)__popc(grp);
                }
                __syncwarp();
            }
            __syncthreads();
            // first slot of (digit, warp): digits ascending, warps in order
            {
                const uint32_t dg = (uint32_t)tid;   // 256 threads, one digit each
                uint32_t c[kRadixWarps], tot = 0;
#pragma unroll
                for (int w = 0; w < kRadixWarps; ++w) {
                    c[w] = hist[w][dg];
                    tot += c[w];
                }
                uint32_t incl = tot;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    const uint32_t y = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o) incl += y;
                }
                if (lane == 31) warp_tot[warp] = incl;
                __syncthreads();
                uint32_t base = incl - tot;
                for (int w = 0; w < warp; ++w) base += warp_tot[w];
#pragma unroll
                for (int w = 0; w < kRadixWarps; ++w) {
                    hist[w][dg] = base;
                    base += c[w];
                }
            }
            __syncthreads();
            // place: each warp's keys in order, equal digits ranked by lane
            for (uint32_t j0 = (uint32_t)warp * kRadixPerWarp; j0 < w_end; j0 += 32) {
                const uint32_t i = j0 + (uint32_t)lane;
                const bool has = i < d;
                const uint32_t k = has ? key[cur][i] : 0u;
                const uint32_t dg = (k >> sh) & 255u;
                const unsigned act = __ballot_sync(kFull, has);
                unsigned grp = 0;
                if (has) {
                    grp = __match_any_sync(act, dg);
                    const uint32_t at = hist[warp][dg] + (uint32_t)__popc(grp & ((1u << lane) - 1u));
                    key[cur ^ 1][at] = k;
                    pos[cur ^ 1][at] = pos[cur][i];
                }
                __syncwarp();
                if (has && lane == __ffs(grp) - 1) hist[warp][dg] += (uint32_t)__popc(grp);
                __syncwarp();
            }
            __syncthreads();
            cur ^= 1;
        }
        for (uint32_t i = tid; i < d; i += blockDim.x) {
            ssrc[b + i] = key[cur][i];
            if (kW) sw[b + i] = in.w[ib + pos[cur][i]];
        }
    }
}

__device__ __forceinline__ uint32_t deg_bin(uint32_t d) {
    return d <= kExactBins ? d : kExactBins + (31u - (uint32_t)__clz(d));
}

// Exclusive offsets in descending bin order over a [kSortWarps][kBins]
// table of per-warp counts, warps in order inside a bin (a stable counting
// sort); the whole CTA takes part.
__device__ void warp_bin_offsets(uint32_t (*hist)[kBins], uint32_t* tot) {
    for (uint32_t b = threadIdx.x; b < kBins; b += blockDim.x) {
        uint32_t t = 0;
        for (int w = 0; w < kSortWarps; ++w) t += hist[w][b];
        tot[b] = t;
    }
    __syncthreads();
    if (threadIdx.x < 32) {   // descending exclusive scan of tot: lane l takes a chunk of bins
        const int lane = threadIdx.x;
        constexpr uint32_t kChunk = (kBins + 31) / 32;
        const int hi = (int)kBins - 1 - lane * (int)kChunk;
        uint32_t sum = 0;
        for (int i = 0; i < (int)kChunk; ++i)
            if (hi - i >= 0) sum += tot[hi - i];
        uint32_t incl = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t t = __shfl_up_sync(kFull, incl, o);
            if (lane >= o) incl += t;
        }
        uint32_t run = incl - sum;
        for (int i = 0; i < (int)kChunk; ++i)
            if (hi - i >= 0) {
                const uint32_t c = tot[hi - i];
                tot[hi - i] = run;
                run += c;
            }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < kBins; b += blockDim.x) {
        uint32_t run = tot[b];
        for (int w = 0; w < kSortWarps; ++w) {
            const uint32_t c = hist[w][b];
            hist[w][b] = run;
            run += c;
        }
    }
    __syncthreads();
}

// Stable scatter of one warp's items [i0, i1) by descending bin: key(i)
// returns the bin, or kBins for an item that is skipped.
template <class Key, class Put>
__device__ void warp_scatter(uint32_t i0, uint32_t i1, uint32_t* offs, Key key, Put put) {
    const int lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t j0 = i0; j0 < i1; j0 += 32) {
        const uint32_t j = j0 + lane;
        const uint32_t k = j < i1 ? key(j) : kBins;
        const bool ok = k < kBins;
        const uint32_t grp = __match_any_sync(kFull, ok ? k : 0x80000000u | (uint32_t)lane);   // alone if skipped
        if (ok) put(j, offs[k] + __popc(grp & lt));
        __syncwarp();
        if (ok && (grp & lt) == 0u) offs[k] += __popc(grp);
        __syncwarp();
    }
}

// One CTA per window of kSellWindow rows: stable counting sort of the rows
// with at most H in-edges by descending in-degree (each warp counts and then
// scatters its 1/kSortWarps of the window), hub rows in id order;
// window-relative outputs.
__global__ void __launch_bounds__(kSortWarps * 32) k_sell_windows(const uint32_t* col_ptr, uint32_t n, uint32_t H,
                                                                  uint32_t* rows_out, uint32_t* hub_out,
                                                                  uint32_t* nonhub_cnt, uint32_t* hub_cnt) {
    __shared__ uint32_t hist[kSortWarps][kBins];
    __shared__ uint32_t tot[kBins];
    __shared__ uint32_t hubs[kSortWarps];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t win = blockIdx.x;
    const uint32_t w0 = win * kSellWindow;
    const uint32_t w1 = (uint32_t)min((uint64_t)w0 + kSellWindow, (uint64_t)n);
    const uint32_t c0 = min(w1, w0 + warp * kSortChunk), c1 = min(w1, c0 + kSortChunk);
    for (uint32_t i = threadIdx.x; i < kSortWarps * kBins; i += blockDim.x) (&hist[0][0])[i] = 0u;
    __syncthreads();
    uint32_t nh = 0;
    for (uint32_t v0 = c0; v0 < c1; v0 += 32) {
        const uint32_t v = v0 + lane;
        bool hub = false;
        if (v < c1) {
            const uint32_t d = col_ptr[v + 1] - col_ptr[v];
            hub = d > H;
            if (!hub) atomicAdd(&hist[warp][deg_bin(d)], 1u);
        }
        nh += __popc(__ballot_sync(kFull, hub));
    }
    if (lane == 0) hubs[warp] = nh;
    __syncthreads();
    warp_bin_offsets(hist, tot);
    uint32_t hub_at = 0, hub_total = 0;
    for (int w = 0; w < kSortWarps; ++w) {
        if (w < warp) hub_at += hubs[w];
        hub_total += hubs[w];
    }
    warp_scatter(
        c0, c1, hist[warp],
        [&](uint32_t v) {
            const uint32_t d = col_ptr[v + 1] - col_ptr[v];
            return d > H ? kBins : deg_bin(d);
        },
        [&](uint32_t v, uint32_t pos) { rows_out[w0 + pos] = v; });
    // hub rows, in id order (warp-ordered ranks)
    const uint32_t lt = (1u << lane) - 1u;
    for (uint32_t v0 = c0; v0 < c1; v0 += 32) {
        const uint32_t v = v0 + lane;
        const bool hub = v < c1 && col_ptr[v + 1] - col_ptr[v] > H;
        const uint32_t hb = __ballot_sync(kFull, hub);
        if (hub) hub_out[w0 + hub_at + __popc(hb & lt)] = v;
        hub_at += __popc(hb);
    }
    if (threadIdx.x == 0) {
        nonhub_cnt[win] = (w1 - w0) - hub_total;
        hub_cnt[win] = hub_total;
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

// single CTA: exclusive prefix of a slice's storage, 32 * round_up(width, 4)
// words (u64), over n slices; out[n] = total
__global__ void __launch_bounds__(1024) k_scan_widths(const uint32_t* width, uint32_t n, bool g4, uint64_t* out) {
    auto slice_words = [g4](uint32_t w) { return 32ull * sell_cols(w, g4); };
    __shared__ unsigned long long part[1024];
    const uint32_t t = threadIdx.x;
    const uint32_t per = (n + 1023) / 1024;
    const uint32_t a = min(n, t * per), b = min(n, a + per);
    unsigned long long s = 0;
    for (uint32_t i = a; i < b; ++i) s += slice_words(width[i]);
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
        run += slice_words(width[i]);
    }
    if (t == 1023) out[n] = part[1023];
}

// one warp per slice: the sources (and weights) in groups of 4 columns, lane
// l's 4 entries of group g at off + 128 g + 4 l (sell_idx), descriptors
__global__ void k_sell_fill(const uint32_t* col_ptr, const uint32_t* ssrc, const uint32_t* sw, const uint32_t* perm,
                            const uint32_t* width, const uint64_t* off, uint32_t n_slices, uint32_t part,
                            uint32_t pad_id, bool g4, uint32_t* sell_src, uint32_t* sell_w, SellSlice* desc) {
    const int lane = threadIdx.x & 31;
    const uint64_t warp0 = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    const uint64_t n_warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t s = warp0; s < n_slices; s += n_warps) {
        const uint32_t r = perm[s * 32 + lane];
        const uint32_t wd = width[s], w4 = sell_cols(wd, g4);
        const uint64_t o = off[s];
        const uint32_t b = r != kSellPad ? col_ptr[r] : 0u;
        const uint32_t d = r != kSellPad ? col_ptr[r + 1] - b : 0u;
        for (uint32_t k = 0; k < w4; ++k) {
            const bool has = k < d;
            const uint64_t at = o + sell_idx(k, (uint32_t)lane, g4);
            sell_src[at] = has ? ssrc[b + k] : pad_id;
            if (sell_w) sell_w[at] = has ? sw[b + k] : 0u;
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

// All slice descriptors stably ordered by decreasing width (exact up to
// kExactBins, by power of two above), in three steps over chunks of
// kSellWindow descriptors: per-warp counts, offsets, per-warp scatter.
__global__ void __launch_bounds__(kSortWarps * 32) k_order_count(const SellSlice* in, uint32_t n, uint32_t* ghist) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ uint32_t hist[kSortWarps][kBins];
    for (uint32_t i = threadIdx.x; i < kSortWarps * kBins; i += blockDim.x) (&hist[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t c0 = min(n, blockIdx.x * kSellWindow + warp * kSortChunk), c1 = min(n, c0 + kSortChunk);
    for (uint32_t i = c0 + lane; i < c1; i += 32) atomicAdd(&hist[warp][deg_bin(in[i].width)], 1u);
    __syncthreads();
    uint32_t* g = ghist + (uint64_t)blockIdx.x * kSortWarps * kBins;
    for (uint32_t i = threadIdx.x; i < kSortWarps * kBins; i += blockDim.x) g[i] = (&hist[0][0])[i];
}

// single CTA: per-(chunk, warp) offsets for every bin, bins descending, chunks
// and warps in order
__global__ void __launch_bounds__(1024) k_order_offsets(uint32_t* ghist, uint32_t n_warps_total) {
    __shared__ uint32_t tot[kBins];
    for (uint32_t b = threadIdx.x; b < kBins; b += blockDim.x) {
        uint32_t t = 0;
        for (uint32_t w = 0; w < n_warps_total; ++w) t += ghist[(uint64_t)w * kBins + b];
        tot[b] = t;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t run = 0;
        for (int b = (int)kBins - 1; b >= 0; --b) {
            const uint32_t c = tot[b];
            tot[b] = run;
            run += c;
        }
    }
    __syncthreads();
    for (uint32_t b = threadIdx.x; b < kBins; b += blockDim.x) {
        uint32_t run = tot[b];
        for (uint32_t w = 0; w < n_warps_total; ++w) {
            const uint32_t c = ghist[(uint64_t)w * kBins + b];
            ghist[(uint64_t)w * kBins + b] = run;
            run += c;
        }
    }
}

__global__ void __launch_bounds__(kSortWarps * 32) k_order_scatter(const SellSlice* in, uint32_t n, uint32_t* ghist,
                                                                   SellSlice* out) {
    const int warp = threadIdx.x >> 5;
    const uint32_t c0 = min(n, blockIdx.x * kSellWindow + warp * kSortChunk), c1 = min(n, c0 + kSortChunk);
    uint32_t* offs = ghist + ((uint64_t)blockIdx.x * kSortWarps + warp) * kBins;
    warp_scatter(
        c0, c1, offs, [&](uint32_t i) { return deg_bin(in[i].width); },
        [&](uint32_t i, uint32_t pos) { out[pos] = in[i]; });
}

// ------------------------------------------------------ vertex relabelling
// new id i = rank of the vertex in a stable order by decreasing in-degree, so
// the most gathered values share cache lines (exact up to kExactBins, by
// power of two above)

__global__ void __launch_bounds__(kSortWarps * 32) k_vdeg_count(const uint32_t* col_ptr, uint32_t n,
                                                                uint32_t* ghist) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    __shared__ uint32_t hist[kSortWarps][kBins];
    for (uint32_t i = threadIdx.x; i < kSortWarps * kBins; i += blockDim.x) (&hist[0][0])[i] = 0u;
    __syncthreads();
    const uint32_t c0 = min(n, blockIdx.x * kSellWindow + warp * kSortChunk), c1 = min(n, c0 + kSortChunk);
    for (uint32_t v = c0 + lane; v < c1; v += 32) atomicAdd(&hist[warp][deg_bin(col_ptr[v + 1] - col_ptr[v])], 1u);
    __syncthreads();
    uint32_t* g = ghist + (uint64_t)blockIdx.x * kSortWarps * kBins;
    for (uint32_t i = threadIdx.x; i < kSortWarps * kBins; i += blockDim.x) g[i] = (&hist[0][0])[i];
}

__global__ void __launch_bounds__(kSortWarps * 32) k_vdeg_scatter(const uint32_t* col_ptr, uint32_t n,
                                                                  uint32_t* ghist, uint32_t* new2old) {
    const int warp = threadIdx.x >> 5;
    const uint32_t c0 = min(n, blockIdx.x * kSellWindow + warp * kSortChunk), c1 = min(n, c0 + kSortChunk);
    uint32_t* offs = ghist + ((uint64_t)blockIdx.x * kSortWarps + warp) * kBins;
    warp_scatter(
        c0, c1, offs, [&](uint32_t v) { return deg_bin(col_ptr[v + 1] - col_ptr[v]); },
        [&](uint32_t v, uint32_t pos) { new2old[pos] = v; });
}

// old2new = inverse of new2old; rdeg[i] = in-degree of new vertex i
__global__ void k_invert(const uint32_t* col_ptr, const uint32_t* new2old, uint32_t n, uint32_t* old2new,
                         uint32_t* rdeg) {
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
        const uint32_t v = new2old[i];
        old2new[v] = i;
        rdeg[i] = col_ptr[v + 1] - col_ptr[v];
    }
}

// three-phase exclusive scan of u32 counts: x[0..n) -> out[0..n], out[n] = total
constexpr uint32_t kScanChunk = 2048;
__global__ void __launch_bounds__(256) k_scan_sums(const uint32_t* x, uint32_t n, uint32_t* sums) {
    __shared__ uint32_t red[8];
    const uint32_t c0 = blockIdx.x * kScanChunk, c1 = min(n, c0 + kScanChunk);
    uint32_t s = 0;
    for (uint32_t i = c0 + threadIdx.x; i < c1; i += blockDim.x) s += x[i];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
    if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        uint32_t t = 0;
        for (int w = 0; w < 8; ++w) t += red[w];
        sums[blockIdx.x] = t;
    }
}

__global__ void __launch_bounds__(1024) k_scan_top(uint32_t* sums, uint32_t m) {
    __shared__ uint32_t part[1024];
    const uint32_t t = threadIdx.x, per = (m + 1023) / 1024;
    const uint32_t a = min(m, t * per), b = min(m, a + per);
    uint32_t s = 0;
    for (uint32_t i = a; i < b; ++i) s += sums[i];
    part[t] = s;
    __syncthreads();
    for (uint32_t o = 1; o < 1024; o <<= 1) {
        const uint32_t v = t >= o ? part[t - o] : 0u;
        __syncthreads();
        part[t] += v;
        __syncthreads();
    }
    uint32_t run = part[t] - s;
    for (uint32_t i = a; i < b; ++i) {
        const uint32_t c = sums[i];
        sums[i] = run;
        run += c;
    }
}

__global__ void __launch_bounds__(256) k_scan_apply(const uint32_t* x, uint32_t n, const uint32_t* sums,
                                                    uint32_t* out) {
    __shared__ uint32_t warp_tot[8];
    const uint32_t c0 = blockIdx.x * kScanChunk;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    // thread t owns 8 consecutive elements of the chunk
    constexpr uint32_t kPer = kScanChunk / 256;
    const uint32_t base = c0 + threadIdx.x * kPer;
    uint32_t v[kPer], s = 0;
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
        v[k] = base + k < n ? x[base + k] : 0u;
        s += v[k];
    }
    uint32_t incl = s;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(kFull, incl, o);
        if (lane >= o) incl += y;
    }
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    uint32_t wbase = 0;
    for (int w = 0; w < warp; ++w) wbase += warp_tot[w];
    uint32_t run = sums[blockIdx.x] + wbase + incl - s;
#pragma unroll
    for (uint32_t k = 0; k < kPer; ++k) {
        if (base + k < n) out[base + k] = run;
        run += v[k];
        if (base + k + 1 == n) out[n] = run;
    }
}

__global__ void k_gather_u32(const uint32_t* in, const uint32_t* map, uint32_t n, uint32_t* out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) out[v] = in[map[v]];
}

__global__ void k_scatter_u32(const uint32_t* in, const uint32_t* map, uint32_t n, uint32_t* out) {
    for (uint32_t v = blockIdx.x * blockDim.x + threadIdx.x; v < n; v += gridDim.x * blockDim.x) out[map[v]] = in[v];
}

uint32_t grid_warps(uint64_t warps, uint32_t block) {
    const uint64_t b = (warps * 32 + block - 1) / block;
    return (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(b, 152ull * 64));
}

}  // namespace

cudaError_t launch_sort_rows(const uint32_t* col_ptr, uint32_t n, const RowSource& in, uint32_t n_src,
                             uint32_t* ssrc, uint32_t* sw, uint2* scratch_runs, uint32_t* scratch_cnt, cudaStream_t s) {
    cudaError_t e = cudaMemsetAsync(scratch_cnt, 0, 4, s);
    if (e != cudaSuccess) return e;
    if (n == 0) return cudaSuccess;
    uint32_t key_bits = 1;   // bits of the largest source id
    while (key_bits < 32 && ((uint64_t)(n_src ? n_src - 1 : 0) >> key_bits) != 0) ++key_bits;
    if (in.w) {
        k_sort_rows_warp<true><<<grid_warps((n + 31) / 32, 256), 256, 0, s>>>(col_ptr, n, in, ssrc, sw, scratch_runs,
                                                                             scratch_cnt);
        k_sort_rows_block<true><<<152 * 6, kRadixWarps * 32, 0, s>>>(col_ptr, in, ssrc, sw, scratch_runs, scratch_cnt,
                                                                      key_bits);
    } else {
        k_sort_rows_warp<false><<<grid_warps((n + 31) / 32, 256), 256, 0, s>>>(col_ptr, n, in, ssrc, sw, scratch_runs,
                                                                              scratch_cnt);
        k_sort_rows_block<false><<<152 * 6, kRadixWarps * 32, 0, s>>>(col_ptr, in, ssrc, sw, scratch_runs, scratch_cnt,
                                                                       key_bits);
    }
    return cudaGetLastError();
}

cudaError_t launch_sell_windows(const uint32_t* col_ptr, uint32_t n, uint32_t H, uint32_t* rows_out,
                                uint32_t* hub_out, uint32_t* nonhub_cnt, uint32_t* hub_cnt, cudaStream_t s) {
    const uint32_t nw = (n + kSellWindow - 1) / kSellWindow;
    if (nw == 0) return cudaSuccess;
    k_sell_windows<<<nw, kSortWarps * 32, 0, s>>>(col_ptr, n, H, rows_out, hub_out, nonhub_cnt, hub_cnt);
    return cudaGetLastError();
}

cudaError_t launch_sell_slices(const uint32_t* col_ptr, uint32_t n, const uint32_t* rows_out,
                               const uint32_t* nonhub_cnt, const uint32_t* slice_base, uint32_t* perm,
                               uint32_t* width, uint64_t* off, uint32_t n_slices, bool g4, cudaStream_t s) {
    const uint32_t nw = (n + kSellWindow - 1) / kSellWindow;
    if (nw) k_sell_slices<<<nw, 256, 0, s>>>(col_ptr, rows_out, nonhub_cnt, slice_base, perm, width);
    k_scan_widths<<<1, 1024, 0, s>>>(width, n_slices, g4, off);
    return cudaGetLastError();
}

cudaError_t launch_sell_fill(const uint32_t* col_ptr, const uint32_t* ssrc, const uint32_t* sw, const uint32_t* perm,
                             const uint32_t* width, const uint64_t* off, uint32_t n_slices, uint32_t part,
                             uint32_t pad_id, bool g4, uint32_t* sell_src, uint32_t* sell_w, SellSlice* desc,
                             cudaStream_t s) {
    if (n_slices == 0) return cudaSuccess;
    k_sell_fill<<<grid_warps(n_slices, 256), 256, 0, s>>>(col_ptr, ssrc, sw, perm, width, off, n_slices, part,
                                                          pad_id, g4, sell_src, sell_w, desc);
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

cudaError_t launch_order_slices(const SellSlice* in, uint32_t n, SellSlice* out, uint32_t* scratch,
                                cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t chunks = (n + kSellWindow - 1) / kSellWindow;
    k_order_count<<<chunks, kSortWarps * 32, 0, s>>>(in, n, scratch);
    k_order_offsets<<<1, 1024, 0, s>>>(scratch, chunks * kSortWarps);
    k_order_scatter<<<chunks, kSortWarps * 32, 0, s>>>(in, n, scratch, out);
    return cudaGetLastError();
}

size_t order_slices_scratch_bytes(uint32_t n) {
    const uint64_t chunks = (n + kSellWindow - 1) / kSellWindow;
    return 4 * (size_t)(chunks + 1) * kSortWarps * kBins;
}

}  // namespace gxp

namespace gxp {

size_t relabel_scratch_bytes(uint32_t n) {
    const uint64_t chunks = (n + kSellWindow - 1) / kSellWindow;
    const uint64_t scan_blocks = (n + kScanChunk - 1) / kScanChunk;
    return 4 * ((size_t)(chunks + 1) * kSortWarps * kBins + (size_t)scan_blocks + 1 + (size_t)n + 1);
}

cudaError_t launch_relabel(const uint32_t* col_ptr, uint32_t n, uint32_t* new2old, uint32_t* old2new, uint32_t* rcol,
                           uint32_t* scratch, cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t chunks = (n + kSellWindow - 1) / kSellWindow;
    const uint32_t scan_blocks = (n + kScanChunk - 1) / kScanChunk;
    uint32_t* ghist = scratch;
    uint32_t* sums = ghist + (size_t)(chunks + 1) * kSortWarps * kBins;
    uint32_t* rdeg = sums + scan_blocks + 1;
    k_vdeg_count<<<chunks, kSortWarps * 32, 0, s>>>(col_ptr, n, ghist);
    k_order_offsets<<<1, 1024, 0, s>>>(ghist, chunks * kSortWarps);
    k_vdeg_scatter<<<chunks, kSortWarps * 32, 0, s>>>(col_ptr, n, ghist, new2old);
    const uint32_t g = std::min<uint32_t>((n + 255) / 256, 152u * 16);
    k_invert<<<g, 256, 0, s>>>(col_ptr, new2old, n, old2new, rdeg);
    k_scan_sums<<<scan_blocks, 256, 0, s>>>(rdeg, n, sums);
    k_scan_top<<<1, 1024, 0, s>>>(sums, scan_blocks);
    k_scan_apply<<<scan_blocks, 256, 0, s>>>(rdeg, n, sums, rcol);
    return cudaGetLastError();
}

cudaError_t launch_exclusive_scan_u32(const uint32_t* x, uint32_t n, uint32_t* out, uint32_t* scratch,
                                      cudaStream_t s) {
    if (n == 0) return cudaMemsetAsync(out, 0, 4, s);
    const uint32_t scan_blocks = (n + kScanChunk - 1) / kScanChunk;
    k_scan_sums<<<scan_blocks, 256, 0, s>>>(x, n, scratch);
    k_scan_top<<<1, 1024, 0, s>>>(scratch, scan_blocks);
    k_scan_apply<<<scan_blocks, 256, 0, s>>>(x, n, scratch, out);
    return cudaGetLastError();
}

cudaError_t launch_permute_u32(const uint32_t* in, const uint32_t* map, uint32_t n, uint32_t* out, bool scatter,
                               cudaStream_t s) {
    if (n == 0) return cudaSuccess;
    const uint32_t g = std::min<uint32_t>((n + 255) / 256, 152u * 16);
    if (scatter) k_scatter_u32<<<g, 256, 0, s>>>(in, map, n, out);
    else k_gather_u32<<<g, 256, 0, s>>>(in, map, n, out);
    return cudaGetLastError();
}

}  // namespace gxp
