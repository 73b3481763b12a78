// Device helpers shared by the pull (sell.cu) and push (frontier.cu)
// supersteps of the min-label algorithms: the per-superstep direction choice
// and the warp-cooperative append of changed vertices to the next frontier.
#pragma once

#include "gxp_internal.hpp"

namespace gxp {

// Direction of the superstep that reads `in` (the previous superstep's
// slot). Every thread of both kernels evaluates it on the same words, so the
// two kernels launched for a superstep agree on which of them does the work.
__device__ __forceinline__ bool push_chosen(const FrontierCfg& f, const StepStats* in) {
    if (f.list_out == nullptr) return false;
    if (f.direction == GXP_DIR_PUSH) return true;
    if (f.direction == GXP_DIR_PULL) return false;
    // partitions: an exchange that did not list its changed copies leaves an
    // incomplete frontier, which only a pull may follow
    if (in->exchanged && !in->list_copies) return false;
    if (in->unlisted) return false;   // the previous pull did not list its changed vertices
    const unsigned long long ne = in->list_ne;
    const unsigned long long work = (ne >> 32) + (ne & 0xFFFFFFFFull);
    return work * (unsigned long long)f.push_div <= f.total_edges;
}

__device__ __forceinline__ uint32_t warp_inclusive_scan(uint32_t x, int lane) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xFFFFFFFFu, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// Lane whose range [incl - n, incl) of a warp's inclusive scan holds k: the
// number of lanes with incl <= k (binary search over the nondecreasing scan).
// All 32 lanes must call it; k at or past the total gives lane 31.
__device__ __forceinline__ int warp_owner(uint32_t incl, uint32_t k) {
    int lo = 0;
#pragma unroll
    for (int s = 16; s > 0; s >>= 1) {
        const uint32_t x = __shfl_sync(0xFFFFFFFFu, incl, lo + s - 1);
        if (x <= k) lo += s;
    }
    return lo;
}

__device__ __forceinline__ uint32_t frontier_items(uint32_t deg) {
    const uint32_t n = (deg / kItemEdges) + ((deg % kItemEdges) != 0u ? 1u : 0u);
    return n ? n : 1u;
}

// Write the items of the lanes' vertices (warp inclusive scan `incl` of
// their item counts `nit`) at list positions base + [0, total).
__device__ __forceinline__ void frontier_write(const FrontierCfg& f, unsigned long long base, uint32_t incl,
                                               uint32_t nit, uint32_t v, int lane) {
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    const uint32_t excl = incl - nit;
    for (uint32_t k0 = 0; k0 < total; k0 += 32u) {
        const uint32_t k = k0 + (uint32_t)lane;
        const int j = warp_owner(incl, k);
        const uint32_t vj = __shfl_sync(0xFFFFFFFFu, v, j);
        const uint32_t ej = __shfl_sync(0xFFFFFFFFu, excl, j);
        if (k < total) {
            if (base + k < f.list_cap) f.list_out[base + k] = make_uint2(vj, k - ej);
            else atomicOr(f.err, kErrBounds);
        }
    }
}

// Append the work items of vertex v (out-degree deg) for every lane with
// `has`, one atomic per warp for the positions; the items are written by all
// lanes together, so a vertex with many out-edges does not serialize on one
// lane. All 32 lanes must call it.
__device__ __forceinline__ void frontier_append(bool has, uint32_t v, uint32_t deg, const FrontierCfg& f,
                                                StepStats* st, int lane) {
    if (__ballot_sync(0xFFFFFFFFu, has) == 0u) return;
    const uint32_t nit = has ? frontier_items(deg) : 0u;
    const uint32_t incl = warp_inclusive_scan(nit, lane);
    const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
    uint32_t edges = has ? deg : 0u;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) edges += __shfl_xor_sync(0xFFFFFFFFu, edges, o);
    unsigned long long base = 0ull;
    if (lane == 0) base = atomicAdd(&st->list_ne, list_pack(total, edges)) >> 32;
    base = __shfl_sync(0xFFFFFFFFu, base, 0);
    frontier_write(f, base, incl, nit, v, lane);
}

// SSSP: d[u] + w, saturating below INF (the pull rule); CC: l[u]
template <bool kW>
__device__ __forceinline__ uint32_t push_message(uint32_t du, uint32_t w) {
    if constexpr (kW) {
        uint32_t s = du + w;
        if (s < du || s == kInf) s = kInf - 1u;
        return s;
    } else {
        return du;
    }
}

// Push superstep of the min-label algorithms (called by every warp of the
// superstep grid when push_chosen): MSGGen over the out-edges of the
// frontier only (the vertices the previous superstep changed); MSGMerge +
// MSGApply become an atomic min into the next values.
// Sources are *slots*: [0, n_own_total) are the vertices themselves (their
// out-edges into their own partition), [n_own_total, ...) the partitions'
// cached copies of remote vertices (slot n_own_total + g for copy g, with
// that partition's in-edges from the vertex as out-edges). One partition has
// vertex slots only. Every edge belongs to exactly one slot, and every
// destination is a vertex of the partition holding the edge, so each
// partition's push writes only its own values. A destination that joins the
// next frontier also gets its changed bit (changed_bits, several partitions),
// from which the exchange uploads it; its cached copies join the next
// frontier when the exchange delivers them (k_sync_pull).
// Values stay double-buffered, so this is the same Jacobi superstep as the
// pull direction (same values, same changed set):
//  * sources' values come from the previous superstep's buffer, which
//    nothing writes during the superstep;
//  * the next buffer holds the values of two supersteps back, which differ
//    from the previous ones only at the frontier; each frontier vertex's
//    first item brings its entry up to date with an atomic min, in any order
//    against the relaxations (min commutes);
//  * a destination joins the next frontier exactly once: by the relaxation
//    whose atomic min first takes it below the previous superstep's value.
// Items (at most 32 out-edges) are spread evenly over all warps of the grid:
// a relaxation is a chain of dependent loads and atomics, so the superstep
// lasts as long as the longest chain a warp walks. A warp takes c <= 32
// consecutive items, scans their lengths and walks the concatenated edges
// 32 at a time, each lane finding its item by binary search over the scan.
// Returns the vertices this warp appended (changed), counted on every lane.
// kNC: the previous values may be read through the non-coherent path (a
// launch that runs one superstep); a persistent loop passes false.
template <bool kW, bool kNC = true>
__device__ __forceinline__ uint32_t push_superstep(const FrontierCfg& f, const uint32_t* out_ptr,
                                                   const uint32_t* out_dst, const uint32_t* out_w,
                                                   const uint32_t* own_cur, uint32_t* own_nxt,
                                                   const uint32_t* ghost, uint32_t n_own_total,
                                                   uint32_t* changed_bits,
                                                   const StepStats* stats_in, StepStats* stats_out,
                                                   uint64_t warp0, uint64_t n_warps, int lane) {
    const unsigned long long ne = stats_in->list_ne;
    const unsigned long long n_items = min(ne >> 32, (unsigned long long)f.list_cap);
    if (warp0 == 0 && lane == 0) {
        stats_out->pushed = 1ull;
        stats_out->push_edges = ne & 0xFFFFFFFFull;
    }
    const uint64_t per = (n_items + n_warps - 1) / n_warps;
    const uint32_t c = per >= 32u ? 32u : (per ? (uint32_t)per : 1u);
    uint32_t n_changed = 0;
    for (uint64_t b = warp0 * c; b < n_items; b += n_warps * c) {
        const uint64_t i = b + (uint64_t)lane;
        uint32_t e_lo = 0, n = 0, du = kInf;
        if ((uint32_t)lane < c && i < n_items) {
            const uint2 it = f.list_in[i];
            const uint32_t u = it.x;   // a slot
            const bool vertex = u < n_own_total;
            du = vertex ? own_cur[u] : ghost[u - n_own_total];
            const uint32_t r1 = out_ptr[u + 1];
            e_lo = out_ptr[u] + it.y * kItemEdges;
            n = min(r1 - e_lo, kItemEdges);
            // bring the next buffer up to date at vertex u (values only
            // decrease, so an entry already at or below du needs nothing)
            if (vertex && it.y == 0u && __ldcg(own_nxt + u) > du) atomicMin(own_nxt + u, du);
            if (kW && du == kInf) n = 0;   // unreachable: sends nothing
        }
        const uint32_t incl = warp_inclusive_scan(n, lane);
        const uint32_t excl = incl - n;
        const uint32_t total = __shfl_sync(0xFFFFFFFFu, incl, 31);
        for (uint32_t k0 = 0; k0 < total; k0 += 32u) {
            const uint32_t k = k0 + (uint32_t)lane;
            const int j = warp_owner(incl, k);
            const uint32_t e = __shfl_sync(0xFFFFFFFFu, e_lo, j) + (k - __shfl_sync(0xFFFFFFFFu, excl, j));
            const uint32_t dj = __shfl_sync(0xFFFFFFFFu, du, j);
            bool app = false;
            uint32_t v = 0, deg = 0;
            if (k < total) {
                v = out_dst[e];
                const uint32_t m = push_message<kW>(dj, kW ? out_w[e] : 0u);
                const uint32_t nv = __ldcg(own_nxt + v), cv = kNC ? __ldg(own_cur + v) : __ldca(own_cur + v);
                if (m < nv && m < cv) app = atomicMin(own_nxt + v, m) >= cv;
                if (app) {
                    deg = __ldg(out_ptr + v + 1) - __ldg(out_ptr + v);
                    if (changed_bits) atomicOr(changed_bits + (v >> 5), 1u << (v & 31u));
                }
            }
            n_changed += (uint32_t)__popc(__ballot_sync(0xFFFFFFFFu, app));
            frontier_append(app, v, deg, f, stats_out, lane);
        }
    }
    return n_changed;
}

}  // namespace gxp
