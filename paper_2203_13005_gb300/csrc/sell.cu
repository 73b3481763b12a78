// Superstep kernel over the sliced-ELL layout: MSGGen + MSGMerge + MSGApply
// (Section IV-A1's algorithm template) in pull form, one warp per work item.
// For SSSP and CC on one partition the same grid runs the push direction
// instead when the frontier is small (frontier.cuh); the choice is made on
// the device from the previous superstep's frontier size.
//
//  * slice of 32 non-hub rows (the edge block of Section II-B, laid out
//    column-major): lane i owns row i. For each of the slice's `width` edge
//    slots the warp reads 32 consecutive source ids (one coalesced 128-byte
//    load), gathers the sources' values with up to kUnroll independent loads
//    in flight per lane, and folds the messages into a per-lane register in
//    the row's edge order (MSGMerge without shuffles or shared memory). Then
//    each lane applies its row (MSGApply); the changed bits of a warp are
//    grouped per bitmap word with __match_any_sync and ORed in with one
//    atomic per word.
//  * hub part: up to kHubPartEdges in-edges of one high-in-degree row,
//    reduced lane-strided in registers and by a fixed warp tree; the last part
//    of a row to arrive combines all parts in part order and applies.
//
// Sums run in a fixed order, so fp32 PageRank is deterministic; PageRank's
// global sums (dangling mass, L1 delta) are exact 64-bit fixed point.
#include "frontier.cuh"
#include "grid_sync.cuh"

#include <algorithm>

#ifndef PR_ITEMS
#define PR_ITEMS 1
#endif

namespace gxp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kSellBlock = 256;
constexpr int kSellWarps = kSellBlock / 32;

template <Algo A> struct Ops;

// kMinBlocks: CTAs per SM the register budget is fitted to
template <> struct Ops<Algo::SSSP> {
    using T = uint32_t;
    static constexpr bool kWeighted = true;
    static constexpr int kUnroll = 8;
    static constexpr int kMinBlocks = 6;
    static constexpr int kItems = 1;
    __device__ static T ident() { return kInf; }
    __device__ static T combine(T a, T b) { return min(a, b); }
    __device__ static T from_bits(uint32_t x) { return x; }
    __device__ static uint32_t to_bits(T x) { return x; }
    // MSGGen: relax; unreachable sources send nothing.
    __device__ static T gen(uint32_t du, uint32_t w) {
        if (du == kInf) return kInf;
        uint32_t s = du + w;
        if (s < du || s == kInf) s = kInf - 1u;   // saturate below INF
        return s;
    }
};

template <> struct Ops<Algo::CC> {
    using T = uint32_t;
    static constexpr bool kWeighted = false;
    static constexpr int kUnroll = 8;
    static constexpr int kMinBlocks = 6;
    static constexpr int kItems = 1;
    __device__ static T ident() { return kInf; }
    __device__ static T combine(T a, T b) { return min(a, b); }
    __device__ static T from_bits(uint32_t x) { return x; }
    __device__ static uint32_t to_bits(T x) { return x; }
    __device__ static T gen(uint32_t lu, uint32_t) { return lu; }
};

// PageRank: 12 gathers in flight per lane at 5 CTAs per SM (48 registers)
// measured 181 us per R-MAT 22 superstep against 197 us for 8 at 6 CTAs
// (same box); 16 at 5 or 4 CTAs, 20 at 4, 8 at 7, and a separate unroll of
// 16 for the hub parts were all slower.
#ifndef PR_UNROLL
#define PR_UNROLL 12
#endif
template <> struct Ops<Algo::PR> {
    using T = float;
    static constexpr bool kWeighted = false;
    static constexpr int kUnroll = PR_UNROLL;
    static constexpr int kMinBlocks = 5;
    static constexpr int kItems = PR_ITEMS;   // work items per warp
    __device__ static T ident() { return 0.0f; }
    __device__ static T combine(T a, T b) { return a + b; }
    __device__ static T from_bits(uint32_t x) { return __uint_as_float(x); }
    __device__ static uint32_t to_bits(T x) { return __float_as_uint(x); }
    // The message array already holds r[u] / outdeg(u) (written by Apply).
    __device__ static T gen(uint32_t cu, uint32_t) { return __uint_as_float(cu); }
};

// Loads of the edge stream (source ids, weights: each read once per
// superstep, evict-first) and of the gathered values (read-only path).
__device__ __forceinline__ uint32_t ld_stream(const uint32_t* p) { return __ldcs(p); }
__device__ __forceinline__ uint4 ld_stream4(const uint4* p) { return __ldcs(p); }
__device__ __forceinline__ uint32_t ld_value(const uint32_t* p) { return __ldg(p); }

__device__ __forceinline__ uint32_t arrive_acq_rel(uint32_t* ctr) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
    return old;
}

template <class Op>
__device__ __forceinline__ typename Op::T warp_all(typename Op::T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = Op::combine(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

// Exact warp sum of 64-bit values below 2^62 (the fixed-point sums and
// counts): three 27-bit limbs, each summed by one warp reduction.
__device__ __forceinline__ unsigned long long warp_sum_u62(unsigned long long x) {
    const uint32_t a0 = (uint32_t)(x & 0x7FFFFFFull), a1 = (uint32_t)((x >> 27) & 0x7FFFFFFull),
                   a2 = (uint32_t)(x >> 54);
    return (unsigned long long)__reduce_add_sync(kFull, a0) +
           ((unsigned long long)__reduce_add_sync(kFull, a1) << 27) +
           ((unsigned long long)__reduce_add_sync(kFull, a2) << 54);
}

// The value of local source u of partition P: an owned vertex, a cached
// copy, or (the padding id of empty slots) the identity slot. kOne: one
// partition, whose local ids are global ids and whose padding id is V.
template <bool kOne>
struct Source {
    const uint32_t* own;    // own_cur + v_begin
    const uint32_t* copy;   // ghost + ghost_base - n_own: copy(u) for u >= n_own
    uint32_t n_own;
    __device__ __forceinline__ Source(const uint32_t* own_cur, const uint32_t* ghost, const PartDev& P)
        : own(own_cur + P.v_begin), copy(ghost + P.ghost_base - (ptrdiff_t)P.n_own), n_own(P.n_own) {}
    __device__ __forceinline__ const uint32_t* at(uint32_t u) const {
        if constexpr (kOne) return own + u;
        else return u < n_own ? own + u : copy + u;
    }
};

// The gathered values. A kernel that runs one superstep reads them through
// the non-coherent path (nothing writes them during the launch); the
// persistent loop, which writes in superstep t what superstep t + 1 reads,
// uses coherent loads, ordered by its grid barrier.
template <bool kLoop>
__device__ __forceinline__ uint32_t vload(const uint32_t* p) {
    if constexpr (kLoop) return __ldca(p);
    else return ld_value(p);
}

// One CTA's share of superstep t over the sliced-ELL layout (see the top of
// the file): work block vb of n_vb. kOne: a single partition (no cached
// copies); kCheck: range-check every source id (gxp_config.check_bounds),
// setting kErrBounds instead of loading; kLoop: called by the persistent
// loop (k_sell_loop).
template <Algo A, bool kOne, bool kCheck, bool kLoop>
__device__ __forceinline__ void sell_cta(const SellArgs& a, const uint64_t t, const uint32_t vb, const uint32_t n_vb) {
    using Op = Ops<A>;
    using T = typename Op::T;
    constexpr int kU = Op::kUnroll;
    __shared__ unsigned long long s_acc[3];
    __shared__ uint32_t s_done;
    __shared__ uint32_t s_ftot[kSellWarps], s_fedges[kSellWarps];   // frontier items, out-edges per warp
    __shared__ unsigned long long s_fbase;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    // superstep t reads value buffer t & 1 and stat slot t, writes the others
    const uint32_t* const own_cur = a.own[t & 1];
    uint32_t* const own_nxt = a.own[(t + 1) & 1];
    const float* const rank_cur = a.rank[t & 1];
    float* const rank_nxt = a.rank[(t + 1) & 1];
    const StepStats* const stats_in = a.stats + t % kStatRing;
    StepStats* const stats_out = a.stats + (t + 1) % kStatRing;
    FrontierCfg fc = a.fc;
    fc.list_in = a.lists[t & 1];
    if (fc.list_out) fc.list_out = a.lists[(t + 1) & 1];
    if (vb == 0) {
        // zero the ring slot two supersteps ahead (never read or written by this one)
        unsigned long long* z = reinterpret_cast<unsigned long long*>(a.stats + (t + 2) % kStatRing);
        for (uint32_t i = tid; i < sizeof(StepStats) / 8; i += kSellBlock) z[i] = 0ull;
    }
    __shared__ bool s_quiet, s_list;
    if (tid == 0) {
        s_acc[0] = s_acc[1] = s_acc[2] = 0ull;
        s_done = 0u;
        s_quiet = false;
        s_list = true;
    }
    const bool gate = fc.list_out != nullptr && fc.list_max_changed != kAlwaysList;
    if (((a.early_exit && t > 0) || gate) && warp == 0) {
        // the vertices the previous superstep changed (this one's frontier)
        const unsigned long long c = warp_sum_u62(stats_in->changed[lane] + stats_in->changed[lane + 32]);
        if (lane == 0) {
            // min-label algorithms at a fixed point: nothing can change any more
            if (a.early_exit && t > 0 && c == 0ull) s_quiet = true;
            if (gate) {   // the same inputs, so the same choice, in every CTA
                const unsigned long long ne = stats_in->list_ne;
                const unsigned long long work = (ne >> 32) + (ne & 0xFFFFFFFFull);
                s_list = c <= fc.list_max_changed &&
                         work * (unsigned long long)fc.push_div <= (unsigned long long)kListSlack * fc.total_edges;
            }
        }
    }
    // PageRank base terms, from the exact dangling mass of the current ranks
    // (every warp forms them itself: no wait on another warp's loads)
    float base = 0.0f, base_src = 0.0f;
    if constexpr (A == Algo::PR) {
        const unsigned long long sd = warp_sum_u62(stats_in->dangling_fx[lane] + stats_in->dangling_fx[lane + 32]);
        pagerank_base(sd, a.damping, a.inv_n, a.ppr_source != kInf, &base, &base_src);
    }
    __syncthreads();
    if (s_quiet) return;   // same for every thread of the grid
    const float damping = a.damping;

    uint32_t n_changed = 0;
    unsigned long long l1 = 0ull, dang = 0ull;

    // MSGApply of local vertex v of partition P with merged message m
    auto apply = [&](const PartDev& P, uint32_t v, T m) -> bool {
        const uint32_t gid = P.v_begin + v;
        if constexpr (A == Algo::PR) {
            const float rn = fmaf(damping, m, gid == a.ppr_source ? base_src : base);
            const float ro = rank_cur[gid];
            const uint32_t od = a.outdeg[gid];
            rank_nxt[gid] = rn;
            const float c = od ? __fdiv_rn(rn, (float)od) : 0.0f;
            const uint32_t cb = __float_as_uint(c);
            own_nxt[gid] = cb;
            const unsigned long long fn = fx_of(rn), fo = fx_of(ro);
            l1 += fn > fo ? fn - fo : fo - fn;
            if (od == 0u) dang += fn;
            // message changes are tracked only when a bitmap is wanted (partitions)
            if constexpr (kOne) return false;
            else return a.changed_bits != nullptr && cb != own_cur[gid];
        } else {
            const uint32_t old = own_cur[gid];
            const uint32_t nw = min(old, (uint32_t)m);
            own_nxt[gid] = nw;
            return nw != old;
        }
    };
    // kCheck: a source id outside the partition's ids (and not its padding id)
    // is reported and replaced by the padding id
    auto checked = [&](const PartDev& P, uint32_t u) -> uint32_t {
        if constexpr (kCheck) {
            if (u >= P.n_own + P.n_ghost && u != P.pad_id) {
                atomicOr(a.err, kErrBounds);
                return P.pad_id;
            }
        }
        return u;
    };

    // a CTA takes kSellWarps * kItems consecutive work items, warp w the items
    // w, w + kSellWarps, ...: the heavy-first order still spreads over the warps
    constexpr int kItems = Op::kItems;
    const uint32_t gw0 = vb * (kSellWarps * kItems) + (uint32_t)warp;
    const uint32_t gw = gw0;
    bool f_has = false;   // pull direction with frontier lists: this lane's changed vertex
    uint32_t f_v = 0;
    bool pushed = false;
    if constexpr (A != Algo::PR) {
        if (push_chosen(fc, stats_in)) {   // same choice in every thread of the grid
            const uint32_t c = push_superstep<Op::kWeighted, !kLoop>(fc, a.out_ptr, a.out_dst, a.out_w, own_cur,
                                                                     own_nxt, a.ghost, a.n_vertices,
                                                                     kOne ? nullptr : a.changed_bits, stats_in,
                                                                     stats_out, gw, (uint64_t)n_vb * kSellWarps, lane);
            if (lane == 0) n_changed += c;
            pushed = true;
        } else if (!s_list && vb == 0 && tid == 0) {
            stats_out->unlisted = 1ull;   // the next superstep pulls
        }
    }
#pragma unroll 1
    for (int it = 0; it < kItems; ++it) {
    const uint32_t gw = gw0 + (uint32_t)it * kSellWarps;
    if (pushed) {
        // the frontier's out-edges were relaxed above
    } else if (gw < a.n_hubs) {
        // ============================================================ hub part
        const HubPart hp = a.hubs[gw];
        const PartDev P = a.parts[kOne ? 0 : hp.part];
        const Source<kOne> S(own_cur, a.ghost, P);
        const uint32_t* src = P.hsrc + hp.e0;
        const uint32_t* wts = P.hw + hp.e0;
        T acc = Op::ident();
        auto hbatch = [&](uint32_t j0, auto load) {   // in-edges [j0, j0 + 32 kU) of the part, lane-strided
            uint32_t u[kU], x[kU], wv[kU];
#pragma unroll
            for (int q = 0; q < kU; ++q) {
                const uint32_t j = j0 + (uint32_t)q * 32u + (uint32_t)lane;
                const bool in = j < hp.ne;
                u[q] = in ? ld_stream(src + j) : 0u;
                wv[q] = (Op::kWeighted && in) ? ld_stream(wts + j) : 0u;
            }
#pragma unroll
            for (int q = 0; q < kU; ++q)
                x[q] = j0 + (uint32_t)q * 32u + (uint32_t)lane < hp.ne ? load(S.at(checked(P, u[q])))
                                                                        : Op::to_bits(Op::ident());
#pragma unroll
            for (int q = 0; q < kU; ++q)
                if (j0 + (uint32_t)q * 32u + (uint32_t)lane < hp.ne) acc = Op::combine(acc, Op::gen(x[q], wv[q]));
        };
        for (uint32_t jb = 0; jb < hp.ne; jb += 32u * kU) hbatch(jb, [](const uint32_t* p) { return vload<kLoop>(p); });
        T total = warp_all<Op>(acc);
        bool do_apply = hp.nparts == 1u;
        if (!do_apply) {
            uint32_t last = 0;
            if (lane == 0) {
                __stcg(&a.hub_val[gw], Op::to_bits(total));
                last = arrive_acq_rel(&a.hub_arrive[hp.t0]) == hp.nparts - 1u ? 1u : 0u;
            }
            last = __shfl_sync(kFull, last, 0);
            if (last) {
                __threadfence();
                T tot = Op::ident();   // parts in a fixed order: lane-strided, then a fixed tree
                for (uint32_t q = (uint32_t)lane; q < hp.nparts; q += 32u)
                    tot = Op::combine(tot, Op::from_bits(__ldcg(&a.hub_val[hp.t0 + q])));
                total = warp_all<Op>(tot);
                if (lane == 0) a.hub_arrive[hp.t0] = 0u;   // ready for the next superstep
                do_apply = true;
            }
        }
        const bool ch = do_apply && lane == 0 && apply(P, hp.v, total);
        if (ch) {
            ++n_changed;
            if (!kOne && a.changed_bits) {
                const uint32_t g = P.v_begin + hp.v;
                atomicOr(&a.changed_bits[g >> 5], 1u << (g & 31u));
            }
        }
        if constexpr (A != Algo::PR) {
            if (ch && fc.list_out) {   // the vertex joins the next frontier
                f_has = true;
                f_v = P.v_begin + hp.v;
            }
        }
    } else if (gw - a.n_hubs < a.n_slices - a.n_zero) {
        // =============================================================== slice
        const SellSlice sl = a.slices[gw - a.n_hubs];
        const PartDev P = a.parts[kOne ? 0 : sl.part];
        const Source<kOne> S(own_cur, a.ghost, P);
        const uint32_t row = P.perm[sl.row0 + lane];
        // groups of 4 columns: lane l's 4 sources of group g are one 128-bit
        // load at group g's 512 bytes (the warp's load is contiguous)
        const uint4* col4 = reinterpret_cast<const uint4*>(P.sell_src + sl.off) + lane;
        const uint4* wcol4 = reinterpret_cast<const uint4*>(P.sell_w + sl.off) + lane;
        T acc = Op::ident();
        static_assert(kU % 4 == 0, "a batch is whole groups of 4 columns");
        auto batch = [&](uint32_t k0, uint32_t ncols) {   // columns [k0, k0 + ncols), k0 % kU == 0
            uint32_t u[kU], x[kU], wv[kU];
            if constexpr (!kOne) {   // several partitions: column by column, 128-byte warp loads
                const uint32_t* col = P.sell_src + sl.off + lane;
                const uint32_t* wcol = P.sell_w + sl.off + lane;
#pragma unroll
                for (int q = 0; q < kU; ++q) {
                    const bool in = (uint32_t)q < ncols;
                    u[q] = in ? ld_stream(col + 32u * (k0 + q)) : 0u;
                    wv[q] = (Op::kWeighted && in) ? ld_stream(wcol + 32u * (k0 + q)) : 0u;
                }
            } else {   // one partition: groups of 4 columns, a 128-bit load per lane and group
#pragma unroll
                for (int h = 0; h < kU / 4; ++h) {
                    const bool in = 4u * h < ncols;   // a group holding at least one column
                    const uint4 s4 = in ? ld_stream4(col4 + 32u * (k0 / 4u + h)) : make_uint4(0u, 0u, 0u, 0u);
                    u[4 * h] = s4.x;
                    u[4 * h + 1] = s4.y;
                    u[4 * h + 2] = s4.z;
                    u[4 * h + 3] = s4.w;
                    if constexpr (Op::kWeighted) {
                        const uint4 w4 = in ? ld_stream4(wcol4 + 32u * (k0 / 4u + h)) : make_uint4(0u, 0u, 0u, 0u);
                        wv[4 * h] = w4.x;
                        wv[4 * h + 1] = w4.y;
                        wv[4 * h + 2] = w4.z;
                        wv[4 * h + 3] = w4.w;
                    } else {
                        wv[4 * h] = wv[4 * h + 1] = wv[4 * h + 2] = wv[4 * h + 3] = 0u;
                    }
                }
            }
#pragma unroll
            for (int q = 0; q < kU; ++q)
                x[q] = (uint32_t)q < ncols ? vload<kLoop>(S.at(checked(P, u[q]))) : Op::to_bits(Op::ident());
#pragma unroll
            for (int q = 0; q < kU; ++q)
                if ((uint32_t)q < ncols) acc = Op::combine(acc, Op::gen(x[q], wv[q]));
        };
        // whole batches of kU columns (kU gathers in flight per lane), then the rest
        const uint32_t full = sl.width - sl.width % kU;
        uint32_t kb = 0;
        for (; kb < full; kb += kU) batch(kb, kU);
        if (kb < sl.width) batch(kb, sl.width - kb);
        const bool ch = row != kSellPad && apply(P, row, acc);
        const unsigned chm = __ballot_sync(kFull, ch);
        if (lane == 0) n_changed += __popc(chm);
        if constexpr (A != Algo::PR) {
            if (ch && fc.list_out) {
                f_has = true;
                f_v = P.v_begin + row;
            }
        }
        if (!kOne && ch && a.changed_bits) {
            // one atomic per bitmap word touched by this warp
            const uint32_t g = P.v_begin + row;
            const unsigned grp = __match_any_sync(chm, g >> 5);
            const unsigned bits = __reduce_or_sync(grp, 1u << (g & 31u));
            if ((uint32_t)lane == (uint32_t)(__ffs(grp) - 1)) atomicOr(&a.changed_bits[g >> 5], bits);
        }
    } else {
        if constexpr (A == Algo::PR && kOne) {
            // ============================================ rows without in-edges
            // kZeroGroup slices of rows whose merged message is the identity:
            // the new rank is the base term (as MSGApply gives for m = 0). All
            // of the group's loads are issued before any store, so their
            // latencies overlap instead of forming one chain per slice.
            const uint32_t zg = gw - a.n_hubs - (a.n_slices - a.n_zero);
            if (zg < (a.n_zero + kZeroGroup - 1) / kZeroGroup) {
                const uint32_t* perm = a.parts[0].perm;
                const uint32_t s0 = a.n_slices - a.n_zero + zg * kZeroGroup;
                uint32_t v[kZeroGroup], od[kZeroGroup];
                float ro[kZeroGroup];
#pragma unroll
                for (int j = 0; j < (int)kZeroGroup; ++j)
                    v[j] = s0 + j < a.n_slices ? __ldg(perm + __ldg(&a.slices[s0 + j].row0) + lane) : kSellPad;
#pragma unroll
                for (int j = 0; j < (int)kZeroGroup; ++j) {
                    const bool has = v[j] != kSellPad;
                    ro[j] = has ? __ldg(rank_cur + v[j]) : 0.0f;
                    od[j] = has ? __ldg(a.outdeg + v[j]) : 0u;
                }
#pragma unroll
                for (int j = 0; j < (int)kZeroGroup; ++j) {
                    if (v[j] == kSellPad) continue;
                    const float rn = v[j] == a.ppr_source ? base_src : base;
                    rank_nxt[v[j]] = rn;
                    own_nxt[v[j]] = __float_as_uint(od[j] ? __fdiv_rn(rn, (float)od[j]) : 0.0f);
                    const unsigned long long fn = fx_of(rn), fo = fx_of(ro[j]);
                    l1 += fn > fo ? fn - fo : fo - fn;
                    if (od[j] == 0u) dang += fn;
                }
            }
        }
    }
    }   // work items

    if constexpr (A != Algo::PR) {
        if (fc.list_out && !pushed && s_list) {   // uniform over the grid
            // the changed vertices join the next frontier: one atomic per CTA
            // reserves the CTA's items, each warp writes its own; a vertex's
            // items cover the out-edges of its slot
            const uint32_t deg = f_has ? __ldg(a.out_ptr + f_v + 1) - __ldg(a.out_ptr + f_v) : 0u;
            const uint32_t nit = f_has ? frontier_items(deg) : 0u;
            const uint32_t incl = warp_inclusive_scan(nit, lane);
            const uint32_t edges = __reduce_add_sync(kFull, deg);
            if (lane == 31) {
                s_ftot[warp] = incl;
                s_fedges[warp] = edges;
            }
            __syncthreads();
            if (tid == 0) {
                uint32_t items = 0, e = 0;
                for (int w = 0; w < kSellWarps; ++w) {
                    const uint32_t t = s_ftot[w];
                    s_ftot[w] = items;   // -> the warp's offset in the CTA's range
                    items += t;
                    e += s_fedges[w];
                }
                s_fbase = items ? atomicAdd(&stats_out->list_ne, list_pack(items, e)) >> 32 : 0ull;
            }
            __syncthreads();
            if (__shfl_sync(kFull, incl, 31)) frontier_write(fc, s_fbase + s_ftot[warp], incl, nit, f_v, lane);
        }
    }

    // warp totals -> CTA totals in shared memory; the last warp flushes them
    const unsigned long long c64 = __reduce_add_sync(kFull, n_changed);
    if constexpr (A == Algo::PR) {
        l1 = warp_sum_u62(l1);
        dang = warp_sum_u62(dang);
    }
    if (lane == 0) {
        if (c64) atomicAdd(&s_acc[0], c64);
        if (l1) atomicAdd(&s_acc[1], l1);
        if (dang) atomicAdd(&s_acc[2], dang);
        __threadfence_block();
        if (atomicAdd(&s_done, 1u) == (uint32_t)kSellWarps - 1u) {
            __threadfence_block();
            const unsigned long long x0 = atomicAdd(&s_acc[0], 0ull), x1 = atomicAdd(&s_acc[1], 0ull),
                                     x2 = atomicAdd(&s_acc[2], 0ull);
            const uint32_t ln = vb % kStatLanes;
            if (x0) atomicAdd(&stats_out->changed[ln], x0);
            if (x1) atomicAdd(&stats_out->l1_fx[ln], x1);
            if (x2) atomicAdd(&stats_out->dangling_fx[ln], x2);
        }
    }
}

template <Algo A, bool kOne, bool kCheck>
__global__ void __launch_bounds__(kSellBlock, (A == Algo::SSSP && !kOne) ? 5 : Ops<A>::kMinBlocks)
    k_sell(const SellArgs a) {
    sell_cta<A, kOne, kCheck, false>(a, a.step_dev ? *a.step_dev : a.step, blockIdx.x, gridDim.x);
}

// Persistent form of a device-driven run (one partition, SSSP / CC, graphs
// whose superstep is a few waves of CTAs): one cooperative launch runs the
// supersteps from ctl->step until ctl->limit, or until the first superstep
// that changed nothing when ctl->quiet_stop. Each CTA takes the work blocks
// vb = blockIdx.x, blockIdx.x + gridDim.x, ... of a superstep (the blocks a
// one-superstep launch would run as CTAs), then all CTAs meet at a grid
// barrier: the Jacobi order of supersteps is the same as one launch per
// superstep, without a launch and a control kernel in between.
template <Algo A, bool kCheck>
__global__ void __launch_bounds__(kSellBlock, Ops<A>::kMinBlocks)
    k_sell_loop(const SellArgs a, RunCtl* ctl, GridBar* bar, uint32_t n_vb, uint64_t timeout_ns, uint32_t force) {
    __shared__ uint32_t s_more;
    uint64_t t = ctl->step;
    const uint64_t limit = ctl->limit;
    const uint32_t quiet_stop = ctl->quiet_stop;
    for (;;) {
        for (uint32_t vb = blockIdx.x; vb < n_vb; vb += gridDim.x) {
            sell_cta<A, true, kCheck, true>(a, t, vb, n_vb);
            __syncthreads();
        }
        if (!grid_barrier(bar, gridDim.x, timeout_ns, force != 0u, a.err)) return;
        ++t;   // supersteps done; slot t holds the last one's counts
        if (threadIdx.x < 32) {
            bool more = t < limit;
            if (more && quiet_stop) {
                const StepStats* st = a.stats + t % kStatRing;
                unsigned long long c = __ldcg(&st->changed[threadIdx.x]) + __ldcg(&st->changed[threadIdx.x + 32]);
#pragma unroll
                for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
                more = c != 0ull;
            }
            if (threadIdx.x == 0) s_more = more ? 1u : 0u;
        }
        __syncthreads();
        if (!s_more) {
            if (blockIdx.x == 0 && threadIdx.x == 0) ctl->step = t;
            return;
        }
    }
}

}  // namespace

namespace {

// Iteration control of a device-driven run (the body of a graph's WHILE
// node, after each superstep): advance the step, and continue while the
// step limit is not reached and, for the min-label algorithms, the superstep
// changed something. The limit alone ends the loop, whatever the supersteps
// compute.
__global__ void __launch_bounds__(32) k_run_control(RunCtl* ctl, const StepStats* ring,
                                                    cudaGraphConditionalHandle h) {
    const int lane = threadIdx.x;
    const uint64_t t = ctl->step + 1;   // supersteps done; slot t holds the last one's counts
    const StepStats& st = ring[t % kStatRing];
    unsigned long long c = st.changed[lane] + st.changed[lane + 32];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_xor_sync(kFull, c, o);
    if (lane == 0) {
        ctl->step = t;
        const bool more = t < ctl->limit && (ctl->quiet_stop == 0u || c != 0ull);
        cudaGraphSetConditional(h, more ? 1u : 0u);
    }
}

}  // namespace

cudaError_t launch_run_control(RunCtl* ctl, const StepStats* ring, cudaGraphConditionalHandle h, cudaStream_t s) {
    k_run_control<<<1, 32, 0, s>>>(ctl, ring, h);
    return cudaGetLastError();
}

template <Algo A>
static void launch_sell(const SellArgs& args, bool one, uint32_t grid, cudaStream_t s) {
    if (one) {
        if (args.check_bounds) k_sell<A, true, true><<<grid, kSellBlock, 0, s>>>(args);
        else k_sell<A, true, false><<<grid, kSellBlock, 0, s>>>(args);
    } else {
        if (args.check_bounds) k_sell<A, false, true><<<grid, kSellBlock, 0, s>>>(args);
        else k_sell<A, false, false><<<grid, kSellBlock, 0, s>>>(args);
    }
}

// Co-resident CTAs of k_sell_loop<A, kCheck> on the current device (queried
// on every call: the device, hence the SM count, may differ between calls).
template <Algo A, bool kCheck>
static cudaError_t loop_resident(uint64_t* resident) {
    int dev = 0, sms = 0, per_sm = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sell_loop<A, kCheck>, kSellBlock, 0);
    *resident = e == cudaSuccess ? (uint64_t)sms * (uint64_t)per_sm : 0;
    return e;
}

template <Algo A, bool kCheck>
static cudaError_t launch_loop_t(const SellArgs& args, RunCtl* ctl, GridBar* bar, uint32_t n_vb, uint64_t timeout_ns,
                                 uint32_t force, cudaStream_t s) {
    uint64_t resident = 0;
    const cudaError_t e = loop_resident<A, kCheck>(&resident);
    if (e != cudaSuccess) return e;
    if (resident == 0 || n_vb > kLoopWaves * resident) return cudaErrorNotSupported;
    const uint32_t grid = (uint32_t)std::min<uint64_t>(n_vb, resident);
    SellArgs a = args;
    void* params[] = {&a, &ctl, &bar, &n_vb, &timeout_ns, &force};
    return cudaLaunchCooperativeKernel((const void*)k_sell_loop<A, kCheck>, dim3(grid), dim3(kSellBlock), params, 0, s);
}

static uint32_t loop_blocks(const SellArgs& args) {
    const uint64_t work = (uint64_t)args.n_hubs + args.n_slices;
    return (uint32_t)std::max<uint64_t>(1, (work + kSellWarps - 1) / kSellWarps);
}

bool sell_loop_fits(Algo alg, const SellArgs& args) {
    if (args.n_parts != 1 || args.n_zero != 0 || args.early_exit || (alg != Algo::SSSP && alg != Algo::CC)) return false;
    uint64_t resident = 0;
    cudaError_t e;
    if (alg == Algo::SSSP) e = args.check_bounds ? loop_resident<Algo::SSSP, true>(&resident)
                                                 : loop_resident<Algo::SSSP, false>(&resident);
    else e = args.check_bounds ? loop_resident<Algo::CC, true>(&resident) : loop_resident<Algo::CC, false>(&resident);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return resident > 0 && loop_blocks(args) <= kLoopWaves * resident;
}

cudaError_t launch_sell_loop(Algo alg, const SellArgs& args, RunCtl* ctl, GridBar* bar, uint64_t timeout_ns,
                             bool force, cudaStream_t s) {
    if (args.n_parts != 1 || args.n_zero != 0 || args.early_exit) return cudaErrorInvalidValue;
    const uint32_t n_vb = loop_blocks(args);
    const uint32_t f = force ? 1u : 0u;
    switch (alg) {
        case Algo::SSSP:
            return args.check_bounds ? launch_loop_t<Algo::SSSP, true>(args, ctl, bar, n_vb, timeout_ns, f, s)
                                     : launch_loop_t<Algo::SSSP, false>(args, ctl, bar, n_vb, timeout_ns, f, s);
        case Algo::CC:
            return args.check_bounds ? launch_loop_t<Algo::CC, true>(args, ctl, bar, n_vb, timeout_ns, f, s)
                                     : launch_loop_t<Algo::CC, false>(args, ctl, bar, n_vb, timeout_ns, f, s);
        default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_superstep_sell(Algo alg, const SellArgs& args, cudaStream_t s) {
    if (args.n_zero > args.n_slices || (args.n_zero && (alg != Algo::PR || args.n_parts != 1)))
        return cudaErrorInvalidValue;
    const uint64_t work = (uint64_t)args.n_hubs + (args.n_slices - args.n_zero) +
                          (args.n_zero + kZeroGroup - 1) / kZeroGroup;
    // an empty layout still runs one block: it clears the stat slot two
    // supersteps ahead (and the step may live in device memory)
    const uint64_t per_cta = (uint64_t)kSellWarps * (alg == Algo::PR ? Ops<Algo::PR>::kItems : 1);
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, (work + per_cta - 1) / per_cta);
    const bool one = args.n_parts == 1;
    switch (alg) {
        case Algo::SSSP: launch_sell<Algo::SSSP>(args, one, grid, s); break;
        case Algo::CC: launch_sell<Algo::CC>(args, one, grid, s); break;
        case Algo::PR: launch_sell<Algo::PR>(args, one, grid, s); break;
        default: return cudaErrorInvalidValue;
    }
    return cudaGetLastError();
}

}  // namespace gxp
