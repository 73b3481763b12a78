// Fused superstep kernel: MSGGen + MSGMerge + MSGApply (Section IV-A1's
// algorithm template) over the dst-sorted edge blocks of Section II-B, run in
// pull form.
//
// Work unit: an edge block ("tile") = the in-edges [e0, e0+ne) of local
// destinations [v0, v0+nv) of one partition, cut on the merge path of
// (vertex ends, edges). Every warp is persistent over a contiguous range of
// tiles and owns a private ring of two shared-memory stages. For tile t+2 one
// lane issues cp.async.bulk copies of the tile's col_ptr slice (the
// vertex-edge mapping table), its source ids (+ weights) and the apply-side
// vertex slices (old value, or rank and out-degree), completing on the
// stage's mbarrier, while the warp computes tile t:
//   MSGGen   lanes read staged source ids lane-consecutively and gather the
//            sources' values with independent loads in flight; each message
//            overwrites its staged source id;
//   MSGMerge each lane reduces an equal merge-path share of the tile
//            sequentially, a 5-step warp segmented scan carries partial rows
//            across lanes, and a finished row's value overwrites the col_ptr
//            slot that row no longer needs;
//   MSGApply lanes take consecutive rows, reading old values from the stage,
//            writing coalesced, and __ballot_sync builds the changed bitmap.
// A row split across tiles (a hub, in-degree > hub_items) publishes one
// partial per tile; the last tile to arrive combines them in tile order.
// Every sum runs in a fixed order, so fp32 PageRank is deterministic; its
// global sums (dangling mass, L1 delta) are exact 64-bit fixed point.
#include <algorithm>

#include "gxp_internal.hpp"

namespace gxp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarps = kBlock / 32;
constexpr int kStages = 2;
constexpr uint64_t kDrainNs = 4000000000ull;   // smallest limit of the give-up drain (4 s)

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t* bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}"
        : "=r"(ok)
        : "r"(smem_addr(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// 1-D bulk copy global -> this CTA's shared memory, completing on `bar`.
// dst, src 16-byte aligned; bytes a multiple of 16.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}

__device__ __forceinline__ uint64_t global_ns() {
    uint64_t t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Wait for phase `parity` of `bar`, giving up after timeout_ns (and after a
// fixed iteration cap as a backstop). Returns false on give-up. With
// `give_up` set (the injected timeout fault) it gives up at once, whether or
// not the phase has completed.
__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t timeout_ns, bool give_up = false) {
    if (give_up) return false;
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31u) == 31u && global_ns() - t0 > timeout_ns) return false;
    }
    return false;
}

// acq_rel arrival: orders this thread's earlier writes before the count
// becomes visible, and makes earlier arrivals' writes visible to the last.
__device__ __forceinline__ uint32_t arrive_acq_rel(uint32_t* ctr) {
    uint32_t old;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(old) : "l"(ctr) : "memory");
    return old;
}

// ------------------------------------------------------ algorithm traits

template <Algo A> struct Traits;

template <> struct Traits<Algo::SSSP> {
    using T = uint32_t;
    static constexpr bool kWeighted = true;
    static constexpr bool kRank = false;
    static constexpr int kUnroll = 8;   // gathers in flight per lane
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

template <> struct Traits<Algo::CC> {
    using T = uint32_t;
    static constexpr bool kWeighted = false;
    static constexpr bool kRank = false;
    static constexpr int kUnroll = 16;
    __device__ static T ident() { return kInf; }
    __device__ static T combine(T a, T b) { return min(a, b); }
    __device__ static T from_bits(uint32_t x) { return x; }
    __device__ static uint32_t to_bits(T x) { return x; }
    __device__ static T gen(uint32_t lu, uint32_t) { return lu; }
};

template <> struct Traits<Algo::PR> {
    using T = float;
    static constexpr bool kWeighted = false;
    static constexpr bool kRank = true;
    static constexpr int kUnroll = 16;
    __device__ static T ident() { return 0.0f; }
    __device__ static T combine(T a, T b) { return a + b; }
    __device__ static T from_bits(uint32_t x) { return __uint_as_float(x); }
    __device__ static uint32_t to_bits(T x) { return __float_as_uint(x); }
    // The message array already holds r[u] / outdeg(u) (written by Apply).
    __device__ static T gen(uint32_t cu, uint32_t) { return __uint_as_float(cu); }
};

// Merge-path split of a tile: the merged sequence interleaves the tile's
// edges 0..ne-1 with its vertex ends 0..n_ends-1, vertex end r coming right
// after edge rowend(r)-1. Returns (r, j) = (vertex ends, edges) among the
// first d items.
__device__ __forceinline__ void merge_split(uint32_t d, uint32_t n_ends, uint32_t ne,
                                            const uint32_t* s_end, uint32_t e0, uint32_t& r,
                                            uint32_t& j) {
    uint32_t lo = d > ne ? d - ne : 0u;
    uint32_t hi = min(d, n_ends);
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (s_end[mid] - e0 <= d - mid - 1u) lo = mid + 1u;
        else hi = mid;
    }
    r = lo;
    j = d - lo;
}

template <class Tr>
__device__ __forceinline__ typename Tr::T warp_combine_all(typename Tr::T v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v = Tr::combine(v, __shfl_xor_sync(kFull, v, o));
    return v;
}

__device__ __forceinline__ uint32_t round4(uint32_t x) { return (x + 3u) & ~3u; }

// Stage geometry (words), from the largest tile: cost <= T + H + vertex cost.
struct Geometry {
    uint32_t vm, em, stage_words, warp_words;
};
__host__ __device__ inline Geometry geometry(Algo a, uint32_t max_items) {
    Geometry g;
    const uint32_t cost = max_items + kVertexCost;
    g.vm = ((cost / kVertexCost + 1u + 8u) + 3u) & ~3u;   // col_ptr slice / vertex slices
    g.em = ((cost + 8u) + 3u) & ~3u;                      // source ids (then messages), weights
    const uint32_t arrays_v = a == Algo::PR ? 3u : 2u;    // col + (rank, outdeg) | (old value)
    const uint32_t arrays_e = a == Algo::SSSP ? 2u : 1u;  // src (+ w)
    g.stage_words = arrays_v * g.vm + arrays_e * g.em;
    g.warp_words = kStages * g.stage_words;
    return g;
}

template <Algo A>
__global__ void __launch_bounds__(kBlock) k_superstep(const SuperstepArgs args) {
    using Tr = Traits<A>;
    using T = typename Tr::T;
    constexpr int kU = Tr::kUnroll;

    extern __shared__ __align__(128) uint32_t smem[];
    __shared__ uint64_t s_bar[kWarps][kStages];
    __shared__ Tile s_tile[kWarps][kStages];
    __shared__ unsigned long long s_acc[3];
    __shared__ uint32_t s_done;

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const uint32_t nwarps = blockDim.x >> 5;   // 1..kWarps, chosen at launch to fit shared memory
    const Geometry geo = geometry(A, args.max_items);
    uint32_t* wbase = reinterpret_cast<uint32_t*>((reinterpret_cast<uintptr_t>(smem) + 127u) & ~uintptr_t(127)) +
                      (uint32_t)warp * geo.warp_words;
    auto st_col = [&](int s) { return wbase + (uint32_t)s * geo.stage_words; };
    auto st_vx = [&](int s) { return wbase + (uint32_t)s * geo.stage_words + geo.vm; };   // old value | rank
    auto st_od = [&](int s) { return wbase + (uint32_t)s * geo.stage_words + 2u * geo.vm; };   // out-degree (PR)
    auto st_src = [&](int s) {
        return wbase + (uint32_t)s * geo.stage_words + (Tr::kRank ? 3u : 2u) * geo.vm;
    };
    auto st_w = [&](int s) { return st_src(s) + geo.em; };

    if (blockIdx.x == 0 && args.stats_clear != nullptr) {
        // zero the ring slot two supersteps ahead (never read or written by this one)
        unsigned long long* z = reinterpret_cast<unsigned long long*>(args.stats_clear);
        for (uint32_t i = tid; i < sizeof(StepStats) / 8; i += blockDim.x) z[i] = 0ull;
    }
    if (tid == 0) {
        s_acc[0] = s_acc[1] = s_acc[2] = 0ull;
        s_done = 0u;
    }
    if (lane == 0) {
        for (int s = 0; s < kStages; ++s) mbar_init(&s_bar[warp][s], 1u);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    float base = 0.0f;
    if constexpr (A == Algo::PR) {
        // base term (1-d)/N + d*D/N from the exact dangling-mass sum of the current ranks
        unsigned long long sd = args.stats_in->dangling_fx[lane] + args.stats_in->dangling_fx[lane + 32];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) sd += __shfl_xor_sync(kFull, sd, o);
        const double d = (double)args.damping;
        base = (float)((1.0 - d) * args.inv_n + d * fx_to_double(sd) * args.inv_n);
    }
    __syncthreads();   // barriers, s_acc, s_done initialised
    const float damping = args.damping;

    uint32_t n_changed = 0;
    unsigned long long l1 = 0ull, dang = 0ull;

    // this warp's contiguous range of tiles
    const uint64_t gw = (uint64_t)blockIdx.x * nwarps + (uint32_t)warp;
    const uint64_t n_warps = (uint64_t)gridDim.x * nwarps;
    const uint32_t t_begin = (uint32_t)(gw * args.n_tiles / n_warps);
    const uint32_t t_end = (uint32_t)((gw + 1) * args.n_tiles / n_warps);

    // tile descriptors, 32 at a time: lane l holds tile d_base + l
    uint32_t d_base = t_begin;
    Tile my_desc{};
    auto load_descs = [&](uint32_t b) {
        d_base = b;
        if (b + (uint32_t)lane < t_end) my_desc = args.tiles[b + lane];
    };
    load_descs(t_begin);
    auto desc_of = [&](uint32_t t) -> Tile {   // warp-uniform t
        if (t - d_base >= 32u) load_descs(t);
        const int src = (int)(t - d_base);
        Tile d;
        d.v0 = __shfl_sync(kFull, my_desc.v0, src);
        d.nv = __shfl_sync(kFull, my_desc.nv, src);
        d.e0 = __shfl_sync(kFull, my_desc.e0, src);
        d.ne = __shfl_sync(kFull, my_desc.ne, src);
        d.part = __shfl_sync(kFull, my_desc.part, src);
        d.flags = __shfl_sync(kFull, my_desc.flags, src);
        d.hub_t0 = __shfl_sync(kFull, my_desc.hub_t0, src);
        d.nparts = __shfl_sync(kFull, my_desc.nparts, src);
        return d;
    };
    // stage tile t into stage s (warp-uniform call; lane 0 issues the copies)
    auto issue = [&](uint32_t t, int s) {
        const Tile d = desc_of(t);
        if (lane == 0) {
            s_tile[warp][s] = d;
            const PartDev P = args.parts[d.part];
            const uint32_t g0 = P.v_begin + d.v0;
            const uint32_t c_lo = d.v0 & ~3u, c_hi = round4(d.v0 + d.nv + 1u);
            const uint32_t e_lo = d.e0 & ~3u, e_hi = round4(d.e0 + d.ne);
            const uint32_t g_lo = g0 & ~3u, g_hi = round4(g0 + d.nv);
            const uint32_t bc = (c_hi - c_lo) * 4u, be = (e_hi - e_lo) * 4u, bg = (g_hi - g_lo) * 4u;
            const uint32_t total = bc + be * (Tr::kWeighted ? 2u : 1u) + bg * (Tr::kRank ? 2u : 1u);
            asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
            mbar_arrive_expect_tx(&s_bar[warp][s], total);
            bulk_g2s(st_col(s), P.col_ptr + c_lo, bc, &s_bar[warp][s]);   // bc >= 16
            if (be) {
                bulk_g2s(st_src(s), P.src + e_lo, be, &s_bar[warp][s]);
                if (Tr::kWeighted) bulk_g2s(st_w(s), P.w + e_lo, be, &s_bar[warp][s]);
            }
            if (bg) {
                if constexpr (Tr::kRank) {
                    bulk_g2s(st_vx(s), args.rank_cur + g_lo, bg, &s_bar[warp][s]);
                    bulk_g2s(st_od(s), args.outdeg + g_lo, bg, &s_bar[warp][s]);
                } else {
                    bulk_g2s(st_vx(s), args.own_cur + g_lo, bg, &s_bar[warp][s]);
                }
            }
        }
    };

    for (int s = 0; s < kStages; ++s)
        if (t_begin + (uint32_t)s < t_end) issue(t_begin + (uint32_t)s, s);
    __syncwarp();

    uint32_t i = 0;
    for (uint32_t tix = t_begin; tix < t_end; ++tix, ++i) {
        const int s = (int)(i % kStages);
        const bool ok = mbar_wait_bounded(&s_bar[warp][s], (i / kStages) & 1u, args.timeout_ns,
                                          args.force_timeout != 0u);
        if (__any_sync(kFull, !ok)) {
            if (lane == 0) atomicOr(args.err, kErrTimeout);
            // Before leaving, every copy this warp has issued must land in its
            // shared memory: those of this tile's stage and of the stages
            // after it (tiles tix .. tix + kStages - 1). The drain has its own
            // limit, at least kDrainNs, independent of timeout_ns; a drain
            // that also runs out is recorded as kErrDrain.
            const uint64_t drain_ns = args.timeout_ns > kDrainNs ? args.timeout_ns : kDrainNs;
            for (uint32_t k = 0; k < (uint32_t)kStages && tix + k < t_end; ++k) {
                const bool landed =
                    mbar_wait_bounded(&s_bar[warp][(i + k) % kStages], ((i + k) / kStages) & 1u, drain_ns);
                if (!__all_sync(kFull, landed) && lane == 0) atomicOr(args.err, kErrDrain);
            }
            break;
        }
        const Tile tile = s_tile[warp][s];
        const PartDev P = args.parts[tile.part];
        const bool head_open = (tile.flags & kHeadOpen) != 0;
        const bool tail_open = (tile.flags & kTailOpen) != 0;
        const uint32_t nv = tile.nv, ne = tile.ne, e0 = tile.e0;
        const uint32_t n_ends = nv - (tail_open ? 1u : 0u);
        const uint32_t items = n_ends + ne;
        const uint32_t g0 = P.v_begin + tile.v0;
        uint32_t* s_col = st_col(s) + (tile.v0 & 3u);   // s_col[r] = col_ptr[v0 + r]
        const uint32_t* s_end = s_col + 1;
        uint32_t* s_msg = st_src(s) + (e0 & 3u);
        const uint32_t* s_w = st_w(s) + (e0 & 3u);
        const uint32_t* s_vx = st_vx(s) + (g0 & 3u);
        const uint32_t* s_od = st_od(s) + (g0 & 3u);

        // ---- MSGGen: messages overwrite the staged source ids
        {
            const uint32_t n_local = P.n_own + P.n_ghost;
            const uint32_t* own = args.own_cur + P.v_begin;
            const uint32_t* ghost = args.ghost + P.ghost_base;
            for (uint32_t jb = 0; jb < ne; jb += 32u * kU) {
                uint32_t x[kU];
                bool valid[kU];
#pragma unroll
                for (int q = 0; q < kU; ++q) {
                    const uint32_t j = jb + (uint32_t)q * 32u + (uint32_t)lane;
                    x[q] = 0u;
                    valid[q] = false;
                    if (j < ne) {
                        const uint32_t u = s_msg[j];
                        if (args.check_bounds && u >= n_local) {
                            atomicOr(args.err, kErrBounds);
                        } else {
                            x[q] = __ldg(u < P.n_own ? own + u : ghost + (u - P.n_own));
                            valid[q] = true;
                        }
                    }
                }
#pragma unroll
                for (int q = 0; q < kU; ++q) {
                    const uint32_t j = jb + (uint32_t)q * 32u + (uint32_t)lane;
                    if (j < ne)
                        s_msg[j] = Tr::to_bits(valid[q] ? Tr::gen(x[q], Tr::kWeighted ? s_w[j] : 0u) : Tr::ident());
                }
            }
        }
        __syncwarp();

        // ---- MSGMerge: per-lane merge-path walk over (vertex ends, edges)
        const uint32_t ipt = (items + 31u) / 32u;
        const uint32_t d0 = min((uint32_t)lane * ipt, items);
        const uint32_t cnt = min(d0 + ipt, items) - d0;
        uint32_t r0, j;
        merge_split(d0, n_ends, ne, s_end, e0, r0, j);
        __syncwarp();   // every lane has searched before row values overwrite s_end
        uint32_t r = r0;
        T acc = Tr::ident();
        T first = Tr::ident();
        bool have_first = false;
        for (uint32_t k = 0; k < cnt; ++k) {
            if (r < n_ends && s_end[r] - e0 <= j) {
                if (r == r0) {   // may continue from earlier lanes: written after the scan
                    first = acc;
                    have_first = true;
                } else {
                    s_col[r + 1] = Tr::to_bits(acc);   // no other lane reads slot r+1 any more
                }
                acc = Tr::ident();
                ++r;
            } else {
                acc = Tr::combine(acc, Tr::from_bits(s_msg[j]));
                ++j;
            }
        }
        // warp segmented inclusive scan of the carries (key = open row)
        const uint32_t key = r;
        T val = acc;
#pragma unroll
        for (int off = 1; off < 32; off <<= 1) {
            const uint32_t ku = __shfl_up_sync(kFull, key, off);
            const T vu = __shfl_up_sync(kFull, val, off);
            if (lane >= off && ku == key) val = Tr::combine(vu, val);
        }
        T prev = __shfl_up_sync(kFull, val, 1);
        const uint32_t kprev = __shfl_up_sync(kFull, key, 1);
        if (lane == 0 || kprev != r0) prev = Tr::ident();
        const T tail_part = __shfl_sync(kFull, val, 31);   // the open tail row's partial
        __syncwarp();   // the previous lane's last check of slot r0+1 is done
        if (have_first) s_col[r0 + 1] = Tr::to_bits(Tr::combine(prev, first));
        __syncwarp();

        // ---- MSGApply of row rr (staged old values) with merged message m
        auto apply = [&](uint32_t rr, T m) -> bool {
            const uint32_t gid = g0 + rr;
            if constexpr (A == Algo::PR) {
                const float rn = fmaf(damping, m, base);
                const float ro = __uint_as_float(s_vx[rr]);
                const uint32_t od = s_od[rr];
                args.rank_nxt[gid] = rn;
                const float c = od ? __fdiv_rn(rn, (float)od) : 0.0f;
                const uint32_t cb = __float_as_uint(c);
                args.own_nxt[gid] = cb;
                const unsigned long long fn = fx_of(rn), fo = fx_of(ro);
                l1 += fn > fo ? fn - fo : fo - fn;
                if (od == 0u) dang += fn;
                // message changes are tracked only when a bitmap is wanted (partitions)
                return args.changed_bits != nullptr && cb != args.own_cur[gid];
            } else {
                const uint32_t old = s_vx[rr];
                const uint32_t nw = min(old, (uint32_t)m);
                args.own_nxt[gid] = nw;
                return nw != old;
            }
        };

        // rows split across tiles: publish a partial; the last tile of the row
        // combines all partials in tile order (part 0 = the starting tile's tail)
        for (int pass = 0; pass < 2; ++pass) {
            uint32_t* slot;
            uint32_t t0, vrow;
            T part;
            if (pass == 0 && head_open) {
                slot = &args.part_head[tix];
                t0 = tile.hub_t0;
                vrow = 0u;
                part = (n_ends > 0u) ? Tr::from_bits(s_col[1]) : tail_part;   // n_ends 0: inside one row
            } else if (pass == 1 && tail_open && !(head_open && nv == 1u)) {
                slot = &args.part_tail[tix];
                t0 = tix;
                vrow = nv - 1u;
                part = tail_part;
            } else {
                continue;
            }
            uint32_t np = 0;
            if (lane == 0) {
                __stcg(slot, Tr::to_bits(part));
                const uint32_t n = __ldg(&args.tiles[t0].nparts);
                np = arrive_acq_rel(&args.hub_cnt[t0]) == n - 1u ? n : 0u;
            }
            np = __shfl_sync(kFull, np, 0);
            if (np) {
                __threadfence();
                T tot = Tr::ident();
                for (uint32_t q = (uint32_t)lane; q < np; q += 32u)
                    tot = Tr::combine(tot, Tr::from_bits(__ldcg(q == 0u ? &args.part_tail[t0] : &args.part_head[t0 + q])));
                tot = warp_combine_all<Tr>(tot);
                if (lane == 0) {
                    args.hub_cnt[t0] = 0u;   // ready for the next superstep
                    if (apply(vrow, tot)) {
                        ++n_changed;
                        if (args.changed_bits) atomicOr(&args.changed_bits[(g0 + vrow) >> 5], 1u << ((g0 + vrow) & 31u));
                    }
                }
            }
        }

        // complete rows, lanes on consecutive rows
        for (uint32_t rb = head_open ? 1u : 0u; rb < n_ends; rb += 32u) {
            const uint32_t rr = rb + (uint32_t)lane;
            const bool ch = rr < n_ends && apply(rr, Tr::from_bits(s_col[rr + 1]));
            const unsigned mask = __ballot_sync(kFull, ch);
            if (lane == 0 && mask) {
                n_changed += __popc(mask);
                if (args.changed_bits) {
                    const uint32_t g = g0 + rb;
                    const uint32_t wd = g >> 5, sh = g & 31u;
                    atomicOr(&args.changed_bits[wd], mask << sh);
                    if (sh && (mask >> (32u - sh))) atomicOr(&args.changed_bits[wd + 1u], mask >> (32u - sh));
                }
            }
        }
        __syncwarp();   // stage s is refilled next
        if (tix + kStages < t_end) issue(tix + kStages, s);
    }

    // warp totals -> CTA totals in shared memory; the last warp flushes them
    unsigned long long c64 = n_changed;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        c64 += __shfl_xor_sync(kFull, c64, o);
        if constexpr (A == Algo::PR) {
            l1 += __shfl_xor_sync(kFull, l1, o);
            dang += __shfl_xor_sync(kFull, dang, o);
        }
    }
    if (lane == 0) {
        if (c64) atomicAdd(&s_acc[0], c64);
        if (l1) atomicAdd(&s_acc[1], l1);
        if (dang) atomicAdd(&s_acc[2], dang);
        __threadfence_block();
        if (atomicAdd(&s_done, 1u) == nwarps - 1u) {
            __threadfence_block();
            const unsigned long long a = atomicAdd(&s_acc[0], 0ull), b = atomicAdd(&s_acc[1], 0ull),
                                     c = atomicAdd(&s_acc[2], 0ull);
            const uint32_t ln = blockIdx.x % kStatLanes;
            if (a) atomicAdd(&args.stats_out->changed[ln], a);
            if (b) atomicAdd(&args.stats_out->l1_fx[ln], b);
            if (c) atomicAdd(&args.stats_out->dangling_fx[ln], c);
        }
    }
}

}  // namespace

constexpr size_t kSmemLimit = 227 * 1024;

// Warps per CTA: as many (up to kWarps) as fit the per-warp stage footprint.
static uint32_t warps_per_cta(Algo a, uint32_t max_items) {
    const size_t per_warp = (size_t)geometry(a, max_items).warp_words * sizeof(uint32_t);
    const size_t static_bytes = 512;
    size_t nw = (kSmemLimit - 128 - static_bytes) / per_warp;
    return (uint32_t)std::min<size_t>(std::max<size_t>(nw, 0), kWarps);
}

size_t superstep_smem_bytes(Algo a, uint32_t max_items) {
    return (size_t)geometry(a, max_items).warp_words * warps_per_cta(a, max_items) * sizeof(uint32_t) + 128;
}

template <Algo A>
static cudaError_t launch_persistent(const SuperstepArgs& args, cudaStream_t s) {
    const uint32_t nw = warps_per_cta(A, args.max_items);
    if (nw == 0) return cudaErrorInvalidValue;   // a single warp's stages exceed shared memory
    const size_t smem = superstep_smem_bytes(A, args.max_items);
    cudaError_t e = cudaFuncSetAttribute(k_superstep<A>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    // SM count and occupancy of the current device, queried per launch (host
    // threads may drive different GPUs; the queries cost microseconds)
    int dev = 0, n_sm = 0, blocks = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&n_sm, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&blocks, k_superstep<A>, (int)(32 * nw), smem)) !=
        cudaSuccess)
        return e;
    const uint64_t blocks_max = (uint64_t)n_sm * (uint64_t)(blocks > 0 ? blocks : 1);
    const uint64_t blocks_needed = ((uint64_t)args.n_tiles + nw - 1) / nw;
    const uint32_t grid = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(blocks_max, blocks_needed));
    k_superstep<A><<<grid, 32 * nw, smem, s>>>(args);
    return cudaGetLastError();
}

cudaError_t launch_superstep(Algo a, const SuperstepArgs& args, size_t, cudaStream_t s) {
    if (args.n_tiles == 0) {
        // nothing to compute, but the stat slot two supersteps ahead must still be cleared
        if (args.stats_clear) return cudaMemsetAsync(args.stats_clear, 0, sizeof(StepStats), s);
        return cudaSuccess;
    }
    switch (a) {
        case Algo::SSSP: return launch_persistent<Algo::SSSP>(args, s);
        case Algo::CC: return launch_persistent<Algo::CC>(args, s);
        case Algo::PR: return launch_persistent<Algo::PR>(args, s);
    }
    return cudaErrorInvalidValue;
}

}  // namespace gxp
