// Fused superstep kernel: MSGGen + MSGMerge + MSGApply over one edge block
// (Section IV-A1's algorithm template, run in pull form over dst-sorted edge
// blocks, Section II-B).
//
// One CTA owns one block ("tile") of in-edges [e0, e0+ne) of local
// destinations [v0, v0+nv):
//   1. stage:  one thread issues cp.async.bulk copies of the tile's slice of
//              the vertex-edge mapping table (col_ptr), its source indices and
//              (SSSP) weights into shared memory, completing on an mbarrier;
//   2. MSGGen: each thread takes an equal share of the tile's merge items
//              (edges + vertex ends, a merge-path split), gathers the source
//              values of its edges and turns them into messages in registers;
//   3. MSGMerge: a thread-sequential segmented reduction over its items,
//              then a CTA-wide segmented scan of the per-thread carries
//              (warp shuffles + one cross-warp step) completes each vertex;
//   4. MSGApply: vertex-parallel apply with coalesced reads/writes of the
//              vertex arrays, changed-vertex bitmap via __ballot_sync and
//              exact fixed-point global sums (PageRank dangling mass, L1 delta).
// A hub vertex whose in-edges span several tiles leaves one partial per tile;
// the last tile to arrive (atomic counter) combines them in tile order, so
// fp32 sums are deterministic.
#include "gxp_internal.hpp"

namespace gxp {
namespace {

constexpr unsigned kFull = 0xFFFFFFFFu;
constexpr int kWarps = kBlock / 32;

// ------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t smem_addr(const void* p) {
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

__device__ __forceinline__ void mbar_init(uint64_t* bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count)
                 : "memory");
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t* bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)),
                 "r"(bytes)
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
// fixed iteration cap as a backstop). Returns false on give-up.
__device__ bool mbar_wait_bounded(uint64_t* bar, uint32_t parity, uint64_t timeout_ns) {
    if (mbar_try_wait(bar, parity)) return true;
    const uint64_t t0 = global_ns();
    for (uint32_t it = 0; it < (1u << 26); ++it) {
        if (mbar_try_wait(bar, parity)) return true;
        if ((it & 31u) == 31u && global_ns() - t0 > timeout_ns) return false;
    }
    return false;
}


// ------------------------------------------------------ algorithm traits

template <Algo A> struct Traits;

template <> struct Traits<Algo::SSSP> {
    using T = uint32_t;
    static constexpr bool kWeighted = true;
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
    __device__ static T shfl_up(T v, int off) { return __shfl_up_sync(kFull, v, off); }
};

template <> struct Traits<Algo::CC> {
    using T = uint32_t;
    static constexpr bool kWeighted = false;
    __device__ static T ident() { return kInf; }
    __device__ static T combine(T a, T b) { return min(a, b); }
    __device__ static T from_bits(uint32_t x) { return x; }
    __device__ static uint32_t to_bits(T x) { return x; }
    __device__ static T gen(uint32_t lu, uint32_t) { return lu; }
    __device__ static T shfl_up(T v, int off) { return __shfl_up_sync(kFull, v, off); }
};

template <> struct Traits<Algo::PR> {
    using T = float;
    static constexpr bool kWeighted = false;
    __device__ static T ident() { return 0.0f; }
    __device__ static T combine(T a, T b) { return a + b; }
    __device__ static T from_bits(uint32_t x) { return __uint_as_float(x); }
    __device__ static uint32_t to_bits(T x) { return __float_as_uint(x); }
    // The message array already holds r[u] / outdeg(u) (written by Apply).
    __device__ static T gen(uint32_t cu, uint32_t) { return __uint_as_float(cu); }
    __device__ static T shfl_up(T v, int off) { return __shfl_up_sync(kFull, v, off); }
};

__device__ __forceinline__ uint32_t round32(uint32_t x) { return (x + 31u) & ~31u; }

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

template <Algo A>
__global__ void __launch_bounds__(kBlock) k_superstep(const SuperstepArgs args) {
    using Tr = Traits<A>;
    using T = typename Tr::T;

    extern __shared__ __align__(128) uint32_t smem[];
    __shared__ uint64_t bar;
    __shared__ uint32_t w_key[kWarps];
    __shared__ T w_val[kWarps];
    __shared__ T s_tail;
    __shared__ float s_base;
    __shared__ unsigned long long s_red[3][kWarps];

    const uint32_t tix = blockIdx.x;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;

    if (blockIdx.x == 0 && args.stats_clear != nullptr) {
        // zero the ring slot two supersteps ahead (never read or written by this one)
        unsigned long long* z = reinterpret_cast<unsigned long long*>(args.stats_clear);
        for (uint32_t i = tid; i < sizeof(StepStats) / 8; i += kBlock) z[i] = 0ull;
    }

    const Tile tile = args.tiles[tix];
    if (tile.nv == 0 && tile.ne == 0) return;   // uniform over the CTA
    const PartDev P = args.parts[tile.part];

    const uint32_t M8 = round32(args.max_items + 8u);
    // bulk-copy destinations must be 16-byte aligned: align the region to 128
    uint32_t* s_col = reinterpret_cast<uint32_t*>((reinterpret_cast<uintptr_t>(smem) + 127u) & ~uintptr_t(127));
    uint32_t* s_src = s_col + M8;
    uint32_t* s_w = s_src + M8;
    T* s_sum = reinterpret_cast<T*>(s_w + (Tr::kWeighted ? M8 : 0u));

    // ---- 1. stage the tile (bulk copies into shared memory)
    const uint32_t c_lo = tile.v0 & ~3u;
    const uint32_t c_hi = (tile.v0 + tile.nv + 1u + 3u) & ~3u;
    const uint32_t e_lo = tile.e0 & ~3u;
    const uint32_t e_hi = (tile.e0 + tile.ne + 3u) & ~3u;
    const uint32_t col_off = tile.v0 - c_lo;
    const uint32_t src_off = tile.e0 - e_lo;
    if (tid == 0) mbar_init(&bar, 1u);
    __syncthreads();
    if (tid == 0) {
        const uint32_t bc = (c_hi - c_lo) * 4u, be = (e_hi - e_lo) * 4u;
        mbar_arrive_expect_tx(&bar, bc + be + (Tr::kWeighted ? be : 0u));
        bulk_g2s(s_col, P.col_ptr + c_lo, bc, &bar);  // bc >= 16 always (nv + 1 >= 1)
        if (be) {
            bulk_g2s(s_src, P.src + e_lo, be, &bar);
            if (Tr::kWeighted) bulk_g2s(s_w, P.w + e_lo, be, &bar);
        }
    }
    if constexpr (A == Algo::PR) {
        // base term (1-d)/N + d*D/N from the exact dangling-mass sum of the current ranks
        if (warp == 0) {
            unsigned long long s = args.stats_in->dangling_fx[lane] + args.stats_in->dangling_fx[lane + 32];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
            if (lane == 0) {
                const double D = fx_to_double(s);
                const double d = (double)args.damping;
                s_base = (float)((1.0 - d) * args.inv_n + d * D * args.inv_n);
            }
        }
    }
    const bool ok = mbar_wait_bounded(&bar, 0u, args.timeout_ns);
    if (__syncthreads_or(!ok)) {
        if (tid == 0) {
            atomicOr(args.err, kErrTimeout);
            mbar_wait_bounded(&bar, 0u, args.timeout_ns);   // let copies in flight land
        }
        return;
    }

    const bool head_open = (tile.flags & kHeadOpen) != 0;
    const bool tail_open = (tile.flags & kTailOpen) != 0;
    const uint32_t n_ends = tile.nv - (tail_open ? 1u : 0u);
    const uint32_t ne = tile.ne;
    const uint32_t items = n_ends + ne;
    const uint32_t ipt = (items + kBlock - 1u) / kBlock;
    const uint32_t* s_end = s_col + col_off + 1u;   // s_end[r] = col_ptr[v0 + r + 1]

    const uint32_t d0 = min((uint32_t)tid * ipt, items);
    const uint32_t d1 = min(d0 + ipt, items);
    uint32_t r0, j0, r1, j1;
    merge_split(d0, n_ends, ne, s_end, tile.e0, r0, j0);
    merge_split(d1, n_ends, ne, s_end, tile.e0, r1, j1);

    // ---- 2. MSGGen: messages of this thread's edges, in registers
    const uint32_t n_local = P.n_own + P.n_ghost;
    const uint32_t* own = args.own_cur + P.v_begin;
    T msg[kMaxIpt];
#pragma unroll
    for (int k = 0; k < kMaxIpt; ++k) {
        const uint32_t j = j0 + (uint32_t)k;
        msg[k] = Tr::ident();
        if (j < j1) {
            const uint32_t u = s_src[src_off + j];
            const uint32_t w = Tr::kWeighted ? s_w[src_off + j] : 0u;
            if (args.check_bounds && u >= n_local) {
                atomicOr(args.err, kErrBounds);
            } else {
                const uint32_t* px = u < P.n_own ? own + u : args.ghost + (P.ghost_base + (u - P.n_own));
                const uint32_t xu = __ldg(px);
                msg[k] = Tr::gen(xu, w);
            }
        }
    }

    // ---- 3. MSGMerge: thread-sequential segmented reduction over the split
    T acc = Tr::ident();
    uint32_t r = r0;
#pragma unroll
    for (int k = 0; k < kMaxIpt; ++k) {
        const uint32_t j = j0 + (uint32_t)k;
        if (j < j1) {
            while (r < r1 && s_end[r] - tile.e0 <= j) {
                s_sum[r] = acc;
                acc = Tr::ident();
                ++r;
            }
            acc = Tr::combine(acc, msg[k]);
        }
    }
    while (r < r1) {
        s_sum[r] = acc;
        acc = Tr::ident();
        ++r;
    }

    // CTA-wide segmented inclusive scan of the carries (key = open vertex).
    uint32_t key = r1;
    T val = acc;
#pragma unroll
    for (int off = 1; off < 32; off <<= 1) {
        const uint32_t ku = __shfl_up_sync(kFull, key, off);
        const T vu = Tr::shfl_up(val, off);
        if (lane >= off && ku == key) val = Tr::combine(vu, val);
    }
    if (lane == 31) {
        w_key[warp] = key;
        w_val[warp] = val;
    }
    __syncthreads();
    if (warp == 0) {
        uint32_t k2 = lane < kWarps ? w_key[lane] : kInf;
        T v2 = lane < kWarps ? w_val[lane] : Tr::ident();
#pragma unroll
        for (int off = 1; off < kWarps; off <<= 1) {
            const uint32_t ku = __shfl_up_sync(kFull, k2, off);
            const T vu = Tr::shfl_up(v2, off);
            if (lane >= off && ku == k2) v2 = Tr::combine(vu, v2);
        }
        if (lane < kWarps) w_val[lane] = v2;
    }
    __syncthreads();
    if (warp > 0 && key == w_key[warp - 1]) val = Tr::combine(w_val[warp - 1], val);
    // carry into this thread = inclusive value of the thread before it
    T prev = Tr::shfl_up(val, 1);
    uint32_t kprev = __shfl_up_sync(kFull, key, 1);
    if (lane == 0) {
        if (warp > 0) {
            prev = w_val[warp - 1];
            kprev = w_key[warp - 1];
        } else {
            prev = Tr::ident();
            kprev = kInf;
        }
    }
    if (r1 > r0 && kprev == r0) s_sum[r0] = Tr::combine(prev, s_sum[r0]);
    if (tid == kBlock - 1) s_tail = val;   // partial of the open tail vertex (key n_ends)
    __syncthreads();

    // ---- 4. MSGApply, vertex-parallel
    uint32_t n_changed = 0;
    unsigned long long l1 = 0ull, dang = 0ull;
    const float damping = args.damping;
    float base = 0.0f;
    if constexpr (A == Algo::PR) base = s_base;

    // vloc: partition-local vertex id
    auto apply = [&](uint32_t vloc, T m) -> bool {
        const uint32_t gid = P.v_begin + vloc;
        if constexpr (A == Algo::PR) {
            const float rn = fmaf(damping, m, base);
            const float ro = args.rank_cur[gid];
            args.rank_nxt[gid] = rn;
            const uint32_t od = args.outdeg[gid];
            const float c = od ? __fdiv_rn(rn, (float)od) : 0.0f;
            const uint32_t cb = __float_as_uint(c);
            args.own_nxt[gid] = cb;
            const unsigned long long fn = fx_of(rn), fo = fx_of(ro);
            l1 += fn > fo ? fn - fo : fo - fn;
            if (od == 0u) dang += fn;
            // message changes are tracked only when a bitmap is wanted (partitions)
            return args.changed_bits != nullptr && cb != args.own_cur[gid];
        } else {
            const uint32_t old = args.own_cur[gid];
            const uint32_t nw = min(old, (uint32_t)m);
            args.own_nxt[gid] = nw;
            return nw != old;
        }
    };

    // hub protocol: publish a partial; the last of the vertex's tiles combines
    // all partials in tile order and applies.
    auto hub_arrive = [&](uint32_t* slot, T part, uint32_t t0, T& total) -> bool {
        __stcg(slot, Tr::to_bits(part));
        __threadfence();
        const uint32_t np = __ldg(&args.tiles[t0].nparts);
        const uint32_t old = atomicAdd(&args.hub_cnt[t0], 1u);
        if (old != np - 1u) return false;
        __threadfence();
        T tot = Tr::from_bits(__ldcg(&args.part_tail[t0]));
        const uint32_t t_end = t0 + np;
        uint32_t tt = t0 + 1u;
        for (; tt + 8u <= t_end; tt += 8u) {
            uint32_t b[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) b[q] = __ldcg(&args.part_head[tt + q]);
#pragma unroll
            for (int q = 0; q < 8; ++q) tot = Tr::combine(tot, Tr::from_bits(b[q]));
        }
        for (; tt < t_end; ++tt) tot = Tr::combine(tot, Tr::from_bits(__ldcg(&args.part_head[tt])));
        args.hub_cnt[t0] = 0u;   // ready for the next superstep
        total = tot;
        return true;
    };

    const uint32_t nv = tile.nv;
    const uint32_t nv_round = (nv + 31u) & ~31u;
    for (uint32_t rr = (uint32_t)tid; rr < nv_round; rr += kBlock) {
        bool ch = false;
        if (rr < nv) {
            const bool is_head = head_open && rr == 0u;
            const bool is_tail = !is_head && tail_open && rr == nv - 1u;
            if (is_head) {
                T total;
                if (hub_arrive(&args.part_head[tix], n_ends ? s_sum[0] : s_tail, tile.hub_t0, total))
                    ch = apply(tile.v0 + rr, total);
            } else if (is_tail) {
                T total;
                if (hub_arrive(&args.part_tail[tix], s_tail, tix, total)) ch = apply(tile.v0 + rr, total);
            } else {
                ch = apply(tile.v0 + rr, s_sum[rr]);
            }
        }
        const unsigned mask = __ballot_sync(kFull, ch);
        if (lane == 0 && mask) {
            n_changed += __popc(mask);
            if (args.changed_bits) {
                const uint32_t g = P.v_begin + tile.v0 + rr;   // global id of lane 0's vertex
                const uint32_t wd = g >> 5, s = g & 31u;
                atomicOr(&args.changed_bits[wd], mask << s);
                if (s && (mask >> (32u - s))) atomicOr(&args.changed_bits[wd + 1u], mask >> (32u - s));
            }
        }
    }

    // CTA totals -> one atomic per statistic, on a lane chosen by the CTA index
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
        s_red[0][warp] = c64;
        s_red[1][warp] = l1;
        s_red[2][warp] = dang;
    }
    __syncthreads();
    if (tid == 0) {
        unsigned long long a = 0, b = 0, c = 0;
#pragma unroll
        for (int q = 0; q < kWarps; ++q) {
            a += s_red[0][q];
            b += s_red[1][q];
            c += s_red[2][q];
        }
        const uint32_t ln = tix % kStatLanes;
        if (a) atomicAdd(&args.stats_out->changed[ln], a);
        if (b) atomicAdd(&args.stats_out->l1_fx[ln], b);
        if (c) atomicAdd(&args.stats_out->dangling_fx[ln], c);
    }
}

}  // namespace

size_t superstep_smem_bytes(Algo a, uint32_t max_items) {
    const size_t m8 = (max_items + 8u + 31u) & ~31u;
    const size_t arrays = (a == Algo::SSSP) ? 4 : 3;
    return arrays * m8 * sizeof(uint32_t) + 128;   // + alignment slack
}

cudaError_t launch_superstep(Algo a, const SuperstepArgs& args, size_t smem, cudaStream_t s) {
    if (args.n_tiles == 0) return cudaSuccess;
    switch (a) {
        case Algo::SSSP:
            cudaFuncSetAttribute(k_superstep<Algo::SSSP>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_superstep<Algo::SSSP><<<args.n_tiles, kBlock, smem, s>>>(args);
            break;
        case Algo::CC:
            cudaFuncSetAttribute(k_superstep<Algo::CC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_superstep<Algo::CC><<<args.n_tiles, kBlock, smem, s>>>(args);
            break;
        case Algo::PR:
            cudaFuncSetAttribute(k_superstep<Algo::PR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            k_superstep<Algo::PR><<<args.n_tiles, kBlock, smem, s>>>(args);
            break;
    }
    return cudaGetLastError();
}

}  // namespace gxp
