// Host runtime of the superstep engine: graph loading (COO/CSC/CSR -> per
// partition dst-sorted CSC with local source ids), device residency, the
// superstep/sync/iteration control (Section II-C), and statistics.
#include "engine.hpp"
#include "trace.hpp"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>

namespace gxp {

void fail(gxp_status code, const std::string& msg) { throw Error{code, msg}; }

void cuda_check(cudaError_t e, const char* what) {
    if (e == cudaSuccess) return;
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();   // clear the non-sticky allocation error
        fail(GXP_E_NOMEM, std::string(what) + ": out of device memory");
    }
    fail(GXP_E_CUDA, std::string(what) + ": " + cudaGetErrorString(e));
}

namespace {

constexpr uint32_t kDefaultTile = 2048;   // edges per hub part; rows above tile/2 in-edges are hubs

inline size_t pad4(size_t n) { return ((n + 3) & ~size_t(3)) + 4; }

bool is_device_ptr(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

// ------------------------------------------------------------------ setup

Engine::Engine(int device, const gxp_config* cfg) : device_(device) {
    gxp_config_default(&cfg_);
    if (cfg) cfg_ = *cfg;
    auto_tiles_ = cfg_.tile_items == 0 && cfg_.hub_items == 0;
    if (cfg_.tile_items == 0) cfg_.tile_items = kDefaultTile;
    if (cfg_.hub_items == 0) cfg_.hub_items = cfg_.tile_items / 2;
    if (cfg_.timeout_ns == 0) cfg_.timeout_ns = 2000000000ull;
    if (cfg_.max_slots == 0) cfg_.max_slots = 64;
    if (cfg_.pipeline_depth == 0) cfg_.pipeline_depth = 3;
    if (cfg_.push_div == 0) cfg_.push_div = 8;
    faults_ = fault_plan(cfg_);
    if (cfg_.direction > GXP_DIR_PUSH) fail(GXP_E_INVAL, "direction must be GXP_DIR_AUTO, _PULL or _PUSH");
    if (cfg_.tile_items > (1u << 24) || cfg_.hub_items > (1u << 24))
        fail(GXP_E_INVAL, "tile_items and hub_items must not exceed 2^24");
    int n_dev = 0;
    cuda_check(cudaGetDeviceCount(&n_dev), "cudaGetDeviceCount");
    if (device < 0 || device >= n_dev) fail(GXP_E_INVAL, "no such CUDA device");
    cuda_check(cudaSetDevice(device), "cudaSetDevice");
    cuda_check(cudaStreamCreateWithFlags(&own_stream_, cudaStreamNonBlocking), "cudaStreamCreate");
    stream_ = own_stream_;
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cuda_check(cudaMemPoolCreate(&pool_, &props), "cudaMemPoolCreate");
    uint64_t keep = ~0ull;
    cuda_check(cudaMemPoolSetAttribute(pool_, cudaMemPoolAttrReleaseThreshold, &keep), "memory pool");
    cuda_check(cudaEventCreate(&ev_a_), "cudaEventCreate");
    cuda_check(cudaEventCreate(&ev_b_), "cudaEventCreate");
    cuda_check(cudaEventCreate(&ev_k_), "cudaEventCreate");
}

Engine::~Engine() {
    cudaSetDevice(device_);
    if (stream_) cudaStreamSynchronize(stream_);
    free_graph_device();
    for (auto& hp : parts_) release_part(hp);
    if (ev_a_) cudaEventDestroy(ev_a_);
    if (ev_b_) cudaEventDestroy(ev_b_);
    if (ev_k_) cudaEventDestroy(ev_k_);
    if (h_ctl_) cudaFreeHost(h_ctl_);
    if (h_ring_) cudaFreeHost(h_ring_);
    if (stream_) cudaStreamSynchronize(stream_);   // the frees above
    if (pool_) cudaMemPoolDestroy(pool_);
    if (own_stream_) cudaStreamDestroy(own_stream_);
}

// Device memory comes from the context's own memory pool, which keeps what
// is freed for reuse (release threshold: never), so reloading a graph of the
// same size maps no new pages: a first load pays cudaMalloc's page mapping,
// later ones take the pool's blocks at once. The allocation is made complete
// (the stream synchronized) before it returns, so any stream may use it, and
// frees are ordered after the context stream's work; every free happens once
// the buffer's users are done, as it did with cudaFree. When the pool cannot
// grow, it is trimmed and the allocation tried once more.
cudaError_t Engine::device_malloc(void** p, size_t bytes) {
    ++n_allocs_;
    if (faults_.alloc_at == n_allocs_) return cudaErrorMemoryAllocation;   // injected fault
    cudaError_t e = cudaMallocFromPoolAsync(p, bytes, pool_, stream_);
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        cudaStreamSynchronize(stream_);
        cudaMemPoolTrimTo(pool_, 0);
        e = cudaMallocFromPoolAsync(p, bytes, pool_, stream_);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(stream_);
    return e;
}

void Engine::device_free(void* p) {
    if (p) cudaFreeAsync(p, stream_);
}

void Engine::before_h2d(const char* what) {
    ++n_h2d_;
    if (faults_.h2d_at == n_h2d_)
        fail(GXP_E_CUDA, std::string(what) + ": host-to-device copy not enqueued (injected fault)");
}

void* Engine::dalloc(size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    if (cfg_.mem_budget && graph_bytes_ + bytes > cfg_.mem_budget)
        fail(GXP_E_NOMEM, "allocation exceeds the context's mem_budget");
    void* p = nullptr;
    cuda_check(device_malloc(&p, bytes), "cudaMalloc");
    graph_allocs_.push_back(p);
    graph_bytes_ += bytes;
    return p;
}

void Engine::free_graph_device() {
    if (stream_) cudaStreamSynchronize(stream_);
    free_batch();   // graphs and pinned buffers that refer to the device buffers below
    for (auto& g : run_graph_) {
        if (g) cudaGraphExecDestroy(g);
        g = nullptr;
    }
    d_ctl_ = nullptr;
    d_bar_ = nullptr;
    h_old2new_.clear();
    lp_ = LpLists{};
    lru_ = Lru{};
    for (void* p : graph_allocs_) device_free(p);
    graph_allocs_.clear();
    graph_bytes_ = 0;
    // every pointer into the buffers just freed (a later graph may not
    // allocate all of them again: one partition has no exchange buffers)
    d_parts_ = nullptr;
    d_slices_ = nullptr;
    d_hubs_ = nullptr;
    n_slices_ = n_hubs_ = n_zero_slices_ = 0;
    d_hub_val_ = d_hub_arrive_ = nullptr;
    d_outdeg_ = nullptr;
    d_own_[0] = d_own_[1] = nullptr;
    d_rank_[0] = d_rank_[1] = nullptr;
    d_ghost_ = d_ghost_gid_ = nullptr;
    d_changed_ = d_boundary_ = nullptr;
    d_gdq_ids_ = d_gdq_vals_ = nullptr;
    d_gdq_base_ = nullptr;
    d_block_counts_ = d_block_offsets_ = d_part_counts_ = nullptr;
    d_done_ctr_ = nullptr;
    d_stats_ = nullptr;
    d_err_ = nullptr;
    for (auto& hp : parts_)
        if (!hp.on_device) hp.d_col_ptr = hp.d_src = hp.d_w = nullptr;
    work_.clear();
    relabeled_ = false;
    d_new2old_ = d_old2new_ = d_perm_tmp_ = nullptr;
    out_ready_ = frontier_ = false;
    d_out_ptr_ = d_out_dst_ = d_out_w_ = nullptr;
    d_list_[0] = d_list_[1] = nullptr;
    finalized_ = false;
    sell_ready_ = false;
    begun_ = false;
}

void Engine::copy_in(void* dst, const void* src, size_t bytes) {
    if (bytes == 0) return;
    if (is_device_ptr(src)) cuda_check(cudaMemcpy(dst, src, bytes, cudaMemcpyDeviceToHost), "copy input");
    else std::memcpy(dst, src, bytes);
}

void Engine::check_device_error() {
    uint32_t err = 0;
    if (d_err_) cuda_check(cudaMemcpy(&err, d_err_, 4, cudaMemcpyDeviceToHost), "read error word");
    if (err & kErrTimeout) fail(GXP_E_TIMEOUT, "a device-side wait exceeded timeout_ns");
    if (err & kErrBounds) fail(GXP_E_BOUNDS, "a device-side bounds check failed");
    if (err & kErrInput) fail(GXP_E_BOUNDS, "a device-side check found CSC offsets out of order");
}

// ------------------------------------------------------------------ graph

void Engine::create_graph(uint64_t n, uint32_t n_parts, const uint64_t* part_begin) {
    if (n == 0 || n >= 0xFFFFFFFFull) fail(GXP_E_INVAL, "n_vertices must be in [1, 2^32 - 2]");
    if (n_parts == 0 || n_parts > 4096) fail(GXP_E_INVAL, "n_parts must be in [1, 4096]");
    std::vector<uint64_t> b(n_parts + 1);
    if (part_begin) {
        std::vector<uint64_t> tmp(n_parts + 1);
        copy_in(tmp.data(), part_begin, sizeof(uint64_t) * (n_parts + 1));
        b = tmp;
        if (b[0] != 0 || b[n_parts] != n) fail(GXP_E_INVAL, "part_begin must start at 0 and end at n_vertices");
        for (uint32_t p = 0; p < n_parts; ++p)
            if (b[p + 1] < b[p]) fail(GXP_E_INVAL, "part_begin must be non-decreasing");
    } else {
        for (uint32_t p = 0; p <= n_parts; ++p) b[p] = n * p / n_parts;
    }
    if (stream_) cudaStreamSynchronize(stream_);
    free_graph_device();
    for (auto& hp : parts_) release_part(hp);
    parts_.assign(n_parts, HostPart{});
    for (uint32_t p = 0; p < n_parts; ++p) {
        parts_[p].v_begin = (uint32_t)b[p];
        parts_[p].n_own = (uint32_t)(b[p + 1] - b[p]);
    }
    n_vertices_ = n;
    n_parts_ = n_parts;
    have_graph_ = true;
}

// Build a partition from its dst-sorted in-edge lists with global source ids.
static void build_local(HostPart& hp, uint64_t n_vertices, bool many_parts,
                        std::vector<uint32_t>&& col_ptr, std::vector<uint32_t>&& gsrc,
                        std::vector<uint32_t>&& w) {
    const uint32_t lo = hp.v_begin, hi = hp.v_begin + hp.n_own;
    hp.ghost_gid.clear();
    if (many_parts) {
        // cached remote sources: sorted unique ids outside [lo, hi)
        const size_t words = (n_vertices + 63) / 64;
        std::vector<uint64_t> mark(words, 0);
        for (uint32_t g : gsrc)
            if (g < lo || g >= hi) mark[g >> 6] |= 1ull << (g & 63);
        std::vector<uint32_t> rank(words + 1, 0);
        for (size_t i = 0; i < words; ++i) rank[i + 1] = rank[i] + (uint32_t)__builtin_popcountll(mark[i]);
        hp.ghost_gid.reserve(rank[words]);
        for (size_t i = 0; i < words; ++i) {
            uint64_t m = mark[i];
            while (m) {
                const int b = __builtin_ctzll(m);
                m &= m - 1;
                hp.ghost_gid.push_back((uint32_t)(i * 64 + b));
            }
        }
        for (uint32_t& g : gsrc) {
            if (g >= lo && g < hi) {
                g -= lo;
            } else {
                const uint64_t bits = mark[g >> 6] & ((1ull << (g & 63)) - 1ull);
                g = hp.n_own + rank[g >> 6] + (uint32_t)__builtin_popcountll(bits);
            }
        }
    } else {
        for (uint32_t& g : gsrc) g -= lo;   // lo == 0, every source is owned
    }
    hp.col_ptr = std::move(col_ptr);
    hp.src = std::move(gsrc);
    hp.w = std::move(w);
    hp.loaded = true;
}

void Engine::load_partition(uint32_t part, gxp_format fmt, uint64_t n_edges, const void* idx0,
                            const uint32_t* idx1, const uint32_t* weights) {
    TraceRange trace_("gxp load partition");
    if (!have_graph_) fail(GXP_E_STATE, "gxp_create_graph must come first");
    if (part >= n_parts_) fail(GXP_E_INVAL, "partition index out of range");
    if (n_edges > 0xFFFFFFFFull) fail(GXP_E_INVAL, "more than 2^32-1 edges in one partition");
    if (n_edges && (!idx0 || !idx1)) fail(GXP_E_INVAL, "null edge array");
    HostPart& hp = parts_[part];
    if (fmt == GXP_FMT_CSC && n_parts_ == 1) {   // straight to the device
        load_csc_device(hp, n_edges, idx0, idx1, weights);
        return;
    }
    const uint32_t lo = hp.v_begin, n_own = hp.n_own;
    const uint64_t V = n_vertices_;
    std::vector<uint32_t> col_ptr(n_own + 1, 0), gsrc(n_edges), w;
    if (weights) w.resize(n_edges);

    if (fmt == GXP_FMT_COO || fmt == GXP_FMT_CSR) {
        std::vector<uint32_t> src(n_edges), dst(n_edges), win;
        if (fmt == GXP_FMT_COO) {
            if (n_edges == 0 && idx0 == nullptr) {
            } else {
                copy_in(src.data(), idx0, 4 * n_edges);
            }
        } else {
            std::vector<uint64_t> row_ptr(V + 1);
            copy_in(row_ptr.data(), idx0, 8 * (V + 1));
            if (row_ptr[0] != 0 || row_ptr[V] != n_edges) fail(GXP_E_INVAL, "CSR row_ptr must run from 0 to n_edges");
            for (uint64_t u = 0; u < V; ++u) {
                if (row_ptr[u + 1] < row_ptr[u]) fail(GXP_E_INVAL, "CSR row_ptr not monotone");
                for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) src[e] = (uint32_t)u;
            }
        }
        if (n_edges) copy_in(dst.data(), idx1, 4 * n_edges);
        if (weights) {
            win.resize(n_edges);
            copy_in(win.data(), weights, 4 * n_edges);
        }
        for (uint64_t e = 0; e < n_edges; ++e) {
            if (src[e] >= V) fail(GXP_E_INVAL, "source id out of range");
            if (dst[e] < lo || dst[e] - lo >= n_own) fail(GXP_E_INVAL, "destination outside the partition");
            col_ptr[dst[e] - lo + 1]++;
        }
        for (uint32_t v = 0; v < n_own; ++v) col_ptr[v + 1] += col_ptr[v];
        std::vector<uint32_t> pos(col_ptr.begin(), col_ptr.end() - 1);
        for (uint64_t e = 0; e < n_edges; ++e) {   // stable counting sort by destination
            const uint32_t p = pos[dst[e] - lo]++;
            gsrc[p] = src[e];
            if (weights) w[p] = win[e];
        }
    } else if (fmt == GXP_FMT_CSC) {
        std::vector<uint64_t> cp(n_own + 1);
        copy_in(cp.data(), idx0, 8 * (size_t)(n_own + 1));
        if (cp[0] != 0 || cp[n_own] != n_edges) fail(GXP_E_INVAL, "CSC col_ptr must run from 0 to n_edges");
        for (uint32_t v = 0; v < n_own; ++v) {
            if (cp[v + 1] < cp[v]) fail(GXP_E_INVAL, "CSC col_ptr not monotone");
            col_ptr[v + 1] = (uint32_t)cp[v + 1];
        }
        if (n_edges) copy_in(gsrc.data(), idx1, 4 * n_edges);
        if (weights) copy_in(w.data(), weights, 4 * n_edges);
        for (uint64_t e = 0; e < n_edges; ++e)
            if (gsrc[e] >= V) fail(GXP_E_INVAL, "source id out of range");
    } else {
        fail(GXP_E_INVAL, "unknown format");
    }
    if (stream_) cudaStreamSynchronize(stream_);
    if (finalized_) free_graph_device();
    release_part(hp);
    build_local(hp, V, n_parts_ > 1, std::move(col_ptr), std::move(gsrc), std::move(w));
}

// Single-partition CSC: the arrays are copied into device memory as given
// (from host or device memory) and checked there; no host copy is made.
void Engine::load_csc_device(HostPart& hp, uint64_t E, const void* cp_in, const uint32_t* src_in,
                             const uint32_t* w_in) {
    if (!cp_in || (E && !src_in)) fail(GXP_E_INVAL, "null CSC array");
    if (stream_) cuda_check(cudaStreamSynchronize(stream_), "sync");
    if (finalized_) free_graph_device();
    release_part(hp);
    const uint32_t n = hp.n_own;
    auto own = [&](size_t bytes) {
        void* q = nullptr;
        if (cfg_.mem_budget && graph_bytes_ + bytes > cfg_.mem_budget)
            fail(GXP_E_NOMEM, "allocation exceeds the context's mem_budget");
        cuda_check(device_malloc(&q, std::max<size_t>(bytes, 16)), "cudaMalloc");
        return q;
    };
    uint64_t* cp64 = nullptr;
    uint32_t* flag = nullptr;
    try {
        hp.d_col_ptr = (uint32_t*)own(4 * pad4(n + 1));
        hp.d_src = (uint32_t*)own(4 * pad4(E));
        if (w_in) hp.d_w = (uint32_t*)own(4 * pad4(E));
        hp.on_device = true;
        cp64 = (uint64_t*)own(8 * ((size_t)n + 1));
        flag = (uint32_t*)own(4);
        cuda_check(cudaMemsetAsync(flag, 0, 4, stream_), "memset");
        cuda_check(cudaMemsetAsync(hp.d_col_ptr, 0, 4 * pad4(n + 1), stream_), "memset");
        cuda_check(cudaMemsetAsync(hp.d_src + E, 0, 4 * (pad4(E) - E), stream_), "memset");
        before_h2d("copy col_ptr");
        cuda_check(cudaMemcpyAsync(cp64, cp_in, 8 * ((size_t)n + 1), cudaMemcpyDefault, stream_), "copy col_ptr");
        if (E) {
            before_h2d("copy sources");
            cuda_check(cudaMemcpyAsync(hp.d_src, src_in, 4 * E, cudaMemcpyDefault, stream_), "copy sources");
        }
        if (w_in) {
            cuda_check(cudaMemsetAsync(hp.d_w + E, 0, 4 * (pad4(E) - E), stream_), "memset");
            if (E) {
                before_h2d("copy weights");
                cuda_check(cudaMemcpyAsync(hp.d_w, w_in, 4 * E, cudaMemcpyDefault, stream_), "copy weights");
            }
        }
        cuda_check(launch_csc_import(cp64, n, E, hp.d_col_ptr, hp.d_src, n, flag, stream_), "check CSC");
        uint32_t bad = 0;
        cuda_check(cudaMemcpyAsync(&bad, flag, 4, cudaMemcpyDeviceToHost, stream_), "read check");
        cuda_check(cudaStreamSynchronize(stream_), "check CSC");
        device_free(cp64);
        device_free(flag);
        cp64 = nullptr;
        flag = nullptr;
        if (bad & 1u) fail(GXP_E_INVAL, "CSC col_ptr must run from 0 to n_edges, non-decreasing");
        if (bad & 2u) fail(GXP_E_INVAL, "source id out of range");
    } catch (...) {
        if (cp64) device_free(cp64);
        if (flag) device_free(flag);
        release_part(hp);
        throw;
    }
    hp.dev_edges = E;
    hp.dev_weighted = w_in != nullptr;
    hp.loaded = true;
}

void Engine::release_part(HostPart& hp) {
    if (hp.on_device) {
        if (stream_) cudaStreamSynchronize(stream_);
        device_free(hp.d_col_ptr);
        device_free(hp.d_src);
        if (hp.d_w) device_free(hp.d_w);
        hp.d_col_ptr = hp.d_src = hp.d_w = nullptr;
        hp.on_device = false;
        hp.dev_edges = 0;
        hp.dev_weighted = false;
        hp.loaded = false;
    }
}

// Host copies of a device-loaded partition, for the paths that work on the host.
void Engine::ensure_host(HostPart& hp) {
    if (!hp.on_device || hp.col_ptr.size() == (size_t)hp.n_own + 1) return;
    const uint64_t E = hp.dev_edges;
    std::vector<uint32_t> cp(hp.n_own + 1), src(E), w(hp.dev_weighted ? E : 0);
    cuda_check(cudaMemcpy(cp.data(), hp.d_col_ptr, 4 * cp.size(), cudaMemcpyDeviceToHost), "download CSC");
    if (E) cuda_check(cudaMemcpy(src.data(), hp.d_src, 4 * E, cudaMemcpyDeviceToHost), "download CSC");
    if (hp.dev_weighted && E) cuda_check(cudaMemcpy(w.data(), hp.d_w, 4 * E, cudaMemcpyDeviceToHost), "download CSC");
    hp.col_ptr = std::move(cp);
    hp.src = std::move(src);
    hp.w = std::move(w);
}

uint32_t* Engine::upload_u32(const std::vector<uint32_t>& h, size_t n_pad) {
    uint32_t* d = (uint32_t*)dalloc(4 * std::max<size_t>(n_pad, 1));
    cuda_check(cudaMemsetAsync(d, 0, 4 * std::max<size_t>(n_pad, 1), stream_), "memset");
    if (!h.empty()) {
        before_h2d("upload");
        cuda_check(cudaMemcpyAsync(d, h.data(), 4 * h.size(), cudaMemcpyHostToDevice, stream_), "upload");
    }
    cuda_check(cudaStreamSynchronize(stream_), "upload");   // the staging vector may die after this
    return d;
}

// Sliced-ELL layout of the rows with at most H in-edges (SELL-32-sigma: rows
// sorted by in-degree within windows of kSellWindow rows, grouped in 32-row
// slices stored column-major, each row's in-edges in ascending source order)
// and hub parts of T edges for the rows with more. Built on first use by a
// superstep (the batched path does not need it).
// Sliced-ELL layout of every partition, built on the device (sell_build.cu):
// rows sorted by source, windows sorted by in-degree, slices filled, hub rows
// split into parts; then all slices ordered heavy-first. A few small counts
// come back to the host to size the arrays.
void Engine::build_sell() {
    TraceRange trace_("gxp layout build");
    uint32_t T = cfg_.tile_items, H = cfg_.hub_items;
    if (auto_tiles_) {
        // by default the longest work item shrinks with the graph: a slice row
        // of up to H in-edges and a hub part of T edges stay short next to the
        // average work per warp (H = 1024 / T = 2048 from ~64 M edges up)
        uint64_t h = std::max<uint64_t>(32, total_edges_ >> 16);
        uint64_t p2 = 32;
        while (p2 * 2 <= h) p2 *= 2;
        H = (uint32_t)std::min<uint64_t>(1024, p2);
        T = std::min<uint32_t>(2048, std::max<uint32_t>(256, 2 * H));
    }
    std::vector<void*> tmp;   // freed when the build ends
    auto talloc = [&](size_t bytes) {
        void* q = nullptr;
        cuda_check(device_malloc(&q, std::max<size_t>(bytes, 16)), "cudaMalloc");
        tmp.push_back(q);
        return q;
    };
    struct FreeTmp {
        std::vector<void*>& v;
        cudaStream_t s;
        ~FreeTmp() {
            cudaStreamSynchronize(s);
            for (void* q : v) cudaFreeAsync(q, s);   // pool blocks (device_malloc)
        }
    } free_tmp{tmp, stream_};
    auto d2h = [&](void* h, const void* d, size_t bytes) {
        cuda_check(cudaMemcpyAsync(h, d, bytes, cudaMemcpyDeviceToHost, stream_), "read counts");
        cuda_check(cudaStreamSynchronize(stream_), "read counts");
    };
    std::vector<SellSlice*> part_desc(n_parts_);
    std::vector<uint32_t> part_ns(n_parts_);
    std::vector<HubPart*> part_hubs(n_parts_);
    std::vector<uint32_t> part_nh(n_parts_);
    uint64_t total_slices = 0;
    uint32_t total_hubs = 0;
    for (uint32_t p = 0; p < n_parts_; ++p) {
        HostPart& hp = parts_[p];
        const bool weighted = hp.weighted();
        const uint32_t n = hp.n_own;
        const uint64_t E = hp.n_edges();
        // 1. rows sorted by (source, weight); the sorted copy also serves the hub parts
        const uint32_t* col_ptr = work_[p].col;   // offsets of the rows the build writes
        uint32_t* ssrc = (uint32_t*)dalloc(4 * pad4(E));
        uint32_t* sw = weighted ? (uint32_t*)dalloc(4 * pad4(E)) : nullptr;
        uint2* big = (uint2*)talloc(8 * ((size_t)n + E / 2048 + 1));
        uint32_t* cnt = (uint32_t*)talloc(4);
        cuda_check(launch_sort_rows(col_ptr, n, work_[p].in, pd_[p].n_own + pd_[p].n_ghost, ssrc, sw, big, cnt,
                                    stream_),
                   "sort rows");
        // 2. windows
        const uint32_t nw = (n + kSellWindow - 1) / kSellWindow;
        uint32_t* rows_out = (uint32_t*)talloc(4 * (size_t)n);
        uint32_t* hub_out = (uint32_t*)talloc(4 * (size_t)n);
        uint32_t* counts = (uint32_t*)talloc(8 * (size_t)nw + 8);   // non-hub counts, then hub counts
        cuda_check(launch_sell_windows(col_ptr, n, H, rows_out, hub_out, counts, counts + nw, stream_),
                   "sort windows");
        std::vector<uint32_t> hc(2 * (size_t)nw + 2, 0);
        if (nw) d2h(hc.data(), counts, 8 * (size_t)nw);
        std::vector<uint32_t> bases(2 * (size_t)nw + 2, 0);   // slice bases, then hub bases
        uint64_t ns = 0, nh_rows = 0;
        for (uint32_t w = 0; w < nw; ++w) {
            bases[w] = (uint32_t)ns;
            bases[nw + w] = (uint32_t)nh_rows;
            ns += (hc[w] + 31) / 32;
            nh_rows += hc[nw + w];
        }
        if (ns * 32 > 0xFFFFFFF0ull) fail(GXP_E_INVAL, "too many rows in one partition");
        uint32_t* d_bases = (uint32_t*)talloc(8 * (size_t)nw + 8);
        if (nw) {
            before_h2d("upload bases");
            cuda_check(cudaMemcpyAsync(d_bases, bases.data(), 8 * (size_t)nw, cudaMemcpyHostToDevice, stream_),
                       "upload bases");
        }
        // 3. slices and their offsets
        uint32_t* perm = (uint32_t*)dalloc(4 * pad4(ns * 32));
        uint32_t* width = (uint32_t*)talloc(4 * ns + 4);
        uint64_t* off = (uint64_t*)talloc(8 * ns + 8);
        cuda_check(launch_sell_slices(col_ptr, n, rows_out, counts, d_bases, perm, width, off, (uint32_t)ns,
                                      n_parts_ == 1, stream_), "slices");
        uint64_t sell_size = 0;
        d2h(&sell_size, off + ns, 8);
        // 4. fill
        uint32_t* sell_src = (uint32_t*)dalloc(4 * pad4(sell_size));
        uint32_t* sell_w = weighted ? (uint32_t*)dalloc(4 * pad4(sell_size)) : nullptr;
        part_desc[p] = (SellSlice*)talloc(sizeof(SellSlice) * (ns + 1));
        part_ns[p] = (uint32_t)ns;
        cuda_check(launch_sell_fill(col_ptr, ssrc, sw, perm, width, off, (uint32_t)ns, p, pd_[p].pad_id,
                                    n_parts_ == 1, sell_src, sell_w, part_desc[p], stream_), "fill slices");
        // 5. hub rows -> parts of T edges
        uint32_t* hub_list = (uint32_t*)talloc(4 * nh_rows + 4);
        uint32_t* part_off = (uint32_t*)talloc(4 * nh_rows + 4);
        cuda_check(launch_hub_rows(col_ptr, n, hub_out, counts + nw, d_bases + nw, hub_list, (uint32_t)nh_rows,
                                   T, part_off, stream_), "hub rows");
        uint32_t nparts = 0;
        d2h(&nparts, part_off + nh_rows, 4);
        if ((uint64_t)total_hubs + nparts > 0xFFFFFFF0ull) fail(GXP_E_INVAL, "too many hub parts");
        part_hubs[p] = (HubPart*)talloc(sizeof(HubPart) * ((size_t)nparts + 1));
        part_nh[p] = nparts;
        cuda_check(launch_hub_parts(col_ptr, hub_list, part_off, (uint32_t)nh_rows, T, p, total_hubs,
                                    part_hubs[p], stream_), "hub parts");
        pd_[p].sell_src = sell_src;
        pd_[p].sell_w = sell_w;
        pd_[p].perm = perm;
        pd_[p].hsrc = ssrc;
        pd_[p].hw = sw;
        total_slices += ns;
        total_hubs += nparts;
    }
    if (total_slices > 0xFFFFFFF0ull) fail(GXP_E_INVAL, "graph too large");
    n_slices_ = (uint32_t)total_slices;
    n_hubs_ = total_hubs;
    before_h2d("upload");
    cuda_check(cudaMemcpyAsync(d_parts_, pd_.data(), sizeof(PartDev) * n_parts_, cudaMemcpyHostToDevice, stream_),
               "upload parts");
    // 6. the partitions' slices, heavy first; hub parts concatenated (t0 already global)
    SellSlice* all = (SellSlice*)talloc(sizeof(SellSlice) * (total_slices + 1));
    uint64_t at = 0;
    for (uint32_t p = 0; p < n_parts_; ++p) {
        if (part_ns[p])
            cuda_check(cudaMemcpyAsync(all + at, part_desc[p], sizeof(SellSlice) * part_ns[p],
                                       cudaMemcpyDeviceToDevice, stream_), "gather slices");
        at += part_ns[p];
    }
    // Heavy first within each partition, partitions one after the other: the
    // grid then works through one partition's rows at a time, so the values
    // it gathers at any moment are that partition's own vertices and cached
    // copies (tens of MB, L2-resident) rather than every partition's copies
    // at once.
    d_slices_ = (SellSlice*)dalloc(sizeof(SellSlice) * std::max<size_t>(total_slices, 1));
    uint32_t* order_scratch = (uint32_t*)talloc(order_slices_scratch_bytes(n_slices_));
    at = 0;
    n_zero_slices_ = 0;
    for (uint32_t p = 0; p < n_parts_; ++p) {
        if (part_ns[p])
            cuda_check(launch_order_slices(all + at, part_ns[p], d_slices_ + at, order_scratch, stream_),
                       "order slices");
        if (n_parts_ == 1 && part_ns[p]) {
            // width 0 sorts last: the order's first offset of that bin counts the other slices
            uint32_t nonzero = 0;
            d2h(&nonzero, order_scratch, 4);
            if (nonzero <= part_ns[p]) n_zero_slices_ = part_ns[p] - nonzero;
        }
        at += part_ns[p];
    }
    const size_t nh1 = std::max<size_t>(total_hubs, 1);
    d_hubs_ = (HubPart*)dalloc(sizeof(HubPart) * nh1);
    at = 0;
    for (uint32_t p = 0; p < n_parts_; ++p) {
        if (part_nh[p])
            cuda_check(cudaMemcpyAsync(d_hubs_ + at, part_hubs[p], sizeof(HubPart) * part_nh[p],
                                       cudaMemcpyDeviceToDevice, stream_), "gather hub parts");
        at += part_nh[p];
    }
    d_hub_val_ = (uint32_t*)dalloc(4 * nh1);
    d_hub_arrive_ = (uint32_t*)dalloc(4 * nh1);
    cuda_check(cudaMemsetAsync(d_hub_arrive_, 0, 4 * nh1, stream_), "memset");
    cuda_check(cudaStreamSynchronize(stream_), "sell build");
    check_device_error();
    sell_ready_ = true;
}

// Upload every partition, count out-degrees, build caches.
void Engine::finalize() {
    TraceRange trace_("gxp finalize");
    for (uint32_t p = 0; p < n_parts_; ++p)
        if (!parts_[p].loaded) fail(GXP_E_STATE, "partition " + std::to_string(p) + " not loaded");
    cuda_check(cudaStreamSynchronize(stream_), "sync");
    free_graph_device();
    const uint32_t V = (uint32_t)n_vertices_;

    n_ghost_total_ = 0;
    total_edges_ = 0;
    weighted_ = true;
    for (auto& hp : parts_) {
        hp.ghost_base = n_ghost_total_;
        if ((uint64_t)n_ghost_total_ + hp.ghost_gid.size() > 0xFFFFFFF0ull) fail(GXP_E_INVAL, "too many cached vertices");
        n_ghost_total_ += (uint32_t)hp.ghost_gid.size();
        total_edges_ += hp.n_edges();
        if (!hp.weighted() && hp.n_edges()) weighted_ = false;
    }

    pd_.assign(n_parts_, PartDev{});
    for (uint32_t p = 0; p < n_parts_; ++p) {
        HostPart& hp = parts_[p];
        // plain CSC copies: the out-degree pass and the bounds check read them
        if (!hp.on_device) {
            hp.d_col_ptr = upload_u32(hp.col_ptr, pad4(hp.n_own + 1));
            hp.d_src = upload_u32(hp.src, pad4(hp.src.size()));
        }
        pd_[p] = PartDev{hp.d_col_ptr, hp.d_src, nullptr, hp.n_own, hp.v_begin,
                         (uint32_t)hp.ghost_gid.size(), hp.ghost_base, hp.n_edges(),
                         nullptr, nullptr, nullptr, nullptr, nullptr,
                         hp.n_own + (n_ghost_total_ - hp.ghost_base), 0u};
    }
    // what the layout build reads: each partition's CSC as loaded (weights on
    // the device), and for a single partition (unless keep_ids) an order of
    // its vertices by decreasing in-degree with the renumbered offsets; the
    // row sort then reads old rows, renumbers their sources and writes new rows
    work_.assign(n_parts_, WorkCsc{});
    for (uint32_t p = 0; p < n_parts_; ++p) {
        HostPart& hp = parts_[p];
        const uint32_t* dw = hp.d_w;
        if (hp.weighted() && !dw) {
            dw = upload_u32(hp.w, pad4(hp.w.size()));
        }
        work_[p] = WorkCsc{hp.d_col_ptr, RowSource{hp.d_col_ptr, hp.d_src, dw, nullptr, nullptr}};
    }
    relabeled_ = false;
    if (n_parts_ == 1 && !cfg_.keep_ids && V > 1) {
        HostPart& hp = parts_[0];
        d_new2old_ = (uint32_t*)dalloc(4 * pad4(V));
        d_old2new_ = (uint32_t*)dalloc(4 * pad4(V));
        d_perm_tmp_ = (uint32_t*)dalloc(4 * pad4(V));
        uint32_t* rcol = (uint32_t*)dalloc(4 * pad4(V + 1));
        cuda_check(cudaMemsetAsync(rcol, 0, 4 * pad4(V + 1), stream_), "memset");
        void* scratch = nullptr;
        cudaError_t e = device_malloc(&scratch, relabel_scratch_bytes(V));
        if (e == cudaSuccess) e = launch_relabel(hp.d_col_ptr, V, d_new2old_, d_old2new_, rcol, (uint32_t*)scratch, stream_);
        cudaError_t e2 = cudaStreamSynchronize(stream_);
        if (scratch) device_free(scratch);
        cuda_check(e, "relabel");
        cuda_check(e2, "relabel");
        work_[0].col = rcol;
        work_[0].in.row_map = d_new2old_;
        work_[0].in.src_map = d_old2new_;
        relabeled_ = true;
        // host copy of the map: sources are renumbered without a device round trip
        h_old2new_.resize(V);
        cuda_check(cudaMemcpy(h_old2new_.data(), d_old2new_, 4ull * V, cudaMemcpyDeviceToHost), "relabel map");
    }
    d_parts_ = (PartDev*)dalloc(sizeof(PartDev) * n_parts_);
    before_h2d("upload");
    cuda_check(cudaMemcpyAsync(d_parts_, pd_.data(), sizeof(PartDev) * n_parts_, cudaMemcpyHostToDevice, stream_),
               "upload parts");
    sell_ready_ = false;
    const std::vector<PartDev>& pd = pd_;

    d_ghost_gid_ = (uint32_t*)dalloc(4 * (size_t)std::max<uint32_t>(n_ghost_total_, 1));
    d_ghost_ = (uint32_t*)dalloc(4 * pad4((size_t)n_ghost_total_ + 1));   // + the identity slot
    for (auto& hp : parts_)
        if (!hp.ghost_gid.empty()) {
            before_h2d("upload ghost ids");
            cuda_check(cudaMemcpyAsync(d_ghost_gid_ + hp.ghost_base, hp.ghost_gid.data(), 4 * hp.ghost_gid.size(),
                                       cudaMemcpyHostToDevice, stream_), "upload ghost ids");
        }
    cuda_check(cudaStreamSynchronize(stream_), "upload");

    // out-degrees over all partitions' edges
    // vertex arrays are padded so 16-byte-aligned bulk copies of any slice stay inside
    d_outdeg_ = (uint32_t*)dalloc(4 * pad4(V));
    cuda_check(cudaMemsetAsync(d_outdeg_, 0, 4 * pad4(V), stream_), "memset");
    uint32_t* outdeg_in = relabeled_ ? d_perm_tmp_ : d_outdeg_;   // input ids, then renumbered
    if (relabeled_) cuda_check(cudaMemsetAsync(outdeg_in, 0, 4 * pad4(V), stream_), "memset");
    for (uint32_t p = 0; p < n_parts_; ++p)
        cuda_check(launch_outdeg(pd[p], parts_[p].d_src, d_ghost_gid_ + parts_[p].ghost_base, outdeg_in, stream_),
                   "out-degrees");
    if (relabeled_)
        cuda_check(launch_permute_u32(outdeg_in, d_old2new_, V, d_outdeg_, true, stream_), "out-degrees");

    for (int b = 0; b < 2; ++b) {
        d_own_[b] = (uint32_t*)dalloc(4 * pad4(V));
        d_rank_[b] = (float*)dalloc(4 * pad4(V));
        cuda_check(cudaMemsetAsync(d_own_[b], 0, 4 * pad4(V), stream_), "memset");
        cuda_check(cudaMemsetAsync(d_rank_[b], 0, 4 * pad4(V), stream_), "memset");
    }
    d_stats_ = (StepStats*)dalloc(sizeof(StepStats) * kStatRing);
    d_err_ = (uint32_t*)dalloc(4);
    cuda_check(cudaMemsetAsync(d_err_, 0, 4, stream_), "memset");
    if (cfg_.check_bounds)
        for (uint32_t p = 0; p < n_parts_; ++p)
            cuda_check(launch_validate_csc(parts_[p].d_col_ptr, parts_[p].n_own, parts_[p].d_src, pd[p].n_edges,
                                           parts_[p].n_own + pd[p].n_ghost, d_err_, stream_), "validate");
    if (n_parts_ > 1) build_caches();
    cuda_check(cudaStreamSynchronize(stream_), "finalize");   // host staging vectors die after this
    check_device_error();
    finalized_ = true;
}

// Boundary bitmap (vertices another partition caches), global-data-queue
// layout for the sync of Algorithm 3, and under a cache budget the kept and
// downloaded copies.
void Engine::build_caches() {
    const uint32_t V = (uint32_t)n_vertices_;
    const size_t words = ((size_t)V + 31) / 32 + 2;
    // boundary vertices: cached by some other partition
    std::vector<uint32_t> bbits(words, 0);
    for (auto& hp : parts_)
        for (uint32_t g : hp.ghost_gid) bbits[g >> 5] |= 1u << (g & 31);
    uint64_t gdq_total = 0;
    max_words_ = 0;
    for (auto& hp : parts_) {
        hp.n_boundary = 0;
        const uint32_t wl = hp.v_begin >> 5, wh = (hp.v_begin + hp.n_own + 31) >> 5;
        for (uint32_t wi = wl; wi < wh; ++wi) {
            uint32_t bits = bbits[wi];
            const uint32_t base = wi * 32u;
            if (base < hp.v_begin) bits &= ~0u << (hp.v_begin - base);
            if (base + 32u > hp.v_begin + hp.n_own) bits &= (hp.v_begin + hp.n_own - base) >= 32u ? ~0u : ((1u << (hp.v_begin + hp.n_own - base)) - 1u);
            hp.n_boundary += (uint32_t)__builtin_popcount(bits);
        }
        hp.gdq_base = gdq_total;
        gdq_total += hp.n_boundary;
        max_words_ = std::max(max_words_, hp.n_own ? wh - wl : 0u);
    }
    if (gdq_total > 0xFFFFFFF0ull) fail(GXP_E_INVAL, "global data queue too large");
    d_boundary_ = (uint32_t*)dalloc(4 * words);
    d_changed_ = (uint32_t*)dalloc(4 * words);
    d_gdq_ids_ = (uint32_t*)dalloc(4 * std::max<uint64_t>(gdq_total, 1));
    d_gdq_vals_ = (uint32_t*)dalloc(4 * std::max<uint64_t>(gdq_total, 1));
    d_gdq_base_ = (uint64_t*)dalloc(8 * n_parts_);
    std::vector<uint64_t> gb(n_parts_);
    for (uint32_t p = 0; p < n_parts_; ++p) gb[p] = parts_[p].gdq_base;
    sync_blocks_x_ = std::max<uint32_t>((max_words_ + 255) / 256, 1);
    d_block_counts_ = (uint32_t*)dalloc(4 * (size_t)n_parts_ * sync_blocks_x_);
    d_block_offsets_ = (uint32_t*)dalloc(4 * (size_t)n_parts_ * sync_blocks_x_);
    d_part_counts_ = (uint32_t*)dalloc(4 * n_parts_);
    d_done_ctr_ = (uint32_t*)dalloc(4);
    before_h2d("upload");
    cuda_check(cudaMemcpyAsync(d_boundary_, bbits.data(), 4 * words, cudaMemcpyHostToDevice, stream_), "upload");
    before_h2d("upload");
    cuda_check(cudaMemcpyAsync(d_gdq_base_, gb.data(), 8 * n_parts_, cudaMemcpyHostToDevice, stream_), "upload");
    cuda_check(cudaMemsetAsync(d_changed_, 0, 4 * words, stream_), "memset");
    cuda_check(cudaMemsetAsync(d_part_counts_, 0, 4 * n_parts_, stream_), "memset");
    cuda_check(cudaMemsetAsync(d_done_ctr_, 0, 4, stream_), "memset");
    // caching under a budget: the LRU state of every copy (lru.cu); the
    // cache starts empty at every gxp_begin
    lru_ = Lru{};
    if (cfg_.cache_slots != 0 && n_ghost_total_ > 0) {
        lru_.on = true;
        lru_.capacity = cfg_.cache_slots == GXP_CACHE_NONE ? 0u : cfg_.cache_slots;
        std::vector<uint32_t> reads(n_ghost_total_, 0), base(n_parts_ + 1, 0);
        for (uint32_t p = 0; p < n_parts_; ++p) {
            const HostPart& hp = parts_[p];
            base[p] = hp.ghost_base;
            base[p + 1] = hp.ghost_base + (uint32_t)hp.ghost_gid.size();
            lru_.max_per_part = std::max<uint32_t>(lru_.max_per_part, (uint32_t)hp.ghost_gid.size());
            for (uint32_t u : hp.src)
                if (u >= hp.n_own) ++reads[hp.ghost_base + (u - hp.n_own)];
        }
        const size_t G = n_ghost_total_;
        lru_.d_base = upload_u32(base, base.size());
        lru_.d_reads = upload_u32(reads, G);
        lru_.d_weight = (uint32_t*)dalloc(4 * G);
        lru_.d_flags = (uint8_t*)dalloc(G);
        lru_.d_hist = (uint32_t*)dalloc(4ull * kLruBins * n_parts_);
        lru_.d_part = (LruPart*)dalloc(sizeof(LruPart) * n_parts_);
        lru_.d_tie = (uint32_t*)dalloc(4 * G);
        lru_.d_tie_scan = (uint32_t*)dalloc(4 * (G + 1));
        lru_.d_scratch = (uint32_t*)dalloc(4 * ((G + 2047) / 2048 + 1));
        cuda_check(cudaMemsetAsync(lru_.d_hist, 0, 4ull * kLruBins * n_parts_, stream_), "memset");
        cuda_check(cudaMemsetAsync(lru_.d_part, 0, sizeof(LruPart) * n_parts_, stream_), "memset");
    }
    // the host copies must outlive the async uploads
    cuda_check(cudaStreamSynchronize(stream_), "upload caches");
}

// ------------------------------------------------------------- algorithms

static Algo to_algo(gxp_algo a) {
    switch (a) {
        case GXP_ALGO_SSSP: return Algo::SSSP;
        case GXP_ALGO_CC: return Algo::CC;
        case GXP_ALGO_PAGERANK: return Algo::PR;
        case GXP_ALGO_PPR: return Algo::PR;   // PageRank with the teleport returning to one source
        case GXP_ALGO_LP: return Algo::LP;
        default: fail(GXP_E_INVAL, "unknown algorithm");
    }
}

void Engine::begin(gxp_algo algo, uint32_t source, float damping) {
    TraceRange trace_("gxp begin");
    if (!have_graph_) fail(GXP_E_STATE, "no graph");
    const Algo a = to_algo(algo);
    const bool personalized = algo == GXP_ALGO_PPR;
    if ((a == Algo::SSSP || personalized) && source >= n_vertices_) fail(GXP_E_INVAL, "source out of range");
    if (a == Algo::PR && !(damping >= 0.0f && damping < 1.0f)) fail(GXP_E_INVAL, "damping must be in [0, 1)");
    if (!finalized_) finalize();
    if (a == Algo::SSSP && !weighted_) fail(GXP_E_INVAL, "SSSP needs edge weights on every partition");
    if (!sell_ready_) build_sell();
    const uint32_t V = (uint32_t)n_vertices_;
    begun_ = false;   // until the state below is complete
    cuda_check(cudaMemsetAsync(d_stats_, 0, sizeof(StepStats) * kStatRing, stream_), "memset");
    uint32_t src_int = source;   // the source in internal ids
    if (relabeled_ && (a == Algo::SSSP || personalized)) src_int = h_old2new_[source];
    const uint32_t ppr_source = personalized ? src_int : kInf;
    cuda_check(launch_init_values(a, ppr_source, V, src_int, d_own_[0], d_rank_[0], d_outdeg_, d_stats_,
                                  relabeled_ ? d_new2old_ : nullptr, stream_),
               "init values");
    cuda_check(launch_init_ghosts(a, n_ghost_total_, d_ghost_gid_, d_own_[0], d_ghost_, stream_), "init caches");
    // the identity slots empty SELL slots read: 0 (sums) or INF (minima)
    cuda_check(launch_identity_slots(d_own_[0] + V, d_own_[1] + V, d_ghost_ + n_ghost_total_,
                                     a == Algo::PR ? 0u : kInf, stream_),
               "identity slots");
    if (d_changed_) cuda_check(cudaMemsetAsync(d_changed_, 0, 4 * (((size_t)V + 31) / 32 + 2), stream_), "memset");
    cur_ = 0;
    lru_reset(a == Algo::SSSP || personalized ? src_int : kInf);
    // (the packed frontier counter needs lists of fewer than 2^32 items)
    if (a == Algo::LP) {
        build_lp();
        // rows without in-edges are never written: both buffers hold their labels
        cuda_check(cudaMemcpyAsync(d_own_[1], d_own_[0], 4ull * V, cudaMemcpyDeviceToDevice, stream_), "copy values");
    }
    frontier_ = (a == Algo::SSSP || a == Algo::CC) && cfg_.direction != GXP_DIR_PULL &&
                (uint64_t)V + n_ghost_total_ + (total_edges_ + kItemEdges - 1) / kItemEdges < (1ull << 32);
    if (frontier_) {
        build_out_edges();
        // both value buffers start equal: the push superstep lowers the next
        // buffer in place, which must hold values no lower than the current
        cuda_check(cudaMemcpyAsync(d_own_[1], d_own_[0], 4ull * V, cudaMemcpyDeviceToDevice, stream_), "copy values");
        cur_ = 0;
        step_ = 0;
        seed_frontier(a == Algo::SSSP ? src_int : kInf);   // CC: every label is new
    }
    algo_ = a;
    ppr_source_ = ppr_source;
    source_ = source;
    damping_ = damping;
    cur_ = 0;
    step_ = accounted_ = 0;
    st_ = gxp_stats{};
    begun_ = true;
}

// Launch arguments of the superstep kernel for superstep step_ (the kernel
// derives the buffers and stat slots of superstep t from t).
SellArgs Engine::sell_args() const {
    SellArgs a{};
    a.slices = d_slices_;
    a.n_slices = n_slices_;
    a.hubs = d_hubs_;
    a.n_hubs = n_hubs_;
    a.parts = d_parts_;
    a.n_parts = n_parts_;
    a.n_vertices = (uint32_t)n_vertices_;
    a.own[0] = d_own_[0];
    a.own[1] = d_own_[1];
    a.rank[0] = d_rank_[0];
    a.rank[1] = d_rank_[1];
    a.stats = d_stats_;
    a.lists[0] = d_list_[0];
    a.lists[1] = d_list_[1];
    a.step = step_;
    a.ghost = d_ghost_;
    a.outdeg = d_outdeg_;
    a.changed_bits = n_parts_ > 1 ? d_changed_ : nullptr;
    a.hub_val = d_hub_val_;
    a.hub_arrive = d_hub_arrive_;
    a.err = d_err_;
    a.check_bounds = cfg_.check_bounds;
    a.damping = damping_;
    a.inv_n = (float)(1.0 / (double)n_vertices_);
    a.ppr_source = ppr_source_;
    a.early_exit = (early_exit_ && algo_ != Algo::PR) ? 1u : 0u;
    a.n_zero = (algo_ == Algo::PR && n_parts_ == 1) ? n_zero_slices_ : 0u;
    if (frontier_) {   // the kernel picks the direction on the device from the frontier's size
        a.fc.list_out = d_list_[1];   // non-null: lists on
        a.fc.direction = cfg_.direction;
        a.fc.push_div = cfg_.push_div;
        a.fc.total_edges = total_edges_;
        a.fc.list_cap = list_cap_;
        a.fc.err = d_err_;
        // several partitions: a pull lists its changed vertices only when the
        // frontier it read was within kListSlack times the push limit (in
        // vertices, at the average degree); there the list's scattered
        // out-degree loads cost every pull superstep ~13% (ER 2^24, 8 parts)
        a.fc.list_max_changed = kAlwaysList;
        if (n_parts_ > 1 && cfg_.direction == GXP_DIR_AUTO && n_vertices_ > 0) {
            const double V = (double)n_vertices_, E = (double)total_edges_;
            a.fc.list_max_changed = (uint64_t)(kListSlack * E / ((double)cfg_.push_div * (1.0 + E / V)));
        }
        a.out_ptr = d_out_ptr_;
        a.out_dst = d_out_dst_;
        a.out_w = algo_ == Algo::SSSP ? d_out_w_ : nullptr;
    }
    return a;
}

LruArgs Engine::lru_args(StepStats* out, const StepStats* quiet) const {
    LruArgs a{};
    a.n_parts = n_parts_;
    a.n_ghost = n_ghost_total_;
    a.ghost_base = lru_.d_base;
    a.ghost_gid = d_ghost_gid_;
    a.reads = lru_.d_reads;
    a.weight = lru_.d_weight;
    a.flags = lru_.d_flags;
    a.ghost = d_ghost_;
    a.capacity = lru_.capacity;
    a.hist = lru_.d_hist;
    a.part_state = lru_.d_part;
    a.tie = lru_.d_tie;
    a.tie_scan = lru_.d_tie_scan;
    a.scan_scratch = lru_.d_scratch;
    a.stats_out = out;
    a.quiet_check = quiet;
    return a;
}

// A new run starts with empty caches; the boundary before its first
// superstep admits the copies that superstep uses (every vertex, or the
// source of SSSP / personalized PageRank) into the stats of superstep 0.
void Engine::lru_reset(uint32_t source_int) {
    if (!lru_.on) return;
    cuda_check(cudaMemsetAsync(lru_.d_flags, 0, n_ghost_total_, stream_), "memset");
    cuda_check(cudaMemsetAsync(lru_.d_weight, 0, 4ull * n_ghost_total_, stream_), "memset");
    LruArgs la = lru_args(d_stats_ + 1, nullptr);
    la.own_val = d_own_[cur_];
    la.frontier_all = source_int == kInf ? 1u : 0u;
    la.frontier_one = source_int;
    cuda_check(launch_lru_boundary(la, lru_.max_per_part, stream_), "cache start");
}

// The vertex ids of the copies partition `part` holds in its cache now
// (ascending).
void Engine::cache_contents(uint32_t part, uint32_t* ids, uint64_t cap, uint64_t* n_out) {
    if (!finalized_) fail(GXP_E_STATE, "no graph is loaded");
    if (part >= n_parts_) fail(GXP_E_INVAL, "partition index out of range");
    if (!n_out) fail(GXP_E_INVAL, "n_out is required");
    const HostPart& hp = parts_[part];
    std::vector<uint32_t> kept;
    if (!lru_.on) {
        kept = hp.ghost_gid;   // no budget: every copy is cached
    } else {
        std::vector<uint8_t> f(hp.ghost_gid.size());
        cuda_check(cudaStreamSynchronize(stream_), "sync");
        if (!f.empty())
            cuda_check(cudaMemcpy(f.data(), lru_.d_flags + hp.ghost_base, f.size(), cudaMemcpyDeviceToHost),
                       "read cache flags");
        for (size_t i = 0; i < f.size(); ++i)
            if (f[i] & 1u) kept.push_back(hp.ghost_gid[i]);
    }
    *n_out = kept.size();
    if (cap < kept.size()) fail(GXP_E_INVAL, "cap smaller than the number of cached copies");
    if (!kept.empty()) {
        if (!ids) fail(GXP_E_INVAL, "null output array");
        cuda_check(cudaMemcpy(ids, kept.data(), 4 * kept.size(), cudaMemcpyDefault), "copy cached ids");
    }
}

uint64_t Engine::superstep(gxp_algo algo, gxp_msggen g, gxp_merge m, gxp_apply ap, bool want) {
    TraceRange trace_("gxp superstep");
    if (!begun_) fail(GXP_E_STATE, "gxp_begin must come first");
    if (to_algo(algo) != algo_ || (algo == GXP_ALGO_PPR) != (ppr_source_ != kInf))
        fail(GXP_E_INVAL, "algorithm differs from the one begun");
    const bool ok = (algo_ == Algo::SSSP && g == GXP_GEN_RELAX && m == GXP_MERGE_MIN && ap == GXP_APPLY_MIN) ||
                    (algo_ == Algo::CC && g == GXP_GEN_LABEL && m == GXP_MERGE_MIN && ap == GXP_APPLY_MIN) ||
                    (algo_ == Algo::PR && g == GXP_GEN_CONTRIB && m == GXP_MERGE_SUM && ap == GXP_APPLY_PAGERANK) ||
                    (algo_ == Algo::LP && g == GXP_GEN_LABEL && m == GXP_MERGE_MODE && ap == GXP_APPLY_SET);
    if (!ok) fail(GXP_E_UNSUPPORTED, "unsupported (msggen, merge, apply) template for this algorithm");
    const int nx = cur_ ^ 1;
    cuda_check(cudaEventRecord(ev_a_, stream_), "event");
    if (algo_ == Algo::LP) {
        LpArgs l{};
        l.parts = lp_.d_parts;
        l.n_parts = n_parts_;
        l.windows = lp_.d_windows;
        l.n_windows = lp_.n_windows;
        l.row_g = lp_.d_row_g;
        l.warp_rows = lp_.d_warp_rows;
        l.n_warp_rows = lp_.n_warp_rows;
        l.chunks = lp_.d_chunks;
        l.n_chunks = lp_.n_chunks;
        l.hubs = lp_.d_hubs;
        l.n_hubs = lp_.n_hubs;
        l.segments = lp_.d_segments;
        l.n_segments = lp_.n_segments;
        l.hub_best = lp_.d_hub_best;
        l.seg_used = lp_.d_seg_used;
        l.keys = lp_.d_keys;
        l.counts = lp_.d_counts;
        l.own_cur = d_own_[cur_];
        l.own_nxt = d_own_[nx];
        l.ghost = d_ghost_;
        l.changed_bits = n_parts_ > 1 ? d_changed_ : nullptr;
        l.stats_in = d_stats_ + step_ % kStatRing;
        l.stats_out = d_stats_ + (step_ + 1) % kStatRing;
        l.stats_clear = d_stats_ + (step_ + 2) % kStatRing;
        l.skip_if_quiet = (early_exit_ && step_ > 0) ? 1u : 0u;
        l.narrow_labels = n_vertices_ <= (1ull << 27) ? 1u : 0u;   // labels are vertex ids
        cuda_check(launch_lp_superstep(l, stream_), "label propagation superstep");
    } else {
        const SellArgs a = sell_args();
        cuda_check(launch_superstep_sell(algo_, a, stream_), "superstep kernel");
    }
    cuda_check(cudaEventRecord(ev_k_, stream_), "event");
    if (n_parts_ > 1) {
        SyncArgs s{};
        s.parts = d_parts_;
        s.n_parts = n_parts_;
        s.changed_bits = d_changed_;
        s.boundary_bits = d_boundary_;
        s.own_val = d_own_[nx];
        s.ghost_gid = d_ghost_gid_;
        s.n_ghost = n_ghost_total_;
        s.ghost = d_ghost_;
        s.cached = lru_.on ? lru_.d_flags : nullptr;
        s.n_pull = n_ghost_total_;
        s.gdq_ids = d_gdq_ids_;
        s.gdq_vals = d_gdq_vals_;
        s.gdq_base = d_gdq_base_;
        s.block_counts = d_block_counts_;
        s.block_offsets = d_block_offsets_;
        s.part_counts = d_part_counts_;
        s.done_ctr = d_done_ctr_;
        s.blocks_x = sync_blocks_x_;
        s.stats_out = d_stats_ + (step_ + 1) % kStatRing;
        if (frontier_) {   // delivered copies join the next superstep's frontier
            s.fc.list_out = d_list_[(step_ + 1) & 1];
            s.fc.list_cap = list_cap_;
            s.fc.err = d_err_;
            s.fc.direction = cfg_.direction;
            s.fc.push_div = cfg_.push_div;
            s.fc.total_edges = total_edges_;
            s.out_ptr = d_out_ptr_;
            s.n_vertices = (uint32_t)n_vertices_;
        }
        // an injected fault drops the whole exchange, as a lost message would;
        // the superstep's delivery mark then stays unset (see account())
        if (faults_.sync_at != ++n_exchanges_) {
            TraceRange trace_sync("gxp exchange (lazy upload, skip, cache)");
            cuda_check(launch_sync(s, max_words_, stream_), "sync kernels");
            // the cache before the next superstep: its frontier is this
            // superstep's changed vertices; what it uses and does not hold
            // is downloaded (counted in the next superstep's stats)
            if (lru_.on) {
                // a superstep after a quiet one (inside gxp_run) did nothing: neither does its boundary
                const bool maybe_quiet = early_exit_ && algo_ != Algo::PR && step_ > 0;
                LruArgs la = lru_args(d_stats_ + (step_ + 2) % kStatRing,
                                      maybe_quiet ? d_stats_ + step_ % kStatRing : nullptr);
                la.own_val = d_own_[nx];
                la.frontier_bits = d_changed_;
                cuda_check(launch_lru_boundary(la, lru_.max_per_part, stream_), "cache update");
            }
        }
        cuda_check(cudaMemsetAsync(d_changed_, 0, 4 * (((size_t)n_vertices_ + 31) / 32 + 2), stream_), "memset");
    }
    cuda_check(cudaEventRecord(ev_b_, stream_), "event");
    cur_ = nx;
    ++step_;
    if (want || step_ - accounted_ >= 32) account(false);
    return st_.last_changed;
}

// Fold the device-side stats of the supersteps not yet read into st_.
// Fold the device-side stats of the supersteps not yet read into st_ (one
// copy of the stat ring). With stop_at_quiet, stop at the first superstep
// that changed nothing and roll the step counter back to it (the supersteps
// enqueued after it ran on a fixed point and changed nothing either); its
// index is returned, else 0.
uint64_t Engine::account(bool stop_at_quiet, bool ring_copied) {
    if (accounted_ == step_) return 0;
    if (!ring_copied) {
        cuda_check(cudaStreamSynchronize(stream_), "superstep");
        ring_host_.resize(kStatRing);
        cuda_check(cudaMemcpy(ring_host_.data(), d_stats_, sizeof(StepStats) * kStatRing, cudaMemcpyDeviceToHost),
                   "read stats");
    }
    check_device_error();
    uint64_t quiet = 0;
    for (uint64_t t = accounted_ + 1; t <= step_; ++t) {
        const StepStats& s = ring_host_[t % kStatRing];
        unsigned long long ch = 0, dg = 0, l1 = 0;
        for (int i = 0; i < kStatLanes; ++i) {
            ch += s.changed[i];
            dg += s.dangling_fx[i];
            l1 += s.l1_fx[i];
        }
        st_.supersteps++;
        st_.edges_scanned += s.pushed ? s.push_edges : total_edges_;
        if (s.pushed) st_.push_supersteps++;
        st_.last_changed = ch;
        if (algo_ == Algo::PR) {
            st_.last_dangling = fx_to_double(dg);
            st_.last_l1_delta = fx_to_double(l1);
        }
        if (n_parts_ > 1) {
            // every exchange marks its superstep's slot; a missing mark means
            // the caches and upload lists of that superstep were never delivered
            if (!s.exchanged)
                fail(GXP_E_LOST, "the exchange between partitions of superstep " + std::to_string(t) +
                                     " did not arrive");
            st_.cache_downloads += s.downloads;
            st_.last_boundary_changed = s.boundary_changed;
            st_.sync_pairs += s.boundary_changed;
            if (s.skipped) st_.syncs_skipped++;
            else st_.syncs_done++;
        }
        if (stop_at_quiet && ch == 0) {
            quiet = t;
            break;
        }
    }
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, ev_a_, ev_b_) == cudaSuccess) st_.last_superstep_ms = ms;
    else cudaGetLastError();
    if (cudaEventElapsedTime(&ms, ev_a_, ev_k_) == cudaSuccess) st_.last_kernel_ms = ms;
    else cudaGetLastError();
    if (quiet && quiet < step_) {
        // the next two supersteps accumulate into these slots: clear the overshoot's values
        for (uint64_t t = quiet + 1; t <= quiet + 2; ++t)
            cuda_check(cudaMemsetAsync(d_stats_ + (t % kStatRing), 0, sizeof(StepStats), stream_), "memset");
        step_ = quiet;
        cur_ = (int)(quiet & 1u);   // the buffer the quiet superstep wrote (later ones may have returned early)
    }
    accounted_ = step_;
    return quiet;
}

// Out-edge copy for the push direction: offsets from the out-degrees and the
// edges of the layout's CSC (renumbered like the layout), grouped by source.
// Several partitions: the edges' sources are slots, the V vertices (their
// out-edges into their own partition) then every partition's cached copies
// (that partition's in-edges from the copied vertex), built from a CSC over
// global rows with slot sources (temporary).
void Engine::build_out_edges() {
    TraceRange trace_("gxp out-edge build");
    if (out_ready_) return;
    const uint32_t V = (uint32_t)n_vertices_;
    const uint64_t E = total_edges_;
    const uint32_t S = V + n_ghost_total_;   // slots
    if ((uint64_t)V + n_ghost_total_ >= 0xFFFFFFF0ull) fail(GXP_E_INVAL, "too many vertices and cached copies");
    n_slots_ = S;
    d_out_ptr_ = (uint32_t*)dalloc(4 * pad4((size_t)S + 1));
    d_out_dst_ = (uint32_t*)dalloc(4 * std::max<uint64_t>(E, 1));
    d_out_w_ = weighted_ ? (uint32_t*)dalloc(4 * std::max<uint64_t>(E, 1)) : nullptr;
    list_cap_ = (uint64_t)S + (E + kItemEdges - 1) / kItemEdges;
    for (auto& l : d_list_) l = (uint2*)dalloc(sizeof(uint2) * std::max<uint64_t>(list_cap_, 1));
    std::vector<void*> tmp;
    auto talloc = [&](size_t bytes) -> void* {
        void* q = nullptr;
        cuda_check(device_malloc(&q, std::max<size_t>(bytes, 16)), "cudaMalloc");
        tmp.push_back(q);
        return q;
    };
    struct FreeTmp {
        std::vector<void*>& v;
        cudaStream_t s;
        ~FreeTmp() {
            cudaStreamSynchronize(s);
            for (void* q : v) cudaFreeAsync(q, s);   // pool blocks (device_malloc)
        }
    } free_tmp{tmp, stream_};
    RowSource in = work_[0].in;
    const uint32_t* deg = d_outdeg_;
    if (n_parts_ > 1) {
        uint32_t* ucol = (uint32_t*)talloc(4 * ((size_t)V + 1));
        uint32_t* usrc = (uint32_t*)talloc(4 * std::max<uint64_t>(E, 1));
        uint32_t* uw = weighted_ ? (uint32_t*)talloc(4 * std::max<uint64_t>(E, 1)) : nullptr;
        uint64_t at = 0;
        for (uint32_t p = 0; p < n_parts_; ++p) {
            cuda_check(launch_unify_csc(pd_[p], V, at, ucol, usrc, p + 1 == n_parts_, stream_), "slot CSC");
            if (uw && pd_[p].n_edges)
                cuda_check(cudaMemcpyAsync(uw + at, work_[p].in.w, 4 * pd_[p].n_edges, cudaMemcpyDeviceToDevice,
                                           stream_), "slot CSC weights");
            at += pd_[p].n_edges;
        }
        uint32_t* sdeg = (uint32_t*)talloc(4 * ((size_t)S + 1));
        cuda_check(launch_slot_degrees(usrc, E, S, sdeg, stream_), "slot degrees");
        in = RowSource{ucol, usrc, uw, nullptr, nullptr};
        deg = sdeg;
    }
    uint32_t* scratch = (uint32_t*)talloc(4 * out_edges_scratch_words(S, E));
    cuda_check(launch_out_edges(in, V, S, E, deg, d_out_ptr_, scratch, d_out_dst_, weighted_ ? d_out_w_ : nullptr,
                                stream_), "out-edges");
    cuda_check(cudaStreamSynchronize(stream_), "out-edges");
    out_ready_ = true;
}

// The frontier the next superstep reads: one vertex, or all (kInf) slots.
// Several partitions start from the slots whose value is finite (every slot
// for CC; SSSP: the source and its cached copies).
void Engine::seed_frontier(uint32_t source_int) {
    FrontierCfg f{};
    f.list_out = d_list_[step_ & 1];
    f.list_cap = list_cap_;
    f.err = d_err_;
    f.direction = cfg_.direction;   // a forced push reads the items of an all-vertex seed
    if (n_parts_ > 1 && source_int != kInf) {
        cuda_check(launch_seed_finite((uint32_t)n_vertices_, n_ghost_total_, d_own_[cur_], d_ghost_, d_out_ptr_, f,
                                      d_stats_ + (step_ % kStatRing), stream_), "seed frontier");
        return;
    }
    cuda_check(launch_seed_frontier(n_slots_, source_int, d_out_ptr_, f, d_stats_ + (step_ % kStatRing), stream_),
               "seed frontier");
}

// Row lists of label propagation, by in-degree class (host-built once per
// graph from the partitions' offsets): 1..kLpSmall in-edges (packed into
// warp windows of adjacent edges, in CSC order), up to kLpChunk, and hub rows
// cut into chunks of kLpChunk with a hash table each, cut into segments.
void Engine::build_lp() {
    TraceRange trace_("gxp label-propagation lists");
    if (lp_.ready) return;
    std::vector<LpPart> parts(n_parts_);
    std::vector<LpRow> chunks, warp_rows;
    std::vector<LpWindow> windows;
    std::vector<uint32_t> row_g;
    std::vector<LpHub> hubs;
    std::vector<LpSegment> segments;
    uint64_t table_slots = 0;
    auto add_row = [&](uint32_t g, uint32_t p, uint32_t e0, uint32_t deg) {
        if (deg == 0) return;
        if (deg <= kLpSmall) {
            // joins the open window if its edges follow on and fit, else opens one
            LpWindow* w = windows.empty() ? nullptr : &windows.back();
            const uint32_t wn = w ? (w->n_part & 63u) : 0u;
            if (!w || (w->n_part >> 6) != p || w->e0 + wn != e0 || wn + deg > 32u) {
                windows.push_back(LpWindow{e0, (uint32_t)row_g.size(), 0u, p << 6});
                w = &windows.back();
            }
            const uint32_t at = w->n_part & 63u;
            w->starts |= 1u << at;
            w->n_part += deg;
            row_g.push_back(g);
        } else if (deg <= kLpWarpRow) {
            warp_rows.push_back(LpRow{g, p, e0, deg, kInf, {0, 0, 0}});
        } else if (deg <= kLpChunk) {
            chunks.push_back(LpRow{g, p, e0, deg, kInf, {0, 0, 0}});
        } else {
            uint32_t lg = 1;
            while ((1ull << lg) < 2ull * deg && lg < 32) ++lg;   // 2^32 slots hold any in-degree's labels
            const uint32_t h = (uint32_t)hubs.size();
            hubs.push_back(LpHub{g, lg, table_slots, (uint32_t)segments.size(), 0});
            for (uint64_t s0 = 0; s0 < (1ull << lg); s0 += kLpSegment)
                segments.push_back(LpSegment{h, (uint32_t)std::min<uint64_t>(kLpSegment, (1ull << lg) - s0),
                                             table_slots + s0});
            table_slots += 1ull << lg;
            for (uint32_t c = 0; c < deg; c += kLpChunk)
                chunks.push_back(LpRow{g, p, e0 + c, std::min(kLpChunk, deg - c), h, {0, 0, 0}});
        }
    };
    for (uint32_t p = 0; p < n_parts_; ++p) {
        HostPart& hp = parts_[p];
        std::vector<uint32_t> cp(hp.n_own + 1);
        cuda_check(cudaMemcpy(cp.data(), hp.d_col_ptr, 4ull * (hp.n_own + 1), cudaMemcpyDeviceToHost), "row offsets");
        const uint32_t* src = hp.d_src;
        if (relabeled_) {   // sources in internal ids, once: no renumbering lookup per edge and superstep
            uint32_t* rs = (uint32_t*)dalloc(4 * std::max<uint64_t>(hp.n_edges(), 1));
            cuda_check(launch_permute_u32(d_old2new_, hp.d_src, (uint32_t)hp.n_edges(), rs, false, stream_),
                       "renumber sources");
            src = rs;
        }
        parts[p] = LpPart{src, hp.v_begin, hp.n_own, hp.ghost_base, 0};
        for (uint32_t l = 0; l < hp.n_own; ++l) {   // input row order
            const uint32_t g = relabeled_ ? h_old2new_[l] : hp.v_begin + l;
            add_row(g, p, cp[l], cp[l + 1] - cp[l]);
        }
    }
    auto upload = [&](const void* h, size_t bytes) {
        void* d = dalloc(std::max<size_t>(bytes, 16));
        if (bytes) {
            before_h2d("upload label propagation lists");
            cuda_check(cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice), "upload label propagation lists");
        }
        return d;
    };
    lp_.d_parts = (LpPart*)upload(parts.data(), sizeof(LpPart) * parts.size());
    lp_.d_windows = (LpWindow*)upload(windows.data(), sizeof(LpWindow) * windows.size());
    lp_.d_row_g = (uint32_t*)upload(row_g.data(), 4 * row_g.size());
    lp_.d_chunks = (LpRow*)upload(chunks.data(), sizeof(LpRow) * chunks.size());
    lp_.d_warp_rows = (LpRow*)upload(warp_rows.data(), sizeof(LpRow) * warp_rows.size());
    lp_.n_warp_rows = (uint32_t)warp_rows.size();
    lp_.d_hubs = (LpHub*)upload(hubs.data(), sizeof(LpHub) * hubs.size());
    lp_.n_windows = (uint32_t)windows.size();
    lp_.n_chunks = (uint32_t)chunks.size();
    lp_.n_hubs = (uint32_t)hubs.size();
    lp_.d_segments = (LpSegment*)upload(segments.data(), sizeof(LpSegment) * segments.size());
    lp_.n_segments = (uint32_t)segments.size();
    lp_.d_seg_used = (uint32_t*)dalloc(4 * std::max<size_t>(segments.size(), 1));
    cuda_check(cudaMemsetAsync(lp_.d_seg_used, 0, 4 * std::max<size_t>(segments.size(), 1), stream_), "memset");
    lp_.d_hub_best = (unsigned long long*)dalloc(8 * std::max<size_t>(hubs.size(), 1));
    cuda_check(cudaMemsetAsync(lp_.d_hub_best, 0, 8 * std::max<size_t>(hubs.size(), 1), stream_), "memset");
    lp_.d_keys = (uint32_t*)dalloc(4 * std::max<uint64_t>(table_slots, 1));
    lp_.d_counts = (uint32_t*)dalloc(4 * std::max<uint64_t>(table_slots, 1));
    cuda_check(cudaMemsetAsync(lp_.d_keys, 0xFF, 4 * std::max<uint64_t>(table_slots, 1), stream_), "memset");
    cuda_check(cudaMemsetAsync(lp_.d_counts, 0, 4 * std::max<uint64_t>(table_slots, 1), stream_), "memset");
    lp_.ready = true;
}

void Engine::sync_result(uint32_t part, uint32_t* ids, void* vals, uint64_t cap, uint64_t* n_out, int* skipped) {
    if (!begun_ || step_ == 0) fail(GXP_E_STATE, "no superstep has run");
    if (part >= n_parts_) fail(GXP_E_INVAL, "partition index out of range");
    if (!n_out) fail(GXP_E_INVAL, "n_out is required");
    account(false);
    if (n_parts_ == 1) {
        *n_out = 0;
        if (skipped) *skipped = 1;
        return;
    }
    StepStats s;
    cuda_check(cudaMemcpy(&s, d_stats_ + (step_ % kStatRing), sizeof(s), cudaMemcpyDeviceToHost), "read stats");
    uint32_t n = 0;
    if (!s.skipped) cuda_check(cudaMemcpy(&n, d_part_counts_ + part, 4, cudaMemcpyDeviceToHost), "read count");
    *n_out = n;
    if (skipped) *skipped = s.skipped ? 1 : 0;
    if (n > cap) fail(GXP_E_INVAL, "cap smaller than the number of uploaded pairs");
    if (n == 0) return;
    if (!ids || !vals) fail(GXP_E_INVAL, "null output array");
    const uint64_t base = parts_[part].gdq_base;
    cuda_check(cudaMemcpy(ids, d_gdq_ids_ + base, 4ull * n, cudaMemcpyDefault), "copy gdq ids");
    cuda_check(cudaMemcpy(vals, d_gdq_vals_ + base, 4ull * n, cudaMemcpyDefault), "copy gdq values");
}

// The device-driven loop of the running min-label algorithm: a graph with
// one WHILE node whose body is the superstep kernel (step read from d_ctl_)
// followed by the control kernel that advances the step and sets the
// condition. Built once per algorithm and graph; false if the driver cannot
// build it (the run then drives the supersteps from the host).
bool Engine::run_graph_ready() {
    if (algo_ == Algo::PR || algo_ == Algo::LP || run_graph_failed_) return false;
    cudaGraphExec_t& ge = run_graph_[algo_ == Algo::SSSP ? 0 : 1];
    if (ge) return true;
    if (!h_ctl_) cuda_check(cudaMallocHost(&h_ctl_, 2 * sizeof(RunCtl)), "pinned run control");
    if (!h_ring_) cuda_check(cudaMallocHost(&h_ring_, sizeof(StepStats) * kStatRing), "pinned stats");
    if (!d_ctl_) d_ctl_ = (RunCtl*)dalloc(sizeof(RunCtl));
    cudaStream_t cs = nullptr;
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaGraphCreate(&g, 0);
    cudaGraphConditionalHandle h = 0;
    if (e == cudaSuccess) e = cudaGraphConditionalHandleCreate(&h, g, 1, cudaGraphCondAssignDefault);
    cudaGraphNodeParams np{};
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    cudaGraphNode_t node = nullptr;
    if (e == cudaSuccess) e = cudaGraphAddNode(&node, g, nullptr, nullptr, 0, &np);
    if (e == cudaSuccess) e = cudaStreamBeginCaptureToGraph(cs, np.conditional.phGraph_out[0], nullptr, nullptr, 0,
                                                            cudaStreamCaptureModeRelaxed);
    if (e == cudaSuccess) {
        SellArgs a = sell_args();
        a.step_dev = &d_ctl_->step;
        a.early_exit = 0u;   // the loop stops at the first quiet superstep
        cudaError_t e1 = launch_superstep_sell(algo_, a, cs);
        cudaError_t e2 = e1 == cudaSuccess ? launch_run_control(d_ctl_, d_stats_, h, cs) : e1;
        cudaGraph_t body = nullptr;
        e = cudaStreamEndCapture(cs, &body);
        if (e == cudaSuccess) e = e2;
    }
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ge, g, 0);
    if (g) cudaGraphDestroy(g);
    if (cs) cudaStreamDestroy(cs);
    if (e != cudaSuccess) {
        cudaGetLastError();
        if (ge) cudaGraphExecDestroy(ge);
        ge = nullptr;
        run_graph_failed_ = true;
        return false;
    }
    return true;
}

uint32_t Engine::run(gxp_algo algo, uint32_t source, float damping, uint32_t max_steps) {
    TraceRange trace_("gxp run");
    begin(algo, source, damping);
    const gxp_msggen g = algo_ == Algo::SSSP ? GXP_GEN_RELAX : algo_ == Algo::PR ? GXP_GEN_CONTRIB : GXP_GEN_LABEL;
    const gxp_merge m = algo_ == Algo::PR ? GXP_MERGE_SUM : algo_ == Algo::LP ? GXP_MERGE_MODE : GXP_MERGE_MIN;
    const gxp_apply ap = algo_ == Algo::PR ? GXP_APPLY_PAGERANK : algo_ == Algo::LP ? GXP_APPLY_SET : GXP_APPLY_MIN;
    uint32_t steps = 0;
    if (algo_ == Algo::PR) {
        for (; steps < max_steps; ++steps) superstep(algo, g, m, ap, false);
        account(false);
        return steps;
    }
    // SSSP / CC on one partition: the loop runs on the device until the first
    // superstep that changes nothing, at most kRunChunk supersteps per launch
    // and one host read per launch. A graph whose superstep is a few waves of
    // CTAs runs all of them in one persistent cooperative kernel (grid
    // barrier between supersteps); larger ones through a CUDA graph whose
    // WHILE node repeats superstep + control.
    const bool one = n_parts_ == 1 && algo_ != Algo::LP;
    SellArgs la{};
    if (one) {
        la = sell_args();
        la.early_exit = 0u;   // the loop stops at the first quiet superstep
    }
    const bool loop = one && sell_loop_fits(algo_, la);
    if (loop) {
        if (!h_ctl_) cuda_check(cudaMallocHost(&h_ctl_, 2 * sizeof(RunCtl)), "pinned run control");
        if (!h_ring_) cuda_check(cudaMallocHost(&h_ring_, sizeof(StepStats) * kStatRing), "pinned stats");
        if (!d_ctl_) d_ctl_ = (RunCtl*)dalloc(sizeof(RunCtl));
        if (!d_bar_) d_bar_ = (GridBar*)dalloc(sizeof(GridBar));
    }
    if (loop || (one && run_graph_ready())) {
        const cudaGraphExec_t ge = loop ? nullptr : run_graph_[algo_ == Algo::SSSP ? 0 : 1];
        while (steps < max_steps) {
            const uint32_t k = std::min<uint32_t>(kRunChunk, max_steps - steps);
            h_ctl_[0] = RunCtl{step_, step_ + k, 1u, 0u};
            before_h2d("run control");
            cuda_check(cudaMemcpyAsync(d_ctl_, h_ctl_, sizeof(RunCtl), cudaMemcpyHostToDevice, stream_), "run control");
            if (loop) cuda_check(cudaMemsetAsync(d_bar_, 0, sizeof(GridBar), stream_), "memset");
            cuda_check(cudaEventRecord(ev_a_, stream_), "event");
            if (loop) {
                cuda_check(launch_sell_loop(algo_, la, d_ctl_, d_bar_, cfg_.timeout_ns, faults_.timeout, stream_),
                           "run loop");
                ++st_.persistent_launches;
            } else {
                cuda_check(cudaGraphLaunch(ge, stream_), "run graph");
            }
            cuda_check(cudaEventRecord(ev_b_, stream_), "event");
            cuda_check(cudaMemcpyAsync(h_ctl_ + 1, d_ctl_, sizeof(RunCtl), cudaMemcpyDeviceToHost, stream_),
                       "run control");
            cuda_check(cudaMemcpyAsync(h_ring_, d_stats_, sizeof(StepStats) * kStatRing, cudaMemcpyDeviceToHost,
                                       stream_), "read stats");
            cuda_check(cudaStreamSynchronize(stream_), "run");
            if (loop) check_device_error();   // a grid barrier that ran out of time
            ring_host_.assign(h_ring_, h_ring_ + kStatRing);
            const uint64_t done = h_ctl_[1].step;
            if (done <= step_ || done > step_ + k) fail(GXP_E_CUDA, "device-driven run lost its step counter");
            steps += (uint32_t)(done - step_);
            step_ = done;
            cur_ = (int)(step_ & 1u);
            const uint64_t n_run = done - accounted_;
            const uint64_t quiet = account(true, true);
            float ms = 0.f;
            if (cudaEventElapsedTime(&ms, ev_a_, ev_b_) == cudaSuccess)
                st_.last_superstep_ms = st_.last_kernel_ms = ms / (double)n_run;
            if (quiet) return (uint32_t)quiet;
        }
        return steps;
    }
    // partitioned graphs: supersteps are enqueued in growing chunks and the
    // host reads their changed counts once per chunk; the run ends at the
    // first superstep that changed nothing (the count includes it) and the
    // ones after a quiet superstep return at once on the device
    uint32_t chunk = 4;
    struct EarlyExit {
        bool& f;
        ~EarlyExit() { f = false; }
    } guard{early_exit_};
    early_exit_ = true;
    while (steps < max_steps) {
        const uint32_t k = std::min<uint32_t>(chunk, max_steps - steps);
        for (uint32_t i = 0; i < k; ++i) superstep(algo, g, m, ap, false);
        const uint64_t quiet = account(true);
        if (quiet) return (uint32_t)quiet;
        steps += k;
        chunk = std::min<uint32_t>(2 * chunk, 16);
    }
    return steps;
}

void Engine::get_values(uint32_t part, void* out, uint64_t n) {
    if (!begun_) fail(GXP_E_STATE, "gxp_begin must come first");
    if (!out) fail(GXP_E_INVAL, "null output");
    uint64_t off = 0, cnt = n_vertices_;
    if (part != 0xFFFFFFFFu) {
        if (part >= n_parts_) fail(GXP_E_INVAL, "partition index out of range");
        off = parts_[part].v_begin;
        cnt = parts_[part].n_own;
    }
    if (n != cnt) fail(GXP_E_INVAL, "n must equal the number of vertices requested");
    const void* src = algo_ == Algo::PR ? (const void*)(d_rank_[cur_] + off) : (const void*)(d_own_[cur_] + off);
    if (relabeled_) {   // internal order -> input ids
        cuda_check(launch_permute_u32((const uint32_t*)src, d_old2new_, (uint32_t)cnt, d_perm_tmp_, false, stream_),
                   "map values");
        src = d_perm_tmp_;
    }
    cuda_check(cudaMemcpyAsync(out, src, 4 * cnt, cudaMemcpyDefault, stream_), "copy values");
    cuda_check(cudaStreamSynchronize(stream_), "copy values");
    check_device_error();
}

void Engine::set_values(uint32_t part, const void* in, uint64_t n) {
    if (!begun_) fail(GXP_E_STATE, "gxp_begin must come first");
    if (algo_ == Algo::PR) fail(GXP_E_UNSUPPORTED, "set_values is implemented for SSSP, CC and LP");
    if (!in) fail(GXP_E_INVAL, "null input");
    uint64_t off = 0, cnt = n_vertices_;
    if (part != 0xFFFFFFFFu) {
        if (part >= n_parts_) fail(GXP_E_INVAL, "partition index out of range");
        off = parts_[part].v_begin;
        cnt = parts_[part].n_own;
    }
    if (n != cnt) fail(GXP_E_INVAL, "n must equal the number of vertices given");
    account(false);
    if (relabeled_) {   // input ids -> internal order
        before_h2d("copy values");
        cuda_check(cudaMemcpyAsync(d_perm_tmp_, in, 4 * cnt, cudaMemcpyDefault, stream_), "copy values");
        cuda_check(launch_permute_u32(d_perm_tmp_, d_old2new_, (uint32_t)cnt, d_own_[cur_], true, stream_),
                   "map values");
    } else {
        before_h2d("copy values");
        cuda_check(cudaMemcpyAsync(d_own_[cur_] + off, in, 4 * cnt, cudaMemcpyDefault, stream_), "copy values");
    }
    cuda_check(launch_init_ghosts(algo_, n_ghost_total_, d_ghost_gid_, d_own_[cur_], d_ghost_, stream_), "refresh caches");
    if (algo_ == Algo::LP)   // rows without in-edges are read from either buffer
        cuda_check(cudaMemcpyAsync(d_own_[cur_ ^ 1], d_own_[cur_], 4ull * n_vertices_, cudaMemcpyDeviceToDevice,
                                   stream_), "copy values");
    if (frontier_) {   // any value may have moved: every vertex is in the next frontier
        cuda_check(cudaMemcpyAsync(d_own_[cur_ ^ 1], d_own_[cur_], 4ull * n_vertices_, cudaMemcpyDeviceToDevice,
                                   stream_), "copy values");
        seed_frontier(kInf);
    }
    cuda_check(cudaStreamSynchronize(stream_), "set values");
}

void Engine::stats(gxp_stats* out) {
    if (begun_) account(false);
    *out = st_;
    out->device_bytes = graph_bytes_;
}

// ------------------------------------------------------ block-size model

// Lemma 1 (Section III-A): per-entity costs k1 (download), k2 (compute),
// k3 (upload), per-block call cost a, d entities. The pipeline-time equation
//   T(b, s) = k1 b + max(k1 b, a + k2 b) + (s - 2) max(k1 b, a + k2 b, k3 b)
//             + max(a + k2 b, k3 b) + k3 b
// is minimised over b by the lemma's three cases; the integer choice scores
// s in {floor, ceil}(d / b_opt) with b = d / s, and b in {floor, ceil}(b_opt)
// with s = ceil(d / b), in the equation.
static double pipeline_time(double b, double s, double k1, double k2, double k3, double a) {
    const double tn = k1 * b, tc = a + k2 * b, tu = k3 * b;
    return tn + std::max(tn, tc) + (s - 2.0) * std::max(std::max(tn, tc), tu) + std::max(tc, tu) + tu;
}

void block_size_model(double k1, double k2, double k3, double a, uint64_t d, uint64_t* b_out,
                      uint64_t* s_out, double* t_out) {
    if (!(k1 > 0 && k2 > 0 && k3 >= 0 && a >= 0) || d < 2 || !b_out || !s_out || !t_out)
        fail(GXP_E_INVAL, "block-size model needs k1, k2 > 0, k3, a >= 0, d >= 2");
    const double dd = (double)d;
    const double q = std::sqrt(a * dd / (k1 + k3));
    const double kmax = std::max(k1, std::max(k2, k3));
    double b_opt = q;
    if (k1 == kmax && k1 > k2 && a / (k1 - k2) < q) b_opt = a / (k1 - k2);
    else if (k3 == kmax && k3 > k2 && a / (k3 - k2) < q) b_opt = a / (k3 - k2);
    if (!(b_opt > 0)) b_opt = 1.0;
    const double s_opt = dd / b_opt;
    double best_t = std::numeric_limits<double>::infinity(), best_b = 0;
    uint64_t best_s = 0;
    auto consider = [&](double b, uint64_t s) {
        const double t = pipeline_time(b, (double)s, k1, k2, k3, a);
        if (t < best_t || (t == best_t && s < best_s)) {
            best_t = t;
            best_b = b;
            best_s = s;
        }
    };
    for (double sc : {std::floor(s_opt), std::ceil(s_opt)}) {
        const uint64_t s = (uint64_t)std::min<double>(std::max<double>(sc, 2.0), dd);
        consider(dd / (double)s, s);
    }
    for (double bc : {std::floor(b_opt), std::ceil(b_opt)}) {
        const uint64_t b = (uint64_t)std::min<double>(std::max<double>(bc, 1.0), std::max<double>(std::floor(dd / 2), 1.0));
        consider((double)b, std::max<uint64_t>(2, (d + b - 1) / b));
    }
    *b_out = (uint64_t)std::ceil(best_b - 1e-9);
    *s_out = best_s;
    *t_out = best_t;
}

}  // namespace gxp
