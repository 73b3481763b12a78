// Host side of the query server (see server.hpp): graph residency, lanes
// with their admission / superstep / retirement loop, and the thread-safe
// query calls.
#include "server.hpp"
#include "trace.hpp"

#include <omp.h>

#include <algorithm>
#include <chrono>
#include <cstring>

namespace gxp {

namespace {

constexpr uint32_t kDefaultIters = 20;

bool on_device(const void* p) {
    if (!p) return false;
    cudaPointerAttributes at{};
    if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

// host view of an input array: the caller's host pointer, or a host copy of a device array
const uint32_t* host_view(const uint32_t* p, uint64_t n, std::vector<uint32_t>& keep) {
    if (!on_device(p)) return p;
    keep.resize(n);
    cuda_check(cudaMemcpy(keep.data(), p, 4 * n, cudaMemcpyDeviceToHost), "copy input");
    return keep.data();
}

}  // namespace

double Server::now() {
    return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

Server::Server(int device, uint64_t mem_budget) : device_(device), mem_budget_(mem_budget) {}

Server::~Server() {
    try {
        stop();
    } catch (...) {
    }
    cudaSetDevice(device_);
    for (auto& g : graphs_)
        for (auto& L : g->lanes)
            if (L) {
                if (L->stream) cudaStreamDestroy(L->stream);
                if (L->h_table) cudaFreeHost(L->h_table);
                if (L->h_improved) cudaFreeHost(L->h_improved);
            }
    for (cudaStream_t s : copy_streams_) cudaStreamDestroy(s);
    for (void* p : allocs_) cudaFree(p);
}

void* Server::dalloc(size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    if (mem_budget_ && bytes_ + bytes > mem_budget_)
        fail(GXP_E_NOMEM, "serving state exceeds the context's mem_budget");
    void* p = nullptr;
    cuda_check(cudaMalloc(&p, bytes), "cudaMalloc");
    allocs_.push_back(p);
    bytes_ += bytes;
    return p;
}

void Server::dfree(void* p, size_t bytes) {
    bytes = std::max<size_t>(bytes, 16);
    auto it = std::find(allocs_.begin(), allocs_.end(), p);
    if (it == allocs_.end()) return;
    allocs_.erase(it);
    cudaFree(p);
    bytes_ -= bytes;
}

// ------------------------------------------------------------------ graphs

uint32_t Server::add_graph(uint64_t n, uint64_t m, const uint32_t* src_in, const uint32_t* dst_in,
                           const uint32_t* w_in) {
    if (running_) fail(GXP_E_STATE, "graphs are added before gxp_serve_start");
    if (n == 0 || n >= 0xFFFFFFFFull) fail(GXP_E_INVAL, "n_vertices must be in [1, 2^32 - 2]");
    if (m > 0xFFFFFFFFull) fail(GXP_E_INVAL, "more than 2^32 - 1 edges");
    if (m && (!src_in || !dst_in)) fail(GXP_E_INVAL, "null edge array");
    cuda_check(cudaSetDevice(device_), "cudaSetDevice");
    std::vector<uint32_t> keep_s, keep_d, keep_w;
    const uint32_t* src = m ? host_view(src_in, m, keep_s) : nullptr;
    const uint32_t* dst = m ? host_view(dst_in, m, keep_d) : nullptr;
    const uint32_t* w = (m && w_in) ? host_view(w_in, m, keep_w) : nullptr;

    // stable counting sort by destination, in parallel: thread t owns the
    // destination range [lo_t, hi_t) and scans every edge in input order
    const int T = std::max(1, std::min(omp_get_max_threads(), 64));
    std::vector<uint64_t> col(n + 1, 0);
    std::vector<uint32_t> outdeg(n, 0);
    bool bad = false;
#pragma omp parallel num_threads(T) reduction(|| : bad)
    {
        const int t = omp_get_thread_num();
        const uint64_t lo = n * t / T, hi = n * (t + 1) / T;
        for (uint64_t e = 0; e < m; ++e) {
            const uint32_t d = dst[e], s = src[e];
            if (d >= n || s >= n) {
                bad = true;
                continue;
            }
            if (d >= lo && d < hi) ++col[d + 1];
            if (s >= lo && s < hi) ++outdeg[s];
        }
    }
    if (bad) fail(GXP_E_INVAL, "vertex id out of range");
    for (uint64_t v = 0; v < n; ++v) col[v + 1] += col[v];
    // resident edges stay 8 bytes: the 64-slot superstep is bound by instruction
    // issue, and unpacking a 4-byte edge costs more than the bytes it saves
    const bool packed = false;
    std::vector<uint2> edges(packed ? 0 : m);
    std::vector<uint32_t> epacked(packed ? m : 0);
    std::vector<uint32_t> esrc(m);
#pragma omp parallel num_threads(T)
    {
        const int t = omp_get_thread_num();
        const uint64_t lo = n * t / T, hi = n * (t + 1) / T;
        std::vector<uint64_t> pos(col.begin() + lo, col.begin() + hi);
        for (uint64_t e = 0; e < m; ++e) {
            const uint32_t d = dst[e];
            if (d < lo || d >= hi) continue;
            const uint64_t p = pos[d - lo]++;
            const uint32_t wt = w ? w[e] : 1u;
            if (packed) epacked[p] = wt << kPackSrcBits | src[e];
            else edges[p] = make_uint2(src[e], wt);
            esrc[p] = src[e];
        }
    }

    // work units of <= kUnitEdges in-edges; rows with more are split and
    // leave one partial row per unit (index + 1 in .w)
    std::vector<uint4> all, nz;
    std::vector<uint2> split;
    all.reserve(n + m / kUnitEdges + 1);
    nz.reserve(n + m / kUnitEdges + 1);
    uint64_t partials = 0;
    for (uint64_t v = 0; v < n; ++v) {
        const uint64_t e0 = col[v], deg = col[v + 1] - e0;
        if (deg <= kUnitEdges) {
            const uint4 u = make_uint4((uint32_t)v, (uint32_t)e0, (uint32_t)deg, 0u);
            all.push_back(u);
            if (deg) nz.push_back(u);
            continue;
        }
        split.push_back(make_uint2((uint32_t)v, (uint32_t)partials));
        for (uint64_t off = 0; off < deg; off += kUnitEdges) {
            const uint32_t len = (uint32_t)std::min<uint64_t>(kUnitEdges, deg - off);
            const uint4 u = make_uint4((uint32_t)v, (uint32_t)(e0 + off), len, (uint32_t)(++partials));
            all.push_back(u);
            nz.push_back(u);
        }
    }
    if (partials >= 0xFFFFFFFFull) fail(GXP_E_INVAL, "too many split rows");
    split.push_back(make_uint2(kInf, (uint32_t)partials));   // sentinel: end of the last split row

    auto G = std::make_unique<ServedGraph>();
    G->n = n;
    G->m = m;
    G->weighted = w_in != nullptr;   // an edgeless graph given a (vacuous) weight array serves SSSP too
    G->n_units_all = all.size();
    G->n_units_nz = nz.size();
    G->n_split_rows = (uint32_t)(split.size() - 1);
    G->n_partials = partials;
    auto up = [&](const void* h, size_t bytes) {
        void* d = dalloc(bytes);
        if (bytes) cuda_check(cudaMemcpy(d, h, bytes, cudaMemcpyHostToDevice), "upload graph");
        return d;
    };
    G->d_units_all = (uint4*)up(all.data(), sizeof(uint4) * all.size());
    G->d_units_nz = (uint4*)up(nz.data(), sizeof(uint4) * nz.size());
    G->packed = packed;
    G->d_edges = packed ? up(epacked.data(), 4 * m) : up(edges.data(), sizeof(uint2) * m);
    G->d_src = (uint32_t*)up(esrc.data(), 4 * m);
    std::vector<float> inv(n);
    for (uint64_t v = 0; v < n; ++v) inv[v] = outdeg[v] ? 1.0f / (float)outdeg[v] : 0.0f;
    G->d_inv_outdeg = (float*)up(inv.data(), 4 * n);
    G->d_split_rows = (uint2*)up(split.data(), sizeof(uint2) * split.size());
    graphs_.push_back(std::move(G));
    return (uint32_t)(graphs_.size() - 1);
}

// ------------------------------------------------------------- lifecycle

void Server::start(const gxp_serve_opts* opts) {
    if (running_) fail(GXP_E_STATE, "server already running");
    if (graphs_.empty()) fail(GXP_E_STATE, "no graph added");
    gxp_serve_opts o{};
    if (opts) o = *opts;
    if (o.max_slots == 0) o.max_slots = 64;
    if (o.max_slots > 64) fail(GXP_E_INVAL, "max_slots must be at most 64");
    if (o.results_per_graph == 0) o.results_per_graph = 2 * o.max_slots;
    queue_cap_ = o.queue_cap ? o.queue_cap : (1u << 20);
    cuda_check(cudaSetDevice(device_), "cudaSetDevice");
    // stream priorities: lanes of smaller graphs (shorter supersteps) first
    int least = 0, greatest = 0;
    cuda_check(cudaDeviceGetStreamPriorityRange(&least, &greatest), "stream priorities");
    std::vector<int> prio(graphs_.size(), least);
    if (o.priorities) {
        std::vector<uint32_t> order(graphs_.size());
        for (uint32_t i = 0; i < order.size(); ++i) order[i] = i;
        std::stable_sort(order.begin(), order.end(), [&](uint32_t x, uint32_t y) { return graphs_[x]->m < graphs_[y]->m; });
        for (uint32_t r = 0; r < order.size(); ++r) prio[order[r]] = std::min(least, greatest + (int)r);
    }
    for (uint32_t gi = 0; gi < graphs_.size(); ++gi) {
        ServedGraph& G = *graphs_[gi];
        const uint64_t n = G.n;
        // result pool: grown, or shrunk by its free buffers, to results_per_graph
        // (buffers of results not yet collected survive a stop / start)
        while (G.all_results.size() < o.results_per_graph) {
            uint32_t* b = (uint32_t*)dalloc(4 * n);
            G.all_results.push_back(b);
            G.free_results.push_back(b);
        }
        while (G.all_results.size() > o.results_per_graph && !G.free_results.empty()) {
            uint32_t* b = G.free_results.back();
            G.free_results.pop_back();
            G.all_results.erase(std::find(G.all_results.begin(), G.all_results.end(), b));
            dfree(b, 4 * n);
        }
        if (!G.lanes[GXP_QUERY_PPR]) {   // lanes are allocated once
            for (int k = 0; k < 2; ++k) {
                if (k == GXP_QUERY_SSSP && !G.weighted) continue;
                auto L = std::make_unique<Lane>();
                L->graph = gi;
                L->kind = (gxp_query_kind)k;
                cuda_check(cudaStreamCreateWithPriority(&L->stream, cudaStreamNonBlocking, prio[gi]),
                           "cudaStreamCreate");
                L->prio = prio[gi];
                cuda_check(cudaMallocHost(&L->h_table, 128 * 4), "cudaMallocHost");
                cuda_check(cudaMallocHost(&L->h_improved, 2 * 4), "cudaMallocHost");
                L->d_slot_source = (uint32_t*)dalloc(64 * 4);
                L->d_slot_damping = (float*)dalloc(64 * 4);
                cuda_check(cudaMemset(L->d_slot_source, 0, 64 * 4), "memset");
                cuda_check(cudaMemset(L->d_slot_damping, 0, 64 * 4), "memset");
                if (k == GXP_QUERY_SSSP) {
                    const size_t words = (n + 31) / 32 + 1;
                    L->d_dist = (uint32_t*)dalloc(256 * n);
                    cuda_check(cudaMemset(L->d_dist, 0xFF, 256 * n), "memset");
                    for (auto& f : L->d_frontier) {
                        f = (uint32_t*)dalloc(4 * words);
                        cuda_check(cudaMemset(f, 0, 4 * words), "memset");
                    }
                    L->d_improved = (uint32_t*)dalloc(8);
                    L->d_changed = (unsigned long long*)dalloc(8);
                } else {
                    for (auto& mm : L->d_msg) {
                        mm = (float*)dalloc(256 * n);
                        cuda_check(cudaMemset(mm, 0, 256 * n), "memset");
                    }
                    L->d_rank = (float*)dalloc(256 * n);
                    cuda_check(cudaMemset(L->d_rank, 0, 256 * n), "memset");
                    L->d_partial = (float*)dalloc(256 * std::max<uint64_t>(G.n_partials, 1));
                    for (auto& dg : L->d_dang) {
                        dg = (unsigned long long*)dalloc(64 * 8);
                        cuda_check(cudaMemset(dg, 0, 64 * 8), "memset");
                    }
                }
                G.lanes[k] = std::move(L);
            }
        }
        for (auto& L : G.lanes)
            if (L) {
                L->max_slots = o.max_slots;
                if (L->prio != prio[gi]) {   // stream priority is fixed at creation
                    cuda_check(cudaStreamSynchronize(L->stream), "stream");
                    cuda_check(cudaStreamDestroy(L->stream), "stream");
                    L->stream = nullptr;
                    cuda_check(cudaStreamCreateWithPriority(&L->stream, cudaStreamNonBlocking, prio[gi]),
                               "cudaStreamCreate");
                    L->prio = prio[gi];
                }
            }
    }
    cuda_check(cudaDeviceSynchronize(), "serve start");
    {
        std::lock_guard<std::mutex> lk(mu_);
        stopping_ = false;
        error_ = GXP_OK;
        running_ = true;
    }
    for (auto& g : graphs_)
        for (auto& L : g->lanes)
            if (L) {
                Lane* lp = L.get();
                L->thread = std::thread([this, lp] { lane_loop(*lp); });
            }
}

void Server::stop() {
    {
        std::lock_guard<std::mutex> lk(mu_);
        if (!running_) return;
        stopping_ = true;
        for (auto& g : graphs_)
            for (auto& L : g->lanes)
                if (L) L->cv.notify_all();
    }
    for (auto& g : graphs_)
        for (auto& L : g->lanes)
            if (L && L->thread.joinable()) L->thread.join();
    std::lock_guard<std::mutex> lk(mu_);
    for (auto& g : graphs_)
        for (auto& L : g->lanes)
            if (L) fail_lane(*L, GXP_E_STATE);
    running_ = false;
    cv_done_.notify_all();
}

// called with mu_ held: every queued or running query of the lane fails
void Server::fail_lane(Lane& L, gxp_status code) {
    ServedGraph& G = *graphs_[L.graph];
    auto fail_q = [&](Query* q) {
        if (q->d_result) {
            G.free_results.push_back(q->d_result);
            q->d_result = nullptr;
        }
        q->state = GXP_QUERY_FAILED;
        q->status = code;
        q->t_done = now();
        done_fifo_.push_back(q->id);
        ++n_failed_;
    };
    for (int s = 0; s < 64; ++s)
        if (L.slot_q[s]) {
            fail_q(L.slot_q[s]);
            L.slot_q[s] = nullptr;
        }
    L.busy = 0;
    for (uint64_t id : L.queue) {
        auto it = queries_.find(id);
        if (it != queries_.end()) fail_q(it->second.get());
        --queued_;
    }
    L.queue.clear();
}

// ------------------------------------------------------------------ lanes

void Server::lane_loop(Lane& L) {
    if (cudaSetDevice(device_) != cudaSuccess) {
        std::lock_guard<std::mutex> lk(mu_);
        error_ = GXP_E_CUDA;
        fail_lane(L, GXP_E_CUDA);
        cv_done_.notify_all();
        return;
    }
    ServedGraph& G = *graphs_[L.graph];
    const uint64_t slot_cap = L.max_slots == 64 ? ~0ull : ((1ull << L.max_slots) - 1ull);
    for (;;) {
        uint64_t admit = 0;
        {
            std::unique_lock<std::mutex> lk(mu_);
            L.cv.wait(lk, [&] {
                if (stopping_ || error_ != GXP_OK) return true;
                const bool can_admit = !L.queue.empty() && !G.free_results.empty() && (L.busy & slot_cap) != slot_cap;
                return L.busy != 0 || can_admit;
            });
            if (stopping_) return;   // stop() fails what is left
            if (error_ != GXP_OK) {  // another lane hit a device error
                fail_lane(L, GXP_E_STATE);
                cv_done_.notify_all();
                return;
            }
            const double t = now();
            while (!L.queue.empty() && !G.free_results.empty() && (L.busy & slot_cap) != slot_cap) {
                const int s = __builtin_ctzll(~L.busy & slot_cap);
                Query* q = queries_.at(L.queue.front()).get();
                L.queue.pop_front();
                --queued_;
                q->d_result = G.free_results.back();
                G.free_results.pop_back();
                q->state = GXP_QUERY_RUNNING;
                q->t_admit = t;
                L.slot_q[s] = q;
                L.slot_steps[s] = 0;
                L.busy |= 1ull << s;
                admit |= 1ull << s;
                L.h_table[s] = q->source;
                std::memcpy(&L.h_table[64 + s], &q->damping, 4);
            }
        }
        try {
            lane_step(L, G, admit);
        } catch (const Error& e) {
            std::lock_guard<std::mutex> lk(mu_);
            if (error_ == GXP_OK) error_ = e.code;
            fail_lane(L, e.code);
            cv_done_.notify_all();
            for (auto& g : graphs_)
                for (auto& other : g->lanes)
                    if (other) other->cv.notify_all();
            return;
        }
    }
}

// One superstep of a lane: initialise admitted slots, advance every busy
// slot, retire finished ones. Only this lane's thread touches its slots.
void Server::lane_step(Lane& L, ServedGraph& G, uint64_t admit) {
    TraceRange trace_("gxp serving lane superstep");
    const bool sssp = L.kind == GXP_QUERY_SSSP;
    const cudaStream_t st = L.stream;
    if (admit) {
        cuda_check(cudaMemcpyAsync(L.d_slot_source, L.h_table, 64 * 4, cudaMemcpyHostToDevice, st), "slot table");
        cuda_check(cudaMemcpyAsync(L.d_slot_damping, L.h_table + 64, 64 * 4, cudaMemcpyHostToDevice, st),
                   "slot table");
        if (sssp)
            cuda_check(launch_sssp_slots_init(L.d_dist, G.n, admit, L.d_slot_source, L.d_frontier[L.cur], st),
                       "slot init");
        else
            cuda_check(launch_ppr_slots_init(L.d_msg[L.cur], G.d_inv_outdeg, G.n, admit, L.d_slot_source,
                                             L.d_dang[L.cur], st),
                       "slot init");
    }
    const int nx = L.cur ^ 1;
    if (sssp) {
        cuda_check(cudaMemsetAsync(L.d_improved, 0, 8, st), "memset");
        MsArgs a{};
        a.units = G.d_units_nz;
        a.u_begin = 0;
        a.u_end = G.n_units_nz;
        a.edges = G.d_edges;
        a.packed = G.packed;
        a.edge_base = 0;
        a.dist = L.d_dist;
        a.frontier_cur = L.d_frontier[L.cur];
        a.frontier_next = L.d_frontier[nx];
        a.changed = L.d_changed;
        a.slot_improved = L.d_improved;
        a.idle_mask = ~L.busy;
        cuda_check(launch_msssp(a, false, serve_grid(G.n_units_nz), st), "sssp superstep");
        cuda_check(cudaMemsetAsync(L.d_frontier[L.cur], 0, 4 * ((G.n + 31) / 32 + 1), st), "memset");
        cuda_check(cudaMemcpyAsync(L.h_improved, L.d_improved, 8, cudaMemcpyDeviceToHost, st), "read flags");
    } else {
        cuda_check(cudaMemsetAsync(L.d_dang[nx], 0, 64 * 8, st), "memset");
        PprArgs a{};
        a.units = G.d_units_all;
        a.n_units = G.n_units_all;
        a.src = G.d_src;
        a.split_rows = G.d_split_rows;
        a.n_split_rows = G.n_split_rows;
        a.inv_outdeg = G.d_inv_outdeg;
        a.msg_cur = L.d_msg[L.cur];
        a.msg_nxt = L.d_msg[nx];
        a.rank = L.d_rank;
        a.partial = L.d_partial;
        a.dang_cur = L.d_dang[L.cur];
        a.dang_next = L.d_dang[nx];
        a.slot_damping = L.d_slot_damping;
        a.slot_source = L.d_slot_source;
        a.active_mask = L.busy;
        for (uint64_t b = L.busy; b; b &= b - 1) {   // slots whose last superstep this is
            const int s = __builtin_ctzll(b);
            if (L.slot_steps[s] + 1 >= L.slot_q[s]->iters) a.finish_mask |= 1ull << s;
        }
        cuda_check(launch_ppr_superstep(a, st), "ppr superstep");
    }
    L.cur = nx;
    cuda_check(cudaStreamSynchronize(st), "superstep");

    // slot_steps and slot_q belong to this thread; the query records are shared
    GatherList gl{};
    for (uint64_t b = L.busy; b; b &= b - 1) {
        const int s = __builtin_ctzll(b);
        ++L.slot_steps[s];
        bool fin;
        if (sssp) fin = !((L.h_improved[s >> 5] >> (s & 31)) & 1u);   // nothing of the slot improved
        else fin = L.slot_steps[s] >= L.slot_q[s]->iters;
        if (fin) {
            gl.slot[gl.n] = (uint32_t)s;
            gl.out[gl.n] = L.slot_q[s]->d_result;
            ++gl.n;
        }
    }
    if (gl.n) {
        const uint32_t* mat = sssp ? L.d_dist : reinterpret_cast<const uint32_t*>(L.d_rank);
        cuda_check(launch_gather_columns(mat, G.n, gl, st), "gather results");
        cuda_check(cudaStreamSynchronize(st), "gather results");
    }
    std::lock_guard<std::mutex> lk(mu_);
    ++L.supersteps;
    for (uint64_t b = L.busy; b; b &= b - 1) ++L.slot_q[__builtin_ctzll(b)]->supersteps;
    if (gl.n == 0) return;
    const double t = now();
    for (uint32_t j = 0; j < gl.n; ++j) {
        const int s = (int)gl.slot[j];
        Query* q = L.slot_q[s];
        q->state = GXP_QUERY_DONE;
        q->t_done = t;
        done_fifo_.push_back(q->id);
        ++n_completed_;
        L.slot_q[s] = nullptr;
        L.busy &= ~(1ull << s);
    }
    cv_done_.notify_all();
}

// ---------------------------------------------------------------- queries

uint64_t Server::submit(uint32_t graph, gxp_query_kind kind, uint32_t source, float damping, uint32_t iters) {
    std::unique_lock<std::mutex> lk(mu_);
    if (!running_ || stopping_) fail(GXP_E_STATE, "server not started");
    if (error_ != GXP_OK) fail(GXP_E_STATE, "server stopped by an earlier device error");
    if (graph >= graphs_.size()) fail(GXP_E_INVAL, "no such graph");
    if (kind != GXP_QUERY_SSSP && kind != GXP_QUERY_PPR) fail(GXP_E_INVAL, "unknown query kind");
    ServedGraph& G = *graphs_[graph];
    if (source >= G.n) fail(GXP_E_INVAL, "source out of range");
    if (kind == GXP_QUERY_SSSP && !G.lanes[GXP_QUERY_SSSP]) fail(GXP_E_UNSUPPORTED, "SSSP needs a weighted graph");
    if (kind == GXP_QUERY_PPR && !(damping >= 0.0f && damping < 1.0f)) fail(GXP_E_INVAL, "damping must be in [0, 1)");
    if (queued_ >= queue_cap_) fail(GXP_E_BUSY, "admission queue full");
    auto q = std::make_unique<Query>();
    q->id = next_id_++;
    q->graph = graph;
    q->kind = kind;
    q->source = source;
    q->damping = kind == GXP_QUERY_PPR ? damping : 0.0f;
    q->iters = kind == GXP_QUERY_PPR ? (iters ? iters : kDefaultIters) : 0u;
    q->t_submit = now();
    const uint64_t id = q->id;
    queries_.emplace(id, std::move(q));
    Lane& L = *G.lanes[kind];
    L.queue.push_back(id);
    ++queued_;
    ++n_submitted_;
    L.cv.notify_one();
    return id;
}

bool Server::poll(uint64_t qid, void* out, uint64_t cap, int timeout_ms) {
    std::unique_lock<std::mutex> lk(mu_);
    auto find = [&]() -> Query* {
        auto it = queries_.find(qid);
        if (it == queries_.end()) fail(GXP_E_INVAL, "unknown query id (never submitted or already collected)");
        return it->second.get();
    };
    Query* q = find();
    auto finished = [&] { return q->state == GXP_QUERY_DONE || q->state == GXP_QUERY_FAILED; };
    if (!finished() && timeout_ms != 0) {
        if (timeout_ms < 0) {
            cv_done_.wait(lk, [&] { return (q = find(), finished()); });
        } else {
            cv_done_.wait_for(lk, std::chrono::milliseconds(timeout_ms), [&] { return (q = find(), finished()); });
        }
    }
    if (!finished()) return false;
    ServedGraph& G = *graphs_[q->graph];
    if (q->state == GXP_QUERY_FAILED) {
        const gxp_status code = q->status;
        if (out) queries_.erase(qid);
        fail(code, "query failed");
    }
    if (!out) return true;
    if (cap < G.n) fail(GXP_E_INVAL, "cap is smaller than the result (n_vertices)");
    if (q->collecting) fail(GXP_E_INVAL, "the result is being collected by another call");
    q->collecting = true;
    uint32_t* res = q->d_result;
    const uint64_t bytes = 4 * G.n;
    lk.unlock();   // the copy runs without the lock; the query stays until it ends
    cudaStream_t cs = nullptr;
    {
        std::lock_guard<std::mutex> cl(copy_mu_);
        if (!copy_streams_.empty()) {
            cs = copy_streams_.back();
            copy_streams_.pop_back();
        }
    }
    cudaError_t err = cudaSetDevice(device_);
    if (err == cudaSuccess && !cs) err = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
    if (err == cudaSuccess) err = cudaMemcpyAsync(out, res, bytes, cudaMemcpyDefault, cs);
    if (err == cudaSuccess) err = cudaStreamSynchronize(cs);
    if (cs) {
        std::lock_guard<std::mutex> cl(copy_mu_);
        copy_streams_.push_back(cs);
    }
    lk.lock();
    if (err != cudaSuccess) {
        q->collecting = false;   // the result stays; the caller may try again
        lk.unlock();
        cuda_check(err, "copy result");
    }
    auto it = queries_.find(qid);
    if (it != queries_.end()) {
        G.free_results.push_back(it->second->d_result);
        queries_.erase(it);
        Lane* L = G.lanes[GXP_QUERY_SSSP] ? G.lanes[GXP_QUERY_SSSP].get() : nullptr;
        if (L) L->cv.notify_one();
        if (G.lanes[GXP_QUERY_PPR]) G.lanes[GXP_QUERY_PPR]->cv.notify_one();
    }
    return true;
}

uint64_t Server::next_done(int timeout_ms) {
    std::unique_lock<std::mutex> lk(mu_);
    auto ready = [&] {
        while (!done_fifo_.empty()) {   // skip ids collected by poll in the meantime
            auto it = queries_.find(done_fifo_.front());
            if (it != queries_.end() && !it->second->reported) return true;
            done_fifo_.pop_front();
        }
        return false;
    };
    if (timeout_ms < 0) cv_done_.wait(lk, ready);
    else if (!ready()) cv_done_.wait_for(lk, std::chrono::milliseconds(timeout_ms), ready);
    if (!ready()) return 0;
    const uint64_t id = done_fifo_.front();
    done_fifo_.pop_front();
    queries_.at(id)->reported = true;
    return id;
}

void Server::info(uint64_t qid, gxp_query_info* out) {
    std::lock_guard<std::mutex> lk(mu_);
    auto it = queries_.find(qid);
    if (it == queries_.end()) fail(GXP_E_INVAL, "unknown query id (never submitted or already collected)");
    const Query& q = *it->second;
    *out = gxp_query_info{};
    out->state = q.state;
    out->supersteps = q.supersteps;
    out->graph = q.graph;
    out->kind = q.kind;
    out->n_values = graphs_[q.graph]->n;
    if (q.state != GXP_QUERY_QUEUED && q.t_admit > 0) out->queue_ms = 1e3 * (q.t_admit - q.t_submit);
    if (q.state == GXP_QUERY_DONE) out->run_ms = 1e3 * (q.t_done - q.t_admit);
}

void Server::report(gxp_serve_report* out) {
    std::lock_guard<std::mutex> lk(mu_);
    *out = gxp_serve_report{};
    out->submitted = n_submitted_;
    out->completed = n_completed_;
    out->failed = n_failed_;
    out->queued = queued_;
    for (auto& g : graphs_)
        for (auto& L : g->lanes)
            if (L) {
                out->running += (uint64_t)__builtin_popcountll(L->busy);
                (L->kind == GXP_QUERY_SSSP ? out->sssp_supersteps : out->ppr_supersteps) += L->supersteps;
            }
    out->device_bytes = bytes_;
}

}  // namespace gxp
