// Batched multi-source SSSP with the pipeline shuffle (Section III-A,
// Algorithms 1-2) and the block-size autotuner (Lemma 1).
//
// Edge blocks are contiguous runs of work units (a destination's in-edges, at
// most kUnitEdges per unit) in destination order. When the edges are streamed
// from pinned host memory, block i moves through three stages on three
// streams: download (H2D copy into ring slot i mod 3), compute (the superstep
// kernel on that slot), upload (D2H of the block's changed-unit counter).
// Rotating n -> c -> u is the slot index advancing: no data is copied between
// stages. A whole superstep can be captured once into a CUDA graph and
// replayed.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <string>

#include "engine.hpp"
#include "trace.hpp"

namespace gxp {

namespace {

void destroy_graph(cudaGraphExec_t& g) {
    if (g) cudaGraphExecDestroy(g);
    g = nullptr;
}

}  // namespace

void Engine::free_batch() {
    Batch& b = batch_;
    if (b.s_h2d) cudaStreamSynchronize(b.s_h2d);
    if (b.s_d2h) cudaStreamSynchronize(b.s_d2h);
    destroy_graph(b.graph[0]);
    destroy_graph(b.graph[1]);
    if (b.h_edges) cudaFreeHost(b.h_edges);
    if (b.h_changed) cudaFreeHost(b.h_changed);
    for (int i = 0; i < 3; ++i) {
        if (b.ev_loaded[i]) cudaEventDestroy(b.ev_loaded[i]);
        if (b.ev_free[i]) cudaEventDestroy(b.ev_free[i]);
    }
    if (b.ev_t0) cudaEventDestroy(b.ev_t0);
    if (b.ev_t1) cudaEventDestroy(b.ev_t1);
    if (b.s_h2d) cudaStreamDestroy(b.s_h2d);
    if (b.s_d2h) cudaStreamDestroy(b.s_d2h);
    // device buffers belong to graph_allocs_ and are freed with the graph
    batch_ = Batch{};
}

void Engine::prepare_batch(bool streamed) {
    if (!have_graph_) fail(GXP_E_STATE, "no graph");
    if (n_parts_ != 1) fail(GXP_E_UNSUPPORTED, "batched SSSP runs on a single-partition graph");
    if (!finalized_) finalize();
    if (!weighted_) fail(GXP_E_INVAL, "SSSP needs edge weights");
    Batch& b = batch_;
    HostPart& hp = parts_[0];
    ensure_host(hp);
    const uint64_t V = n_vertices_, E = hp.src.size();
    if (!b.ready) {
        b.units.clear();
        b.unit_edge.clear();
        for (uint32_t v = 0; v < hp.n_own; ++v) {
            const uint32_t e0 = hp.col_ptr[v], d = hp.col_ptr[v + 1] - e0;
            for (uint32_t k = 0; k < d; k += kUnitEdges) {
                b.units.push_back(make_uint4(v, e0 + k, std::min<uint32_t>(kUnitEdges, d - k), d > kUnitEdges ? 1u : 0u));
                b.unit_edge.push_back(e0 + k);
            }
        }
        b.unit_edge.push_back(E);
        // streamed edges are packed into 4 bytes when they fit (the stream is
        // bound by the host link); resident edges stay 8 bytes (the kernel is
        // bound by instruction issue, and unpacking costs more than it saves)
        uint32_t wmax = 0;
        for (uint32_t x : hp.w) wmax = std::max(wmax, x);
        b.packed = packable(V, wmax);
        b.esize = b.packed ? 4u : 8u;
        b.d_units = (uint4*)dalloc(sizeof(uint4) * std::max<size_t>(b.units.size(), 1));
        if (!b.units.empty()) {
            before_h2d("upload units");
            cuda_check(cudaMemcpy(b.d_units, b.units.data(), sizeof(uint4) * b.units.size(), cudaMemcpyHostToDevice),
                       "upload units");
        }
        b.d_dist = (uint32_t*)dalloc(sizeof(uint32_t) * 64 * V);
        const size_t words = (V + 31) / 32 + 1;
        b.d_frontier[0] = (uint32_t*)dalloc(4 * words);
        b.d_frontier[1] = (uint32_t*)dalloc(4 * words);
        b.d_frontier[2] = (uint32_t*)dalloc(4 * words);
        b.d_loop_changed = (unsigned long long*)dalloc(8 * 4);
        b.d_bar = (GridBar*)dalloc(sizeof(GridBar));
        b.d_steps = (uint32_t*)dalloc(4);
        b.d_sources = (uint32_t*)dalloc(4 * 64);
        cuda_check(cudaStreamCreateWithFlags(&b.s_h2d, cudaStreamNonBlocking), "stream");
        cuda_check(cudaStreamCreateWithFlags(&b.s_d2h, cudaStreamNonBlocking), "stream");
        for (int i = 0; i < 3; ++i) {
            cuda_check(cudaEventCreateWithFlags(&b.ev_loaded[i], cudaEventDisableTiming), "event");
            cuda_check(cudaEventCreateWithFlags(&b.ev_free[i], cudaEventDisableTiming), "event");
        }
        cuda_check(cudaEventCreate(&b.ev_t0), "event");
        cuda_check(cudaEventCreate(&b.ev_t1), "event");
        b.ready = true;
    }
    auto fill = [&](void* dst, bool packed) {
        if (packed) {
            uint32_t* d = static_cast<uint32_t*>(dst);
            for (uint64_t e = 0; e < E; ++e) d[e] = hp.w[e] << kPackSrcBits | hp.src[e];
        } else {
            uint2* d = static_cast<uint2*>(dst);
            for (uint64_t e = 0; e < E; ++e) d[e] = make_uint2(hp.src[e], hp.w[e]);
        }
    };
    const size_t ebytes = (size_t)b.esize * E;
    if (streamed && !b.pinned_ready) {
        cuda_check(cudaHostAlloc(&b.h_edges, std::max<size_t>(ebytes, 8), cudaHostAllocDefault), "pinned edge buffer");
        fill(b.h_edges, b.packed);
        b.pinned_ready = true;
    }
    if (!streamed && !b.resident) {
        b.d_edges = dalloc(std::max<size_t>(8 * E, 8));
        std::vector<uint2> tmp(E);
        fill(tmp.data(), false);
        before_h2d("upload");
        cuda_check(cudaMemcpy(b.d_edges, tmp.data(), 8 * E, cudaMemcpyHostToDevice), "upload edges");
        b.resident = true;
    }
}

// Unit-index cuts of edge blocks of about `block_edges` edges each.
std::vector<uint64_t> Engine::block_cuts(uint64_t block_edges) const {
    const Batch& b = batch_;
    std::vector<uint64_t> cuts{0};
    const uint64_t n = b.units.size();
    uint64_t start = 0;
    while (start < n) {
        const uint64_t target = b.unit_edge[start] + std::max<uint64_t>(block_edges, 1);
        uint64_t end = std::upper_bound(b.unit_edge.begin() + start, b.unit_edge.end() - 1, target - 1) - b.unit_edge.begin();
        end = std::max<uint64_t>(end, start + 1);
        end = std::min<uint64_t>(end, n);
        cuts.push_back(end);
        start = end;
    }
    return cuts;
}

// One superstep over all edge blocks (enqueued on stream_, the other two
// streams forked from and joined back into it).
void Engine::superstep_batch(const std::vector<uint64_t>& cuts, bool streamed, bool pipelined, bool dry, int parity) {
    TraceRange trace_("gxp batched superstep (pipeline shuffle)");
    Batch& b = batch_;
    const size_t nb = cuts.size() - 1;
    const uint64_t words = (n_vertices_ + 31) / 32 + 1;
    uint32_t* fr_cur = b.d_frontier[parity];
    uint32_t* fr_next = b.d_frontier[parity ^ 1];
    if (!dry) cuda_check(cudaMemsetAsync(fr_next, 0, 4 * words, stream_), "memset");
    cuda_check(cudaMemsetAsync(b.d_changed, 0, 8 * std::max<size_t>(nb, 1), stream_), "memset");
    MsArgs a{};
    a.units = b.d_units;
    a.packed = streamed && b.packed;
    a.dist = b.d_dist;
    a.frontier_cur = fr_cur;
    a.frontier_next = fr_next;
    a.active = dry ? nullptr : b.d_active;
    if (!streamed) {
        a.u_begin = 0;
        a.u_end = b.units.size();
        a.edges = b.d_edges;
        a.edge_base = 0;
        a.changed = b.d_changed;
        cuda_check(launch_msssp(a, dry, msssp_grid(b.units.size()), stream_), "batch kernel");
        cuda_check(cudaMemcpyAsync(b.h_changed, b.d_changed, 8, cudaMemcpyDeviceToHost, stream_), "upload");
        return;
    }
    // fork the download and upload streams off the compute stream
    cudaEvent_t fork = b.ev_loaded[0];
    cuda_check(cudaEventRecord(b.ev_free[0], stream_), "event");
    cuda_check(cudaStreamWaitEvent(b.s_h2d, b.ev_free[0], 0), "wait");
    cuda_check(cudaStreamWaitEvent(b.s_d2h, b.ev_free[0], 0), "wait");
    (void)fork;
    for (size_t i = 0; i < nb; ++i) {
        const int slot = (int)(i % 3);
        const uint64_t e0 = b.unit_edge[cuts[i]], e1 = b.unit_edge[cuts[i + 1]];
        // download (n): wait until the compute that last used this slot is done
        if (i >= 3 || !pipelined) {
            if (i >= 1) cuda_check(cudaStreamWaitEvent(b.s_h2d, b.ev_free[pipelined ? slot : (int)((i - 1) % 3)], 0), "wait");
        }
        cuda_check(cudaMemcpyAsync(b.d_ring[slot], static_cast<const char*>(b.h_edges) + (size_t)b.esize * e0,
                                   (size_t)b.esize * (e1 - e0), cudaMemcpyHostToDevice, b.s_h2d), "download block");
        cuda_check(cudaEventRecord(b.ev_loaded[slot], b.s_h2d), "event");
        // compute (c)
        cuda_check(cudaStreamWaitEvent(stream_, b.ev_loaded[slot], 0), "wait");
        a.u_begin = cuts[i];
        a.u_end = cuts[i + 1];
        a.edges = b.d_ring[slot];
        a.edge_base = e0;
        a.changed = b.d_changed + i;
        cuda_check(launch_msssp(a, dry, msssp_grid(cuts[i + 1] - cuts[i]), stream_), "batch kernel");
        cuda_check(cudaEventRecord(b.ev_free[slot], stream_), "event");
        // upload (u): the block's changed-unit counter
        cuda_check(cudaStreamWaitEvent(b.s_d2h, b.ev_free[slot], 0), "wait");
        cuda_check(cudaMemcpyAsync(b.h_changed + i, b.d_changed + i, 8, cudaMemcpyDeviceToHost, b.s_d2h), "upload");
    }
    // join
    cuda_check(cudaEventRecord(b.ev_loaded[1], b.s_h2d), "event");
    cuda_check(cudaStreamWaitEvent(stream_, b.ev_loaded[1], 0), "wait");
    cuda_check(cudaEventRecord(b.ev_loaded[2], b.s_d2h), "event");
    cuda_check(cudaStreamWaitEvent(stream_, b.ev_loaded[2], 0), "wait");
}

// Device time of one superstep at `block_edges` (median of reps), on the
// current dist/frontier contents.
double Engine::time_pipeline(uint64_t block_edges, bool pipelined, bool dry, int reps) {
    Batch& b = batch_;
    const auto cuts = block_cuts(block_edges);
    uint64_t max_block = 0;
    for (size_t i = 0; i + 1 < cuts.size(); ++i)
        max_block = std::max<uint64_t>(max_block, b.unit_edge[cuts[i + 1]] - b.unit_edge[cuts[i]]);
    if (max_block > b.ring_edges || cuts.size() - 1 > b.max_blocks)
        fail(GXP_E_STATE, "ring or counters too small for the timed block size");
    std::vector<float> t;
    for (int r = 0; r < reps + 1; ++r) {
        cuda_check(cudaEventRecord(b.ev_t0, stream_), "event");
        superstep_batch(cuts, true, pipelined, dry, 0);
        cuda_check(cudaEventRecord(b.ev_t1, stream_), "event");
        cuda_check(cudaEventSynchronize(b.ev_t1), "sync");
        float ms = 0;
        cuda_check(cudaEventElapsedTime(&ms, b.ev_t0, b.ev_t1), "elapsed");
        if (r > 0) t.push_back(ms);   // the first run warms up
    }
    std::sort(t.begin(), t.end());
    return t[t.size() / 2];
}

void Engine::sssp_batch(const uint32_t* sources, uint32_t n_src, uint32_t* dist_out, const gxp_batch_opts* opts_in,
                        gxp_batch_report* rep) {
    TraceRange trace_("gxp batched SSSP");
    gxp_batch_opts opts{};
    if (opts_in) opts = *opts_in;
    if (n_src == 0 || n_src > 64) fail(GXP_E_INVAL, "n_sources must be in [1, 64]");
    if (!sources) fail(GXP_E_INVAL, "null sources");
    std::vector<uint32_t> src(n_src);
    copy_in(src.data(), sources, 4ull * n_src);
    for (uint32_t s : src)
        if (s >= n_vertices_) fail(GXP_E_INVAL, "source out of range");
    const bool streamed = opts.streamed != 0;
    const bool pipelined = !streamed || opts.pipelined != 0;
    prepare_batch(streamed);
    Batch& b = batch_;
    const uint64_t E = b.unit_edge.back(), V = n_vertices_;
    const uint64_t words = (V + 31) / 32 + 1;
    gxp_batch_report r{};
    r.edges_per_superstep = E;

    // block size: given, or Lemma 1 from measured coefficients + a local sweep
    uint64_t block_edges = E;
    if (streamed) {
        const uint64_t sample = std::min<uint64_t>(std::max<uint64_t>(E, 1), 1ull << 24);
        auto ensure = [&](uint64_t ring, size_t blocks) {
            if (ring > b.ring_edges) {
                for (int i = 0; i < 3; ++i) b.d_ring[i] = dalloc((size_t)b.esize * ring);
                b.ring_edges = ring;
            }
            if (blocks > b.max_blocks) {
                b.d_changed = (unsigned long long*)dalloc(8 * blocks);
                if (b.h_changed) cudaFreeHost(b.h_changed);
                cuda_check(cudaHostAlloc((void**)&b.h_changed, 8 * blocks, cudaHostAllocDefault), "pinned counters");
                b.max_blocks = blocks;
            }
        };
        // the tune cache's key: the graph's shape, the streamed edge size and the GPU
        std::string tune_key;
        gxp_tune_record cached{};
        bool from_cache = false;
        if (!opts.block_edges && opts.tune_cache) {
            cudaDeviceProp prop{};
            cuda_check(cudaGetDeviceProperties(&prop, device_), "device properties");
            const double deg = V ? (double)E / (double)V : 0.0;
            tune_key = "sssp_batch V=" + std::to_string(V) + " E=" + std::to_string(E) +
                       " deg=" + std::to_string(deg >= 1.0 ? (int)std::floor(std::log2(deg)) : 0) +
                       " esize=" + std::to_string(b.esize) + " gpu=" + prop.name;
            from_cache = tune_cache_get(opts.tune_cache, tune_key.c_str(), &cached) && cached.block_edges >= 1.0;
        }
        if (opts.block_edges) {
            block_edges = opts.block_edges;
        } else if (from_cache) {
            r.k1 = cached.k1;
            r.k2 = cached.k2;
            r.k3 = cached.k3;
            r.a = cached.a;
            r.model_block_edges = cached.model_block_edges;
            r.sweep_best_ms = cached.sweep_best_ms;
            r.tune_from_cache = 1;
            block_edges = (uint64_t)cached.block_edges;
        } else {
            ensure(sample + kUnitEdges, 64);
            // k1: download cost per edge (pinned H2D)
            cudaEvent_t t0 = b.ev_t0, t1 = b.ev_t1;
            float best = 1e30f;
            for (int i = 0; i < 3; ++i) {
                cuda_check(cudaEventRecord(t0, stream_), "event");
                cuda_check(cudaMemcpyAsync(b.d_ring[0], b.h_edges, (size_t)b.esize * sample, cudaMemcpyHostToDevice,
                                           stream_), "copy");
                cuda_check(cudaEventRecord(t1, stream_), "event");
                cuda_check(cudaEventSynchronize(t1), "sync");
                float ms;
                cuda_check(cudaEventElapsedTime(&ms, t0, t1), "elapsed");
                best = std::min(best, ms);
            }
            r.k1 = best / (double)sample;
            // k2: compute cost per edge at full load (every source active, dist 0)
            cuda_check(cudaMemsetAsync(b.d_dist, 0, sizeof(uint32_t) * 64 * V, stream_), "memset");
            cuda_check(cudaMemsetAsync(b.d_frontier[0], 0xFF, 4 * words, stream_), "memset");
            const auto cuts_s = block_cuts(sample);
            MsArgs a{};
            a.units = b.d_units;
            a.packed = b.packed;
            a.u_begin = 0;
            a.u_end = cuts_s[1];
            a.edges = b.d_ring[0];
            a.edge_base = 0;
            a.dist = b.d_dist;
            a.frontier_cur = b.d_frontier[0];
            a.frontier_next = b.d_frontier[1];
            a.changed = b.d_changed;
            const uint64_t e_s = b.unit_edge[cuts_s[1]];
            best = 1e30f;
            for (int i = 0; i < 4; ++i) {
                cuda_check(cudaEventRecord(t0, stream_), "event");
                cuda_check(launch_msssp(a, true, msssp_grid(cuts_s[1]), stream_), "kernel");
                cuda_check(cudaEventRecord(t1, stream_), "event");
                cuda_check(cudaEventSynchronize(t1), "sync");
                float ms;
                cuda_check(cudaEventElapsedTime(&ms, t0, t1), "elapsed");
                if (i) best = std::min(best, ms);
            }
            r.k2 = best / (double)std::max<uint64_t>(e_s, 1);
            // a: fixed cost of a block (copy + launch + upload) from 32 near-empty blocks
            ensure(sample + kUnitEdges, 64);
            {
                std::vector<uint64_t> tiny{0};
                for (uint64_t i = 1; i <= 32 && i <= b.units.size(); ++i) tiny.push_back(i);
                std::vector<float> ts;
                for (int rep_i = 0; rep_i < 3; ++rep_i) {
                    cuda_check(cudaEventRecord(t0, stream_), "event");
                    superstep_batch(tiny, true, false, true, 0);
                    cuda_check(cudaEventRecord(t1, stream_), "event");
                    cuda_check(cudaEventSynchronize(t1), "sync");
                    float ms;
                    cuda_check(cudaEventElapsedTime(&ms, t0, t1), "elapsed");
                    ts.push_back(ms);
                }
                std::sort(ts.begin(), ts.end());
                r.a = ts[1] / (double)std::max<size_t>(tiny.size() - 1, 1);
            }
            r.k3 = 0.0;   // the upload stage moves 8 bytes per block: part of a
            uint64_t bm = 0, sm = 0;
            double tm = 0;
            block_size_model(r.k1, r.k2, r.k3, r.a, std::max<uint64_t>(E, 2), &bm, &sm, &tm);
            r.model_block_edges = (double)bm;
            r.model_ms = tm;
            // local sweep around the model's block count
            std::vector<uint64_t> cands;
            for (double f : {0.5, 1.0, 2.0}) {
                const uint64_t s = std::max<uint64_t>(2, (uint64_t)std::llround((double)sm * f));
                cands.push_back((E + s - 1) / s);
            }
            cands.push_back(bm);
            std::sort(cands.begin(), cands.end());
            cands.erase(std::unique(cands.begin(), cands.end()), cands.end());
            double best_t = 1e300;
            for (uint64_t c : cands) {
                const auto cc = block_cuts(c);
                uint64_t mx = 0;
                for (size_t i = 0; i + 1 < cc.size(); ++i) mx = std::max<uint64_t>(mx, b.unit_edge[cc[i + 1]] - b.unit_edge[cc[i]]);
                ensure(mx, cc.size());
                const double t = time_pipeline(c, true, true, 2);
                if (t < best_t) {
                    best_t = t;
                    block_edges = c;
                }
            }
            r.sweep_best_ms = best_t;
            if (opts.tune_cache) {
                const gxp_tune_record rec{r.k1, r.k2, r.k3, r.a, r.model_block_edges, (double)block_edges, best_t};
                if (!tune_cache_put(opts.tune_cache, tune_key.c_str(), rec))
                    fail(GXP_E_INVAL, std::string("cannot write the tune cache ") + opts.tune_cache);
            }
        }
    }
    const auto cuts = streamed ? block_cuts(block_edges) : std::vector<uint64_t>{0, b.units.size()};
    if (streamed) {
        uint64_t mx = 0;
        for (size_t i = 0; i + 1 < cuts.size(); ++i) mx = std::max<uint64_t>(mx, b.unit_edge[cuts[i + 1]] - b.unit_edge[cuts[i]]);
        if (mx > b.ring_edges) {
            for (int i = 0; i < 3; ++i) b.d_ring[i] = dalloc((size_t)b.esize * mx);
            b.ring_edges = mx;
        }
    }
    if (!b.d_active) b.d_active = (unsigned long long*)dalloc(8);
    if (cuts.size() - 1 > b.max_blocks || !b.d_changed) {
        const size_t nb = std::max<size_t>(cuts.size() - 1, 1);
        b.d_changed = (unsigned long long*)dalloc(8 * nb);
        if (b.h_changed) cudaFreeHost(b.h_changed);
        cuda_check(cudaHostAlloc((void**)&b.h_changed, 8 * nb, cudaHostAllocDefault), "pinned counters");
        b.max_blocks = nb;
    }
    r.block_edges = block_edges;
    r.blocks = (uint32_t)(cuts.size() - 1);

    // initial state: dist INF except each source's own slot, frontier = sources
    before_h2d("upload");
    cuda_check(cudaMemcpyAsync(b.d_sources, src.data(), 4ull * n_src, cudaMemcpyHostToDevice, stream_), "sources");
    cuda_check(cudaMemsetAsync(b.d_frontier[0], 0, 4 * words, stream_), "memset");
    cuda_check(launch_msssp_init(b.d_dist, V, b.d_sources, n_src, b.d_frontier[0], stream_), "init");

    // CUDA graphs of one superstep, one per frontier parity
    const bool use_graph = opts.use_graph != 0;
    if (use_graph && (!b.graph[0] || b.graph_block_edges != block_edges || b.graph_streamed != streamed ||
                      b.graph_pipelined != pipelined)) {
        destroy_graph(b.graph[0]);
        destroy_graph(b.graph[1]);
        cuda_check(cudaStreamSynchronize(stream_), "sync");
        for (int par = 0; par < 2; ++par) {
            cudaGraph_t g = nullptr;
            cuda_check(cudaStreamBeginCapture(stream_, cudaStreamCaptureModeThreadLocal), "begin capture");
            superstep_batch(cuts, streamed, pipelined, false, par);
            cuda_check(cudaStreamEndCapture(stream_, &g), "end capture");
            cudaError_t e = cudaGraphInstantiate(&b.graph[par], g, 0);
            cudaGraphDestroy(g);
            cuda_check(e, "instantiate");
        }
        b.graph_block_edges = block_edges;
        b.graph_streamed = streamed;
        b.graph_pipelined = pipelined;
    }

    cuda_check(cudaMemsetAsync(b.d_active, 0, 8, stream_), "memset");
    const uint32_t max_steps = opts.max_steps ? opts.max_steps : 0xFFFFFFFFu;
    // resident edges: the whole run in one persistent cooperative kernel
    // (k_msssp_loop, a grid barrier between supersteps, the changed count
    // tested on the device); streamed edges: one superstep (copies and
    // kernels of the pipeline) per launch, the changed count read between
    bool persistent = !streamed;
    if (persistent) {
        cuda_check(cudaMemsetAsync(b.d_frontier[1], 0, 4 * words, stream_), "memset");
        cuda_check(cudaMemsetAsync(b.d_loop_changed, 0, 8 * 4, stream_), "memset");
        cuda_check(cudaMemsetAsync(b.d_bar, 0, sizeof(GridBar), stream_), "memset");
        MsArgs a{};
        a.units = b.d_units;
        a.u_begin = 0;
        a.u_end = b.units.size();
        a.edges = b.d_edges;
        a.packed = 0;
        a.edge_base = 0;
        a.dist = b.d_dist;
        a.active = b.d_active;
        cuda_check(cudaEventRecord(b.ev_t0, stream_), "event");
        const cudaError_t e = launch_msssp_loop(a, b.d_frontier, b.d_loop_changed, words, max_steps, b.d_bar,
                                                cfg_.timeout_ns, faults_.timeout, d_err_, b.d_steps, stream_);
        if (e == cudaErrorNotSupported || e == cudaErrorCooperativeLaunchTooLarge) {
            cudaGetLastError();   // launch per superstep instead
            persistent = false;
        } else {
            cuda_check(e, "batch loop");
        }
    }
    if (!persistent) cuda_check(cudaEventRecord(b.ev_t0, stream_), "event");
    int parity = 0;
    uint32_t steps = 0;
    while (!persistent && steps < max_steps) {
        if (use_graph) cuda_check(cudaGraphLaunch(b.graph[parity], stream_), "graph launch");
        else superstep_batch(cuts, streamed, pipelined, false, parity);
        cuda_check(cudaStreamSynchronize(stream_), "superstep");
        unsigned long long changed = 0;
        for (size_t i = 0; i + 1 < cuts.size(); ++i) changed += b.h_changed[i];
        parity ^= 1;
        ++steps;
        if (changed == 0) break;
    }
    cuda_check(cudaEventRecord(b.ev_t1, stream_), "event");
    cuda_check(cudaEventSynchronize(b.ev_t1), "sync");
    if (persistent) {
        check_device_error();   // a grid barrier that ran out of time
        cuda_check(cudaMemcpy(&steps, b.d_steps, 4, cudaMemcpyDeviceToHost), "read steps");
    }
    float ms = 0;
    cuda_check(cudaEventElapsedTime(&ms, b.ev_t0, b.ev_t1), "elapsed");
    r.ms_total = ms;
    r.supersteps = steps;
    r.persistent = persistent ? 1u : 0u;
    unsigned long long active = 0;
    cuda_check(cudaMemcpyAsync(&active, b.d_active, 8, cudaMemcpyDeviceToHost, stream_), "read counts");
    if (dist_out)
        cuda_check(cudaMemcpy2DAsync(dist_out, 4ull * n_src, b.d_dist, 256, 4ull * n_src, V, cudaMemcpyDefault, stream_),
                   "copy distances");
    cuda_check(cudaStreamSynchronize(stream_), "copy distances");
    r.active_edges = active;
    if (rep) *rep = r;
}

}  // namespace gxp
