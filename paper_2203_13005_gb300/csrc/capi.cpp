// extern "C" entry points of libgxp.so (declared in include/gxp.h). Each one
// converts C++ errors into gxp_status; nothing throws across the ABI.
#include <new>
#include <string>

#include <memory>

#include "engine.hpp"
#include "server.hpp"

struct gxp_ctx {
    gxp::Engine eng;
    int device;
    uint64_t mem_budget;
    std::unique_ptr<gxp::Server> server;   // created by the first gxp_serve_add_graph
    gxp_ctx(int dev, const gxp_config* cfg) : eng(dev, cfg), device(dev), mem_budget(cfg ? cfg->mem_budget : 0) {}
};

namespace {

thread_local std::string g_init_error;

bool is_poisoning(gxp_status s) {
    return s == GXP_E_CUDA || s == GXP_E_TIMEOUT || s == GXP_E_BOUNDS || s == GXP_E_LOST;
}

template <class F>
gxp_status guarded(gxp_ctx* ctx, F&& f) {
    if (!ctx) return GXP_E_INVAL;
    if (ctx->eng.poisoned) {
        ctx->eng.last_error = "context unusable after an earlier device error: " + ctx->eng.last_error;
        return GXP_E_STATE;
    }
    try {
        f(ctx->eng);
        return GXP_OK;
    } catch (const gxp::Error& e) {
        ctx->eng.last_error = e.msg;
        if (is_poisoning(e.code)) ctx->eng.poisoned = true;
        return e.code;
    } catch (const std::bad_alloc&) {
        ctx->eng.last_error = "host allocation failed";
        return GXP_E_NOMEM;
    } catch (...) {
        ctx->eng.last_error = "unexpected internal error";
        return GXP_E_STATE;
    }
}

// Serving calls: thread-safe, so errors go to the calling thread's message
// (gxp_last_error(NULL)) and never poison the superstep engine.
template <class F>
gxp_status served(gxp_ctx* ctx, bool create, F&& f) {
    if (!ctx) {
        g_init_error = "null context";
        return GXP_E_INVAL;
    }
    try {
        if (!ctx->server) {
            if (!create) gxp::fail(GXP_E_STATE, "no graph added for serving");
            ctx->server = std::make_unique<gxp::Server>(ctx->device, ctx->mem_budget);
        }
        f(*ctx->server);
        return GXP_OK;
    } catch (const gxp::Error& e) {
        g_init_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        g_init_error = "host allocation failed";
        return GXP_E_NOMEM;
    } catch (...) {
        g_init_error = "unexpected internal error";
        return GXP_E_STATE;
    }
}

}  // namespace

extern "C" {

GXP_API void gxp_config_default(gxp_config* cfg) {
    if (!cfg) return;
    *cfg = gxp_config{};
}

GXP_API gxp_status gxp_init(int device, const gxp_config* cfg, gxp_ctx** out) {
    if (!out) return GXP_E_INVAL;
    *out = nullptr;
    try {
        *out = new gxp_ctx(device, cfg);
        return GXP_OK;
    } catch (const gxp::Error& e) {
        g_init_error = e.msg;
        return e.code;
    } catch (const std::bad_alloc&) {
        g_init_error = "host allocation failed";
        return GXP_E_NOMEM;
    } catch (...) {
        g_init_error = "unexpected internal error";
        return GXP_E_STATE;
    }
}

GXP_API void gxp_destroy(gxp_ctx* ctx) { delete ctx; }

GXP_API const char* gxp_status_string(gxp_status s) {
    switch (s) {
        case GXP_OK: return "GXP_OK";
        case GXP_E_INVAL: return "GXP_E_INVAL";
        case GXP_E_NOMEM: return "GXP_E_NOMEM";
        case GXP_E_CUDA: return "GXP_E_CUDA";
        case GXP_E_TIMEOUT: return "GXP_E_TIMEOUT";
        case GXP_E_BOUNDS: return "GXP_E_BOUNDS";
        case GXP_E_STATE: return "GXP_E_STATE";
        case GXP_E_UNSUPPORTED: return "GXP_E_UNSUPPORTED";
        case GXP_E_BUSY: return "GXP_E_BUSY";
        case GXP_E_LOST: return "GXP_E_LOST";
    }
    return "GXP_E_UNKNOWN";
}

GXP_API const char* gxp_last_error(const gxp_ctx* ctx) {
    return ctx ? ctx->eng.last_error.c_str() : g_init_error.c_str();
}

GXP_API gxp_status gxp_set_stream(gxp_ctx* ctx, void* stream) {
    return guarded(ctx, [&](gxp::Engine& e) { e.set_stream(static_cast<cudaStream_t>(stream)); });
}

GXP_API gxp_status gxp_create_graph(gxp_ctx* ctx, uint64_t n_vertices, uint32_t n_parts,
                                    const uint64_t* part_begin) {
    return guarded(ctx, [&](gxp::Engine& e) { e.create_graph(n_vertices, n_parts, part_begin); });
}

GXP_API gxp_status gxp_load_partition(gxp_ctx* ctx, uint32_t part, gxp_format fmt, uint64_t n_edges,
                                      const void* idx0, const uint32_t* idx1, const uint32_t* weights) {
    return guarded(ctx, [&](gxp::Engine& e) { e.load_partition(part, fmt, n_edges, idx0, idx1, weights); });
}

GXP_API gxp_status gxp_begin(gxp_ctx* ctx, gxp_algo algo, uint32_t source, float damping) {
    return guarded(ctx, [&](gxp::Engine& e) { e.begin(algo, source, damping); });
}

GXP_API gxp_status gxp_get_values(gxp_ctx* ctx, uint32_t part, void* out, uint64_t n) {
    return guarded(ctx, [&](gxp::Engine& e) { e.get_values(part, out, n); });
}

GXP_API gxp_status gxp_set_values(gxp_ctx* ctx, uint32_t part, const void* in, uint64_t n) {
    return guarded(ctx, [&](gxp::Engine& e) { e.set_values(part, in, n); });
}

GXP_API gxp_status gxp_superstep(gxp_ctx* ctx, gxp_algo algo, gxp_msggen msggen, gxp_merge merge,
                                 gxp_apply apply, uint64_t* n_changed) {
    return guarded(ctx, [&](gxp::Engine& e) {
        const uint64_t c = e.superstep(algo, msggen, merge, apply, n_changed != nullptr);
        if (n_changed) *n_changed = c;
    });
}

GXP_API gxp_status gxp_sync(gxp_ctx* ctx, uint32_t part, uint32_t* ids, void* vals, uint64_t cap,
                            uint64_t* n_out, int* skipped) {
    return guarded(ctx, [&](gxp::Engine& e) { e.sync_result(part, ids, vals, cap, n_out, skipped); });
}

GXP_API gxp_status gxp_tune_cache_get(const char* path, const char* key, gxp_tune_record* out) {
    if (!path || !key || !out) return GXP_E_INVAL;
    try {
        return gxp::tune_cache_get(path, key, out) ? GXP_OK : GXP_E_INVAL;
    } catch (...) {
        return GXP_E_INVAL;
    }
}

GXP_API gxp_status gxp_tune_cache_put(const char* path, const char* key, const gxp_tune_record* rec) {
    if (!path || !key || !rec) return GXP_E_INVAL;
    try {
        return gxp::tune_cache_put(path, key, *rec) ? GXP_OK : GXP_E_INVAL;
    } catch (...) {
        return GXP_E_INVAL;
    }
}

GXP_API gxp_status gxp_cache_get(gxp_ctx* ctx, uint32_t part, uint32_t* ids, uint64_t cap, uint64_t* n_out) {
    return guarded(ctx, [&](gxp::Engine& e) { e.cache_contents(part, ids, cap, n_out); });
}

GXP_API gxp_status gxp_run(gxp_ctx* ctx, gxp_algo algo, uint32_t source, float damping, uint32_t max_steps,
                           uint32_t* steps_done) {
    return guarded(ctx, [&](gxp::Engine& e) {
        const uint32_t s = e.run(algo, source, damping, max_steps);
        if (steps_done) *steps_done = s;
    });
}

GXP_API gxp_status gxp_stats_get(gxp_ctx* ctx, gxp_stats* out) {
    if (!out) return GXP_E_INVAL;
    return guarded(ctx, [&](gxp::Engine& e) { e.stats(out); });
}

GXP_API gxp_status gxp_sssp_batch(gxp_ctx* ctx, const uint32_t* sources, uint32_t n_sources, uint32_t* dist_out,
                                  const gxp_batch_opts* opts, gxp_batch_report* report) {
    return guarded(ctx, [&](gxp::Engine& e) { e.sssp_batch(sources, n_sources, dist_out, opts, report); });
}

GXP_API gxp_status gxp_serve_add_graph(gxp_ctx* ctx, uint64_t n_vertices, uint64_t n_edges, const uint32_t* src,
                                       const uint32_t* dst, const uint32_t* weights, uint32_t* graph) {
    return served(ctx, true, [&](gxp::Server& s) {
        const uint32_t g = s.add_graph(n_vertices, n_edges, src, dst, weights);
        if (graph) *graph = g;
    });
}

GXP_API gxp_status gxp_serve_start(gxp_ctx* ctx, const gxp_serve_opts* opts) {
    return served(ctx, false, [&](gxp::Server& s) { s.start(opts); });
}

GXP_API gxp_status gxp_serve_stop(gxp_ctx* ctx) {
    return served(ctx, false, [&](gxp::Server& s) { s.stop(); });
}

GXP_API gxp_status gxp_query_submit(gxp_ctx* ctx, uint32_t graph, gxp_query_kind kind, uint32_t source,
                                    float damping, uint32_t iters, uint64_t* qid) {
    if (!qid) return GXP_E_INVAL;
    return served(ctx, false, [&](gxp::Server& s) { *qid = s.submit(graph, kind, source, damping, iters); });
}

GXP_API gxp_status gxp_query_poll(gxp_ctx* ctx, uint64_t qid, void* out, uint64_t cap, int timeout_ms, int* done) {
    if (done) *done = 0;
    return served(ctx, false, [&](gxp::Server& s) {
        const bool d = s.poll(qid, out, cap, timeout_ms);
        if (done) *done = d ? 1 : 0;
    });
}

GXP_API gxp_status gxp_query_next_done(gxp_ctx* ctx, int timeout_ms, uint64_t* qid) {
    if (!qid) return GXP_E_INVAL;
    *qid = 0;
    return served(ctx, false, [&](gxp::Server& s) { *qid = s.next_done(timeout_ms); });
}

GXP_API gxp_status gxp_query_info_get(gxp_ctx* ctx, uint64_t qid, gxp_query_info* out) {
    if (!out) return GXP_E_INVAL;
    return served(ctx, false, [&](gxp::Server& s) { s.info(qid, out); });
}

GXP_API gxp_status gxp_serve_report_get(gxp_ctx* ctx, gxp_serve_report* out) {
    if (!out) return GXP_E_INVAL;
    return served(ctx, false, [&](gxp::Server& s) { s.report(out); });
}

GXP_API gxp_status gxp_block_size_model(double k1, double k2, double k3, double a, uint64_t d, uint64_t* b,
                                        uint64_t* s, double* t) {
    try {
        gxp::block_size_model(k1, k2, k3, a, d, b, s, t);
        return GXP_OK;
    } catch (const gxp::Error& e) {
        g_init_error = e.msg;
        return e.code;
    }
}

}  // extern "C"
