// Host-side engine behind the C-ABI: one context = one device, one graph of
// partitions, one running algorithm. All device work goes through the
// kernels declared in gxp_internal.hpp.
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "fault.hpp"
#include "gxp_internal.hpp"

namespace gxp {

// Error carrying a gxp_status across the C++ layer; converted at the ABI.
struct Error {
    gxp_status code;
    std::string msg;
};

[[noreturn]] void fail(gxp_status code, const std::string& msg);
void cuda_check(cudaError_t e, const char* what);

struct HostPart {
    uint32_t v_begin = 0, n_own = 0;
    bool loaded = false;
    std::vector<uint32_t> col_ptr;    // [n_own + 1] local CSC offsets
    std::vector<uint32_t> src;        // local source ids (own: gid - v_begin; ghost: n_own + slot)
    std::vector<uint32_t> w;          // weights (empty = unweighted)
    std::vector<uint32_t> ghost_gid;  // sorted global ids of the cached remote sources
    // device copies (owned by Engine's allocation list)
    uint32_t* d_col_ptr = nullptr;
    uint32_t* d_src = nullptr;
    uint32_t* d_w = nullptr;
    uint32_t ghost_base = 0;
    uint64_t gdq_base = 0, n_boundary = 0;
    // CSC loaded straight into device memory (single-partition CSC loads): the
    // device arrays above belong to the partition and the host vectors stay
    // empty until something needs them (ensure_host)
    bool on_device = false;
    uint64_t dev_edges = 0;
    bool dev_weighted = false;

    uint64_t n_edges() const { return on_device ? dev_edges : src.size(); }
    bool weighted() const { return on_device ? dev_weighted : !w.empty(); }
};

class Engine {
public:
    Engine(int device, const gxp_config* cfg);
    ~Engine();

    void set_stream(cudaStream_t s) { stream_ = s ? s : own_stream_; }
    cudaStream_t stream() const { return stream_; }

    void create_graph(uint64_t n_vertices, uint32_t n_parts, const uint64_t* part_begin);
    void load_partition(uint32_t part, gxp_format fmt, uint64_t n_edges, const void* idx0,
                        const uint32_t* idx1, const uint32_t* weights);
    void begin(gxp_algo algo, uint32_t source, float damping);
    uint64_t superstep(gxp_algo algo, gxp_msggen g, gxp_merge m, gxp_apply a, bool want_changed);
    void sync_result(uint32_t part, uint32_t* ids, void* vals, uint64_t cap, uint64_t* n_out, int* skipped);
    void cache_contents(uint32_t part, uint32_t* ids, uint64_t cap, uint64_t* n_out);
    uint32_t run(gxp_algo algo, uint32_t source, float damping, uint32_t max_steps);
    void get_values(uint32_t part, void* out, uint64_t n);
    void set_values(uint32_t part, const void* in, uint64_t n);
    void stats(gxp_stats* out);
    void sssp_batch(const uint32_t* sources, uint32_t n_sources, uint32_t* dist_out, const gxp_batch_opts* opts,
                    gxp_batch_report* rep);

    std::string last_error;
    bool poisoned = false;

    uint64_t n_vertices() const { return n_vertices_; }

private:
    void* dalloc(size_t bytes);
    // every device allocation and host-to-device copy of the context goes
    // through these, so that an injected fault can fail the n-th one
    cudaError_t device_malloc(void** p, size_t bytes);
    void device_free(void* p);
    cudaMemPool_t pool_ = nullptr;   // the context's device memory (device_malloc)
    void before_h2d(const char* what);
    FaultPlan faults_;
    uint64_t n_allocs_ = 0, n_h2d_ = 0, n_exchanges_ = 0;
    void free_graph_device();
    void finalize();
    void build_sell();
    void build_caches();
    uint32_t* upload_u32(const std::vector<uint32_t>& h, size_t n_pad);
    // ring_copied: ring_host_ already holds the device ring (stream synchronized)
    uint64_t account(bool stop_at_quiet, bool ring_copied = false);
    std::vector<StepStats> ring_host_;
    void check_device_error();
    void copy_in(void* dst, const void* src, size_t bytes);   // host or device src -> host dst
    void load_csc_device(HostPart& hp, uint64_t n_edges, const void* col_ptr, const uint32_t* src,
                         const uint32_t* weights);
    void release_part(HostPart& hp);
    void ensure_host(HostPart& hp);
    void prepare_batch(bool streamed);
    void free_batch();
    double time_pipeline(uint64_t block_edges, bool pipelined, bool dry, int reps);
    void superstep_batch(const std::vector<uint64_t>& cuts, bool streamed, bool pipelined, bool dry, int parity);
    std::vector<uint64_t> block_cuts(uint64_t block_edges) const;

    int device_;
    gxp_config cfg_;
    cudaStream_t own_stream_ = nullptr, stream_ = nullptr;
    cudaEvent_t ev_a_ = nullptr, ev_b_ = nullptr, ev_k_ = nullptr;   // superstep start, end, kernel end

    // graph
    uint64_t n_vertices_ = 0;
    uint32_t n_parts_ = 0;
    std::vector<HostPart> parts_;
    bool have_graph_ = false, finalized_ = false, sell_ready_ = false;
    std::vector<PartDev> pd_;   // host copy of the per-partition device views
    struct WorkCsc {            // what the layout build reads
        const uint32_t* col = nullptr;   // offsets of the rows it writes
        RowSource in{};                  // where each row's edges come from
    };
    std::vector<WorkCsc> work_;
    bool relabeled_ = false;    // single partition renumbered by decreasing in-degree
    uint32_t* d_new2old_ = nullptr;
    uint32_t* d_old2new_ = nullptr;
    uint32_t* d_perm_tmp_ = nullptr;

    // device graph-level buffers
    std::vector<void*> graph_allocs_;
    uint64_t graph_bytes_ = 0;
    PartDev* d_parts_ = nullptr;
    SellSlice* d_slices_ = nullptr;
    HubPart* d_hubs_ = nullptr;
    uint32_t n_slices_ = 0, n_hubs_ = 0;
    uint32_t n_zero_slices_ = 0;   // one partition: trailing slices of rows without in-edges
    uint32_t *d_hub_val_ = nullptr, *d_hub_arrive_ = nullptr;
    uint32_t* d_outdeg_ = nullptr;
    uint32_t* d_own_[2] = {nullptr, nullptr};
    float* d_rank_[2] = {nullptr, nullptr};
    uint32_t* d_ghost_ = nullptr;
    uint32_t* d_ghost_gid_ = nullptr;
    uint32_t n_ghost_total_ = 0;
    uint32_t *d_changed_ = nullptr, *d_boundary_ = nullptr;
    uint32_t *d_gdq_ids_ = nullptr, *d_gdq_vals_ = nullptr;
    uint64_t* d_gdq_base_ = nullptr;
    uint32_t *d_block_counts_ = nullptr, *d_block_offsets_ = nullptr, *d_part_counts_ = nullptr;
    uint32_t* d_done_ctr_ = nullptr;
    // LRU-based caching under a budget (cache_slots): per-copy state, see lru.cu
    struct Lru {
        bool on = false;
        uint32_t capacity = 0, max_per_part = 0;
        uint32_t *d_base = nullptr, *d_reads = nullptr, *d_weight = nullptr, *d_hist = nullptr;
        uint32_t *d_tie = nullptr, *d_tie_scan = nullptr, *d_scratch = nullptr;
        uint8_t* d_flags = nullptr;
        LruPart* d_part = nullptr;
    } lru_;
    LruArgs lru_args(StepStats* out, const StepStats* quiet) const;
    void lru_reset(uint32_t source_int);
    uint32_t sync_blocks_x_ = 0, max_words_ = 0;
    StepStats* d_stats_ = nullptr;
    uint32_t* d_err_ = nullptr;
    bool weighted_ = false;

    // batched multi-source SSSP (single partition)
    struct Batch {
        bool ready = false, resident = false, pinned_ready = false;
        std::vector<uint4> units;          // {dst, first edge, edges, split}
        std::vector<uint64_t> unit_edge;   // first edge of each unit, + total at the end
        uint4* d_units = nullptr;
        void* h_edges = nullptr;           // pinned streamed edges, destination order (esize bytes each)
        void* d_edges = nullptr;           // resident copy, (source, weight) uint2
        void* d_ring[3] = {nullptr, nullptr, nullptr};
        uint32_t esize = 8;                // streamed edge: 8 = (source, weight) uint2, 4 = packed uint32
        bool packed = false;
        uint64_t ring_edges = 0;
        uint32_t* d_dist = nullptr;        // [V][64]
        uint32_t* d_frontier[3] = {nullptr, nullptr, nullptr};   // [2]: the persistent run's third bitmap
        unsigned long long* d_loop_changed = nullptr;   // [4] the persistent run's changed counters
        GridBar* d_bar = nullptr;
        uint32_t* d_steps = nullptr;
        unsigned long long* d_changed = nullptr;   // per-block counters
        unsigned long long* d_active = nullptr;    // active in-edges over a run (the roofline's row gathers)
        unsigned long long* h_changed = nullptr;   // pinned mirror (upload stage)
        uint32_t* d_sources = nullptr;
        size_t max_blocks = 0;
        cudaStream_t s_h2d = nullptr, s_d2h = nullptr;
        cudaEvent_t ev_loaded[3] = {}, ev_free[3] = {}, ev_t0 = nullptr, ev_t1 = nullptr;
        cudaGraphExec_t graph[2] = {nullptr, nullptr};
        uint64_t graph_block_edges = 0;
        bool graph_streamed = false, graph_pipelined = false;
    } batch_;
    // algorithm state
    bool begun_ = false;
    Algo algo_ = Algo::SSSP;
    uint32_t source_ = 0;
    uint32_t ppr_source_ = kInf;   // personalized PageRank: its source; else kInf
    // push direction (min-label algorithms, one partition): out-edge copy and
    // the two frontier lists (superstep t reads list t & 1, writes the other)
    bool frontier_ = false;        // the running algorithm keeps frontier lists
    bool out_ready_ = false;
    uint32_t* d_out_ptr_ = nullptr;
    uint32_t* d_out_dst_ = nullptr;
    uint32_t* d_out_w_ = nullptr;
    uint2* d_list_[2] = {nullptr, nullptr};
    uint64_t list_cap_ = 0;
    uint32_t n_slots_ = 0;         // push sources: the vertices, then (several partitions) the cached copies
    void build_out_edges();
    void seed_frontier(uint32_t source_int);
    // label propagation: rows by in-degree class, hub hash tables
    struct LpLists {
        bool ready = false;
        LpPart* d_parts = nullptr;
        LpWindow* d_windows = nullptr;
        uint32_t* d_row_g = nullptr;
        LpRow* d_chunks = nullptr;
        LpRow* d_warp_rows = nullptr;
        uint32_t n_warp_rows = 0;
        LpHub* d_hubs = nullptr;
        LpSegment* d_segments = nullptr;
        unsigned long long* d_hub_best = nullptr;
        uint32_t* d_seg_used = nullptr;
        uint32_t n_windows = 0, n_chunks = 0, n_hubs = 0, n_segments = 0;
        uint32_t* d_keys = nullptr;
        uint32_t* d_counts = nullptr;
    } lp_;
    void build_lp();
    // device-driven runs (min-label algorithms, one partition)
    static constexpr uint32_t kRunChunk = 32;   // supersteps per graph launch (the stat ring holds 64)
    cudaGraphExec_t run_graph_[2] = {nullptr, nullptr};   // SSSP, CC
    bool run_graph_failed_ = false;
    RunCtl* d_ctl_ = nullptr;
    GridBar* d_bar_ = nullptr;     // the persistent run's grid barrier
    RunCtl* h_ctl_ = nullptr;      // pinned: [0] to the device, [1] back
    StepStats* h_ring_ = nullptr;  // pinned copy of the stat ring
    std::vector<uint32_t> h_old2new_;   // host copy of the renumbering (source ids)
    bool run_graph_ready();
    SellArgs sell_args() const;
    bool early_exit_ = false;      // inside gxp_run: supersteps after a quiet one return at once
    bool auto_tiles_ = false;      // tile / hub sizes chosen from the graph's size
    float damping_ = 0.85f;
    int cur_ = 0;
    uint64_t step_ = 0, accounted_ = 0;
    gxp_stats st_{};
    uint64_t total_edges_ = 0;
};

// The autotuner's JSON cache (tune_cache.cpp).
bool tune_cache_get(const char* path, const char* key, gxp_tune_record* out);
bool tune_cache_put(const char* path, const char* key, const gxp_tune_record& rec);

// Lemma 1 block-size model (host arithmetic).
void block_size_model(double k1, double k2, double k3, double a, uint64_t d, uint64_t* b,
                      uint64_t* s, double* t);

}  // namespace gxp
