// Query server: continuous batching of SSSP and personalized-PageRank
// queries over graphs resident on one GPU.
//
// Each served graph has one lane per query kind. A lane owns 64 query slots
// (one column of a [V][64] state matrix each) and a host thread that loops:
// admit queued queries into free slots, run one superstep for every busy
// slot at once, retire the slots whose query finished (SSSP: no distance of
// the slot improved; PPR: its iteration count reached), copying each
// finished column out as a contiguous result vector. Queries that arrive
// while others run join at the next superstep boundary.
//
// Admission is by slot and by memory: a query also needs one of its graph's
// device result buffers, held from admission until the caller collects the
// result, so results nobody collects hold back new admissions.
#pragma once

#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "engine.hpp"

namespace gxp {

struct Query {
    uint64_t id = 0;
    uint32_t graph = 0;
    gxp_query_kind kind = GXP_QUERY_SSSP;
    uint32_t source = 0;
    float damping = 0.85f;
    uint32_t iters = 20;
    uint32_t state = GXP_QUERY_QUEUED;
    gxp_status status = GXP_OK;
    uint32_t* d_result = nullptr;   // from the graph's result pool while admitted
    uint32_t supersteps = 0;
    double t_submit = 0, t_admit = 0, t_done = 0;   // seconds, steady clock
    bool reported = false;                          // handed out by next_done
    bool collecting = false;                        // a poll is copying the result out
};

class Server;

struct Lane {
    uint32_t graph = 0;
    gxp_query_kind kind = GXP_QUERY_SSSP;
    uint32_t max_slots = 64;
    cudaStream_t stream = nullptr;
    int prio = 0;                                  // CUDA stream priority of `stream`
    std::thread thread;
    std::condition_variable cv;
    std::deque<uint64_t> queue;
    Query* slot_q[64] = {};
    uint32_t slot_steps[64] = {};
    uint64_t busy = 0;
    int cur = 0;
    uint64_t supersteps = 0;
    // device state
    uint32_t* d_dist = nullptr;                    // SSSP [V][64]
    uint32_t* d_frontier[2] = {nullptr, nullptr};  // SSSP
    uint32_t* d_improved = nullptr;                // SSSP [2]
    unsigned long long* d_changed = nullptr;       // SSSP unit counter
    float* d_msg[2] = {nullptr, nullptr};          // PPR [V][64]
    float* d_rank = nullptr;                       // PPR [V][64]
    float* d_partial = nullptr;                    // PPR [n_partials][64]
    unsigned long long* d_dang[2] = {nullptr, nullptr};
    uint32_t* d_slot_source = nullptr;             // [64]
    float* d_slot_damping = nullptr;               // [64]
    // pinned host staging
    uint32_t* h_table = nullptr;                   // source[64], damping bits[64]
    uint32_t* h_improved = nullptr;                // [2]
};

struct ServedGraph {
    uint64_t n = 0, m = 0;
    bool weighted = false;
    uint4* d_units_all = nullptr;   // every vertex (PPR)
    uint64_t n_units_all = 0;
    uint4* d_units_nz = nullptr;    // vertices with in-edges (SSSP)
    uint64_t n_units_nz = 0;
    void* d_edges = nullptr;        // (source, weight) uint2 or packed uint32, destination order
    bool packed = false;
    uint32_t* d_src = nullptr;      // source, destination order
    float* d_inv_outdeg = nullptr;  // 1 / out-degree, 0 for vertices without out-edges
    uint2* d_split_rows = nullptr;
    uint32_t n_split_rows = 0;
    uint64_t n_partials = 0;
    std::vector<uint32_t*> free_results;
    std::vector<uint32_t*> all_results;
    std::unique_ptr<Lane> lanes[2];
};

class Server {
public:
    Server(int device, uint64_t mem_budget);
    ~Server();

    uint32_t add_graph(uint64_t n, uint64_t m, const uint32_t* src, const uint32_t* dst, const uint32_t* w);
    void start(const gxp_serve_opts* opts);
    void stop();
    uint64_t submit(uint32_t graph, gxp_query_kind kind, uint32_t source, float damping, uint32_t iters);
    bool poll(uint64_t qid, void* out, uint64_t cap, int timeout_ms);
    uint64_t next_done(int timeout_ms);
    void info(uint64_t qid, gxp_query_info* out);
    void report(gxp_serve_report* out);

private:
    void* dalloc(size_t bytes);
    void dfree(void* p, size_t bytes);
    void lane_loop(Lane& L);
    void lane_step(Lane& L, ServedGraph& G, uint64_t admit_mask);
    void fail_lane(Lane& L, gxp_status code);
    static double now();

    int device_;
    uint64_t mem_budget_;
    uint64_t bytes_ = 0;
    std::vector<void*> allocs_;
    std::vector<std::unique_ptr<ServedGraph>> graphs_;
    bool running_ = false, stopping_ = false;
    gxp_status error_ = GXP_OK;
    uint32_t queue_cap_ = 1u << 20;
    uint64_t queued_ = 0;

    std::mutex mu_;
    std::condition_variable cv_done_;
    std::unordered_map<uint64_t, std::unique_ptr<Query>> queries_;
    std::deque<uint64_t> done_fifo_;
    uint64_t next_id_ = 1;
    uint64_t n_submitted_ = 0, n_completed_ = 0, n_failed_ = 0;

    std::mutex copy_mu_;
    std::vector<cudaStream_t> copy_streams_;
};

}  // namespace gxp
