// Internal declarations of libgxp: device data layout, kernel launchers and
// the host-side context. Not part of the C-ABI (include/gxp.h is).
#pragma once

#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <mutex>
#include <string>
#include <vector>

#include "gxp.h"

namespace gxp {

constexpr uint32_t kInf = 0xFFFFFFFFu;
constexpr int kBlock = 128;          // threads per superstep CTA (4 independent warps)
constexpr uint32_t kVertexCost = 4;  // merge-path weight of a vertex end when cutting tiles
constexpr int kMaxTileItems = 3072;  // tile_items + hub_items limit (shared-memory budget)
constexpr int kStatLanes = 64;       // stat accumulators are spread over lanes to
                                     // avoid same-address atomic serialization
constexpr int kStatRing = 64;        // superstep stat slots kept on the device

// Device error word bits (ORed by kernels, read by the host at sync points).
constexpr uint32_t kErrBounds = 1u;
constexpr uint32_t kErrTimeout = 2u;
constexpr uint32_t kErrDrain = 4u;     // a give-up drain ran out before its copies landed
constexpr uint32_t kErrInput = 8u;     // CSC offsets not running from 0 to n_edges, non-decreasing

// Fixed-point scale of the exact global sums (dangling mass, L1 delta):
// an fp32 value x in [0, 2] is held as round(x * 2^60) in a uint64.
constexpr int kFxShift = 60;

enum class Algo : int { SSSP = 0, CC = 1, PR = 2, LP = 3 };

// One edge block ("tile") paired with its vertex block (Section II-B): the
// in-edges [e0, e0+ne) of local destinations [v0, v0+nv) of one partition.
// Blocks are cut at vertex boundaries except inside hub vertices whose
// in-degree exceeds hub_items; such a vertex spans several blocks, and its
// partial merges are combined by the last block to finish it.
struct Tile {
    uint32_t v0;       // first local destination vertex
    uint32_t nv;       // destination vertices touched (incl. an open head/tail)
    uint32_t e0;       // first edge (partition-local CSC index)
    uint32_t ne;       // edge count
    uint32_t part;     // partition index
    uint32_t flags;    // kHeadOpen | kTailOpen
    uint32_t hub_t0;   // kHeadOpen: global index of the tile where the head vertex starts
    uint32_t nparts;   // tile that starts an open tail vertex: tiles that vertex spans
};
constexpr uint32_t kHeadOpen = 1u;
constexpr uint32_t kTailOpen = 2u;

// Sliced-ELL layout of the non-hub rows (SELL-32-sigma): rows are sorted by
// in-degree inside windows of kSellWindow rows and grouped into slices of 32;
// a slice stores its rows' in-edges column-major, for a single partition in
// groups of 4 columns (edges 4g..4g+3 of row slot l at off + 128 g + 4 l, see
// sell_idx), padded with the partition's padding id.
struct SellSlice {
    uint32_t part;     // partition index
    uint32_t row0;     // first entry of the slice in the partition's perm array
    uint32_t width;    // edges per row slot (the slice's largest in-degree)
    uint32_t pad0;
    uint64_t off;      // first element of the slice in the partition's sell arrays
};
constexpr uint32_t kSellPad = 0xFFFFFFFFu;   // empty row slot of a slice (perm)
// Element of column k, row slot l in a slice's storage. A single partition
// stores its columns in groups of 4 (g4: a lane reads 4 of its row's sources
// with one 128-bit load); several partitions column by column (measured
// faster on their uniform graphs, whose widths the rounding would pad more).
__host__ __device__ constexpr uint64_t sell_idx(uint32_t k, uint32_t l, bool g4) {
    return g4 ? 128ull * (k >> 2) + 4ull * l + (k & 3u) : 32ull * k + l;
}
// columns a slice stores: its width, rounded up to a whole group with g4
__host__ __device__ constexpr uint32_t sell_cols(uint32_t width, bool g4) { return g4 ? (width + 3u) & ~3u : width; }
constexpr uint32_t kSellWindow = 65536;      // rows sorted by degree within windows of this size
constexpr uint32_t kZeroGroup = 4;           // slices of rows without in-edges per warp (PageRank)

// A slice of the in-edges of one hub row (in-degree above the SELL limit),
// reduced by one warp; the last part of a row to arrive combines all parts.
struct HubPart {
    uint32_t v;        // partition-local destination vertex
    uint32_t part;     // partition index
    uint32_t e0;       // first edge in the partition's hub edge arrays
    uint32_t ne;       // edges in this part
    uint32_t t0;       // global index of the row's first part
    uint32_t nparts;   // parts of this row
    uint32_t pad[2];
};

// Per-partition device view (array in device memory, indexed by Tile::part).
struct PartDev {
    const uint32_t* col_ptr;   // [n_own + 1] CSC offsets, padded to a multiple of 4 + 4
    const uint32_t* src;       // [n_edges] local source index, padded likewise
    const uint32_t* w;         // [n_edges] weights or nullptr
    uint32_t n_own;            // owned vertices
    uint32_t v_begin;          // global id of local vertex 0
    uint32_t n_ghost;          // cached remote vertices (local ids n_own ..)
    uint32_t ghost_base;       // offset of this partition's ghosts in the ghost array
    uint64_t n_edges;
    // sliced-ELL layout (engine path)
    const uint32_t* sell_src;  // column-major slices, pad_id in empty slots
    const uint32_t* sell_w;    // weights in the same layout, or nullptr
    const uint32_t* perm;      // slice row slot -> local vertex (kSellPad = empty)
    const uint32_t* hsrc;      // hub rows' in-edges, row after row
    const uint32_t* hw;        // and weights, or nullptr
    // local id of the identity slot that empty SELL slots name: one partition,
    // n_own (own[V], past the last vertex); several, the slot past every
    // partition's cached copies (ghost[n_ghost_total]). The slot holds the
    // merge's identity (0 for sums, INF for minima) and is never written by
    // a superstep, so padding needs no test in the kernel.
    uint32_t pad_id;
    uint32_t pad1;
};

// Accumulators of one superstep (one ring slot).
struct StepStats {
    unsigned long long changed[kStatLanes];
    unsigned long long dangling_fx[kStatLanes];   // sum of fx(r) over out-degree-0 vertices
    unsigned long long l1_fx[kStatLanes];         // sum |fx(r_new) - fx(r_old)|
    unsigned long long boundary_changed;          // pairs uploaded by the sync (all partitions)
    unsigned long long skipped;                   // 1 if the exchange was skipped
    // frontier of the next superstep (min-label algorithms, single partition):
    // items appended to its list (high 32 bits) and the out-edges of the
    // vertices they cover (low 32 bits), advanced together by one atomic
    unsigned long long list_ne;
    unsigned long long pushed;                    // 1: the superstep ran in push direction,
    unsigned long long push_edges;                //    relaxing this many out-edges
    unsigned long long exchanged;                 // 1 once the superstep's exchange between
                                                  // partitions ran (skipped or not)
    unsigned long long downloads;                 // copies the superstep used that were not cached
    // 1: the exchange lists the changed cached copies in the next frontier.
    // Decided once by k_sync_count from the own vertices' appends and the
    // changed boundary vertices: the copies' appends then advance list_ne,
    // so a test each CTA of k_sync_pull made for itself would see a moving
    // count and the CTAs could disagree (some copies listed, others not).
    unsigned long long list_copies;
    // 1: the superstep pulled without listing its changed vertices
    // (FrontierCfg::list_max_changed), so the next one must pull too
    unsigned long long unlisted;
};
__host__ __device__ constexpr unsigned long long list_pack(uint32_t items, uint32_t edges) {
    return ((unsigned long long)items << 32) | edges;
}

// Frontier lists: the vertices changed by a superstep, as work items of at
// most kItemEdges out-edges each ({vertex, chunk}: out-edges [32 chunk,
// 32 chunk + 32) of the vertex; a vertex without out-edges has one empty
// item). Per list: at most n_vertices + ceil(n_edges / 32) items (below
// 2^32, or the lists are not used); the out-edges of one list are at most
// n_edges < 2^32, so the packed counter's halves never carry into each other.
constexpr uint32_t kItemEdges = 32;
struct FrontierCfg {
    const uint2* list_in;        // this superstep's frontier (count: stats_in->list_ne >> 32)
    uint2* list_out;             // the next one; nullptr = no frontier lists (pull only)
    uint32_t direction;          // gxp_direction
    uint32_t push_div;
    uint64_t total_edges;
    uint64_t list_cap;           // items each list holds
    uint32_t* err;               // kErrBounds if a list would overflow (never, for valid graphs)
    // A pull superstep lists the vertices it changes (the next frontier) only
    // when the frontier it read was small enough to make a push next likely:
    // at most this many changed vertices, and items + out-edges within
    // kListSlack times the push limit. Listing costs a pull superstep an
    // out-degree load and an item write per changed vertex, which pays only
    // when the next superstep pushes. kAlwaysList: always list.
    uint64_t list_max_changed;
};
constexpr uint64_t kAlwaysList = ~0ull;
constexpr uint32_t kListSlack = 4;



// Everything the superstep kernel touches.
struct SuperstepArgs {
    const Tile* tiles;
    const PartDev* parts;
    uint32_t n_tiles;
    const uint32_t* own_cur;     // [V] current values (u32 or f32 bits), global id order;
                                 // own_cur, rank_cur and outdeg are padded to a multiple of 4
    uint32_t* own_nxt;           // [V] next values
    const uint32_t* ghost;       // [sum of n_ghost] cached remote values
    const float* rank_cur;       // PageRank ranks [V] (fp32)
    float* rank_nxt;
    const uint32_t* outdeg;      // [V] global out-degree (PageRank)
    uint32_t* changed_bits;      // [ceil(V/32)] or nullptr
    uint32_t* part_head;         // [n_tiles] partials of rows split across tiles (value bits)
    uint32_t* part_tail;         // [n_tiles]
    uint32_t* hub_cnt;           // [n_tiles] arrival counters (self-resetting)
    StepStats* stats_in;         // slot of the current state (PageRank: its dangling mass)
    StepStats* stats_out;        // slot the superstep accumulates into
    StepStats* stats_clear;      // slot zeroed for the superstep after next
    uint32_t* err;               // device error word
    uint64_t timeout_ns;         // limit of any device-side wait
    uint32_t force_timeout;      // injected fault: every wait gives up at once (then drains)
    uint32_t check_bounds;
    float damping;
    double inv_n;                // 1 / N
    uint32_t max_items;          // largest tile (merge items)
};

// Everything the sliced-ELL superstep kernel touches.
struct SellArgs {
    const SellSlice* slices;
    uint32_t n_slices;
    const HubPart* hubs;
    uint32_t n_hubs;
    const PartDev* parts;
    uint32_t n_parts;            // 1: the single-partition kernel (no cached copies, no bitmap)
    uint32_t n_vertices;         // V: the first cached-copy slot of the push direction
    // superstep t reads value buffer t & 1, stat slot t % kStatRing and
    // frontier list t & 1; it writes buffer / list (t + 1) & 1 and slot t + 1,
    // and clears slot t + 2
    uint32_t* own[2];
    float* rank[2];
    StepStats* stats;            // [kStatRing]
    uint2* lists[2];             // frontier lists (min-label algorithms, one partition) or nullptr
    uint64_t step;               // t, unless
    const uint64_t* step_dev;    // t lives in device memory (device-driven runs)
    const uint32_t* ghost;
    const uint32_t* outdeg;
    uint32_t* changed_bits;
    uint32_t* hub_val;           // [n_hubs] published partials (value bits)
    uint32_t* hub_arrive;        // [n_hubs] arrival counters, indexed by a row's first part
    uint32_t* err;
    uint32_t check_bounds;
    float damping;
    float inv_n;                 // 1 / N
    uint32_t ppr_source;         // PageRank: kInf; personalized PageRank: the source vertex
    uint32_t early_exit;         // 1: a superstep (t > 0) after a quiet one returns at once
    // PageRank on one partition: the last n_zero slices (heavy-first order)
    // hold rows without in-edges; a warp applies kZeroGroup of them at once
    uint32_t n_zero;
    // SSSP / CC: fc.list_out != nullptr turns the frontier lists on (the
    // kernel points list_in / list_out at lists[]); the out-edge copy is
    // what the push direction reads. Its sources are slots: the V vertices,
    // then (several partitions) the cached copies, slot V + g for copy g.
    FrontierCfg fc;
    const uint32_t* out_ptr;     // [slots + 1] out-edge offsets, internal ids
    const uint32_t* out_dst;     // [E] destinations (vertices), grouped by source slot
    const uint32_t* out_w;       // [E] weights, or nullptr (CC)
};

// Arguments of the batched multi-source SSSP superstep kernel (one edge block).
constexpr uint32_t kUnitEdges = 256;   // in-edges of one destination per warp work unit
// packed edge (4 bytes): weight << 24 | source, when sources < 2^24 and weights < 256
constexpr uint32_t kPackSrcBits = 24;
inline bool packable(uint64_t n_vertices, uint32_t max_weight) {
    return n_vertices <= (1ull << kPackSrcBits) && max_weight < 256u;
}
struct MsArgs {
    const uint4* units;          // {dst, first edge (global), edges, split-row flag}
    uint64_t u_begin, u_end;     // this block's units
    const void* edges;           // edges[i] is global edge edge_base + i: (source, weight) uint2,
                                 // or with `packed` one uint32 (weight << 24 | source)
    uint32_t packed;
    uint64_t edge_base;
    uint32_t* dist;              // [V][64]
    const uint32_t* frontier_cur;
    uint32_t* frontier_next;
    unsigned long long* changed; // units that improved a slot (this block's counter)
    unsigned long long* active;  // nullable: running count of in-edges whose source was in the frontier
    uint32_t* slot_improved;     // nullable: [2] bit s of word 0 / s - 32 of word 1 = slot s improved
    uint64_t idle_mask;          // slots to skip (no query in them); 0 = compute all 64
};

// Finished query slots whose columns are copied out as result vectors.
struct GatherList {
    uint32_t n;
    uint32_t slot[64];
    uint32_t* out[64];
};

// Arguments of the personalized-PageRank superstep over 64 query slots
// (serving). Matrices are [V][64] fp32, one 256-byte row per vertex.
struct PprArgs {
    const uint4* units;              // {dst, first edge, edges, partial index + 1 | 0}
    uint64_t n_units;                // covers every vertex (empty rows too)
    const uint32_t* src;             // source id of each edge, destination order
    const uint2* split_rows;         // [n_split_rows + 1] {row, first partial}; last .y = n_partials
    uint32_t n_split_rows;
    const float* inv_outdeg;         // [V] 1 / outdeg, 0 for vertices without out-edges
    const float* msg_cur;            // [V][64] r_t / outdeg
    float* msg_nxt;                  // [V][64]
    float* rank;                     // [V][64] r_{t+1}, written for slots in finish_mask
    float* partial;                  // [n_partials][64]
    const unsigned long long* dang_cur;   // [64] exact dangling mass of r_t per slot
    unsigned long long* dang_next;        // [64] (zeroed before the superstep)
    const float* slot_damping;       // [64]
    const uint32_t* slot_source;     // [64]
    uint64_t active_mask;            // slots holding a query
    uint64_t finish_mask;            // slots whose last superstep this is
};

// Mode-label propagation (lp.cu). Rows are listed by in-degree class:
// 1..32 in-edges (packed into warp windows), up to kLpWarpRow (a warp per
// row) and up to kLpChunk (a CTA per row), both counting in shared-memory
// hash tables, more (a hub: chunks of kLpChunk
// counted the same way and added into a global hash table of its own, which
// segments of kLpSegment slots then reduce). Rows without in-edges keep their
// labels and are not listed.
constexpr uint32_t kLpSmall = 32;
constexpr uint32_t kLpWarpRow = 256;   // rows up to this many in-edges: a warp each
constexpr uint32_t kLpChunk = 2048;
constexpr uint32_t kLpSegment = 4096;
struct LpPart {                 // where a row's in-edges and their labels are
    const uint32_t* src;        // CSC sources as local ids (a renumbered partition's, renumbered once)
    uint32_t v_begin, n_own, ghost_base, pad;
};
struct LpRow {                  // a row, or a chunk of a hub row
    uint32_t g;                 // value index (global internal id)
    uint32_t part;
    uint32_t e0;                // first in-edge (partition CSC index)
    uint32_t n;                 // in-edges
    uint32_t hub;               // hub index for a hub chunk, else kInf
    uint32_t pad[3];
};
// Consecutive rows of 1..32 in-edges whose edges are adjacent, packed into
// one warp's 32 lanes: lane k reads edge e0 + k; bit k of `starts` marks
// the lanes where a row begins (the rows' value indices are row_g[first ..]).
struct LpWindow {
    uint32_t e0;
    uint32_t first;
    uint32_t starts;
    uint32_t n_part;            // edges (low 6 bits) | partition << 6
};
struct LpHub {
    uint32_t g;
    uint32_t log2_size;         // table slots = 2^log2_size >= 2 in-degree
    uint64_t table;             // first slot
    uint32_t seg0;              // its first segment (segment i covers slots [i kLpSegment, ...) of the table)
    uint32_t pad;
};
struct LpSegment {              // kLpSegment slots (or fewer) of one hub's table
    uint32_t hub;
    uint32_t n;
    uint64_t slot0;
};
struct LpArgs {
    const LpPart* parts;
    uint32_t n_parts;           // 1: no cached copies (sources are indices into own_cur)
    const LpWindow* windows;    // rows of 1..kLpSmall in-edges
    uint32_t n_windows;
    const uint32_t* row_g;      // their value indices
    const LpRow* warp_rows;     // kLpSmall < in-edges <= kLpWarpRow
    uint32_t n_warp_rows;
    const LpRow* chunks;        // kLpWarpRow < in-edges <= kLpChunk (hub = kInf), and hub chunks
    uint32_t n_chunks;
    const LpHub* hubs;
    uint32_t n_hubs;
    const LpSegment* segments;  // the hub tables cut into segments
    uint32_t n_segments;
    uint32_t* keys;             // hub tables: label per slot (kInf = empty) ...
    uint32_t* counts;           // ... and its count; left empty after each superstep
    unsigned long long* hub_best;   // [n_hubs] best (count, -label) over the segments; zeroed after use
    uint32_t* seg_used;             // [n_segments] 1 once a label took a slot of the segment; cleared after use
    const uint32_t* own_cur;
    uint32_t* own_nxt;
    const uint32_t* ghost;
    uint32_t* changed_bits;     // partitions: bitmap of changed vertices, or nullptr
    const StepStats* stats_in;
    StepStats* stats_out;
    StepStats* stats_clear;
    uint32_t skip_if_quiet;     // 1: return at once if the previous superstep changed nothing
    uint32_t narrow_labels;     // 1: labels < 2^27 (32-bit (row, label) keys suffice)
};
cudaError_t launch_lp_superstep(const LpArgs& a, cudaStream_t s);

// Arguments of the two sync kernels (changed ∩ boundary -> gdq -> caches).
struct SyncArgs {
    const PartDev* parts;
    uint32_t n_parts;
    const uint32_t* changed_bits;
    const uint32_t* boundary_bits;
    const uint32_t* own_val;          // values after the superstep, [V]
    const uint32_t* ghost_gid;        // [n_ghost] global id of each cached copy (sorted per partition)
    uint32_t n_ghost;                 // cached copies over all partitions
    uint32_t* ghost;                  // [n_ghost] caches to update
    const uint8_t* cached;            // [n_ghost] LRU flags (bit 0: cached), or nullptr = all cached
    uint32_t n_pull;
    uint32_t* gdq_ids;                // [sum of boundary counts]
    uint32_t* gdq_vals;
    const uint64_t* gdq_base;         // [n_parts] offset of each partition's gdq
    uint32_t* block_counts;           // [n_parts * blocks_x]
    uint32_t* block_offsets;          // [n_parts * blocks_x]
    uint32_t* part_counts;            // [n_parts]
    uint32_t* done_ctr;               // arrival counter of the count kernel
    uint32_t blocks_x;
    StepStats* stats_out;
    // frontier lists on (push direction possible): every cached copy whose
    // vertex changed joins the next frontier as slot n_vertices + g
    FrontierCfg fc;                   // fc.list_out = the next superstep's list, or nullptr
    const uint32_t* out_ptr;          // slot out-edge offsets
    uint32_t n_vertices;
};

// ------------------------------------------------------------ launchers
cudaError_t launch_build_tiles(const uint32_t* d_col_ptr, uint32_t n_own, uint32_t n_edges,
                               uint32_t tile_items, uint32_t hub_items, uint32_t part,
                               uint32_t tile_base, uint32_t n_tiles, Tile* d_tiles,
                               uint64_t* d_scratch_cuts, cudaStream_t s);
uint32_t tile_count(uint32_t n_own, uint64_t n_edges, uint32_t tile_items);

cudaError_t launch_outdeg(const PartDev& p, const uint32_t* d_src, const uint32_t* d_ghost_gid,
                          uint32_t* d_outdeg, cudaStream_t s);
cudaError_t launch_csc_import(const uint64_t* cp64, uint32_t n, uint64_t n_edges, uint32_t* cp32,
                              const uint32_t* src, uint32_t n_local, uint32_t* err, cudaStream_t s);
// sources >= n_local set kErrBounds; offsets that do not run from 0 to n_edges
// without decreasing set kErrInput
cudaError_t launch_validate_csc(const uint32_t* d_col_ptr, uint32_t n_own, const uint32_t* d_src,
                                uint64_t n_edges, uint32_t n_local, uint32_t* d_err, cudaStream_t s);

cudaError_t launch_init_values(Algo a, uint32_t ppr_source, uint32_t n_vertices, uint32_t source,
                               uint32_t* own_cur, float* rank_cur, const uint32_t* outdeg,
                               StepStats* stats0, const uint32_t* label_of, cudaStream_t s);
cudaError_t launch_identity_slots(uint32_t* a, uint32_t* b, uint32_t* c, uint32_t v, cudaStream_t s);   // *a = *b = *c = v
cudaError_t launch_init_ghosts(Algo a, uint32_t n_ghost_total, const uint32_t* ghost_gid_all,
                               const uint32_t* own_cur, uint32_t* ghost, cudaStream_t s);

cudaError_t launch_superstep(Algo a, const SuperstepArgs& args, size_t smem_bytes, cudaStream_t s);
cudaError_t launch_superstep_sell(Algo a, const SellArgs& args, cudaStream_t s);

// Device-driven run: the step counter the superstep kernel reads
// (SellArgs::step_dev) and the loop's bounds.
struct RunCtl {
    uint64_t step;          // supersteps done
    uint64_t limit;         // the loop stops when step reaches it
    uint32_t quiet_stop;    // 1: also stop after a superstep that changed nothing
    uint32_t pad;
};
cudaError_t launch_run_control(RunCtl* ctl, const StepStats* ring, cudaGraphConditionalHandle h, cudaStream_t s);
// Grid barrier state of the persistent run (zeroed before each launch).
struct GridBar {
    uint32_t count;   // CTAs arrived at the current barrier
    uint32_t gen;     // barriers passed
};
// Persistent device-driven run of SSSP / CC on one partition (k_sell_loop):
// the supersteps of ctl in one cooperative launch of at most one CTA per
// co-resident slot. Returns cudaErrorNotSupported, launching nothing, when
// a superstep needs more than kLoopWaves grids of co-resident CTAs (the
// graph-driven loop then serves); a barrier wait past timeout_ns (or any,
// with `force`) sets kErrTimeout in args.err and ends the launch.
constexpr uint32_t kLoopWaves = 2;
bool sell_loop_fits(Algo a, const SellArgs& args);
cudaError_t launch_sell_loop(Algo a, const SellArgs& args, RunCtl* ctl, GridBar* bar, uint64_t timeout_ns,
                             bool force, cudaStream_t s);
size_t superstep_smem_bytes(Algo a, uint32_t max_items);

cudaError_t launch_sync(const SyncArgs& args, uint32_t max_words, cudaStream_t s);

// LRU-based caching under a budget (lru.cu): the superstep-boundary update of
// every partition's cached copies. Weights saturate at kLruWMax.
constexpr uint32_t kLruWMax = 65535;
constexpr uint32_t kLruBins = kLruWMax + 1;
struct LruPart {
    uint32_t cand;      // candidates (cached or used) at this boundary
    uint32_t w_star;    // the lowest weight kept
    uint32_t ties;      // candidates of weight w_star kept (lowest ids first); kInf = all candidates
    uint32_t pad;
};
struct LruArgs {
    uint32_t n_parts, n_ghost;
    const uint32_t* ghost_base;       // [n_parts + 1] first copy of each partition
    const uint32_t* ghost_gid;        // [n_ghost] vertex of each copy (ascending per partition)
    const uint32_t* reads;            // [n_ghost] the partition's in-edges from that vertex
    uint32_t* weight;                 // [n_ghost]
    uint8_t* flags;                   // [n_ghost] bit 0 cached, bit 1 candidate (transient)
    uint32_t* ghost;                  // [n_ghost] copy values (downloads write here)
    const uint32_t* own_val;          // owners' current values
    // the frontier of the coming superstep: every vertex, a bitmap, or one vertex
    uint32_t frontier_all;
    const uint32_t* frontier_bits;
    uint32_t frontier_one;
    uint32_t capacity;                // copies kept per partition
    uint32_t* hist;                   // [n_parts][kLruBins], zero between boundaries
    LruPart* part_state;              // [n_parts], cand zero between boundaries
    uint32_t* tie;                    // [n_ghost]
    uint32_t* tie_scan;               // [n_ghost + 1]
    uint32_t* scan_scratch;           // (n_ghost + 2047) / 2048 + 1 words
    StepStats* stats_out;             // `downloads` of the coming superstep
    const StepStats* quiet_check;     // non-null: no-op when that superstep changed nothing
};
cudaError_t launch_lru_boundary(const LruArgs& a, uint32_t max_ghosts_per_part, cudaStream_t s);

// push direction (frontier.cu)
struct RowSource;
// out-edge copy of the CSC `in` (rows renumbered as the layout build does):
// out_ptr = exclusive scan of outdeg (internal ids); scratch holds
// out_edges_scratch_words(n, n_edges) words
// (rows: n, sources: n_src >= n; out_ptr[n_src + 1])
cudaError_t launch_out_edges(const RowSource& in, uint32_t n, uint32_t n_src, uint64_t n_edges,
                             const uint32_t* outdeg, uint32_t* out_ptr, uint32_t* scratch, uint32_t* out_dst,
                             uint32_t* out_w, cudaStream_t s);
size_t out_edges_scratch_words(uint32_t n_src, uint64_t n_edges);
// several partitions: the CSC over global rows whose sources are slots
// (own vertex u -> v_begin + u, cached copy u -> V + ghost_base + u - n_own)
// and the out-degree of every slot (counted into outdeg, zeroed first)
cudaError_t launch_unify_csc(const PartDev& p, uint32_t n_vertices, uint64_t edge_base, uint32_t* ucol,
                             uint32_t* usrc, bool last, cudaStream_t s);
cudaError_t launch_slot_degrees(const uint32_t* usrc, uint64_t n_edges, uint32_t n_slots, uint32_t* outdeg,
                                cudaStream_t s);
// every slot whose value is below INF joins the list (partitioned starts)
cudaError_t launch_seed_finite(uint32_t n_vertices, uint32_t n_ghost, const uint32_t* own, const uint32_t* ghost,
                               const uint32_t* out_ptr, const FrontierCfg& f, StepStats* stats, cudaStream_t s);
// f.list_out <- items of vertex `source` (all vertices when source == kInf);
// the counts go to stats->list_ne (zeroed here first)
cudaError_t launch_seed_frontier(uint32_t n, uint32_t source, const uint32_t* out_ptr, const FrontierCfg& f,
                                 StepStats* stats, cudaStream_t s);
// exclusive scan of n u32 counts into out[0..n] (out[n] = total); scratch:
// (n + 2047) / 2048 + 1 words (sell_build.cu)
cudaError_t launch_exclusive_scan_u32(const uint32_t* x, uint32_t n, uint32_t* out, uint32_t* scratch,
                                      cudaStream_t s);

cudaError_t launch_msssp(const MsArgs& a, bool dry, uint32_t grid, cudaStream_t s);
// Persistent resident run (k_msssp_loop): supersteps over the units of `a`
// until one improves nothing or max_steps, one cooperative launch; frontier
// rotates over three bitmaps of `words` words (frontier[0] holds the sources,
// frontier[1] must be zero), changed over four counters (the first two zero);
// *steps_out gets the supersteps run. A grid-barrier wait past timeout_ns (or any, with `force`)
// sets kErrTimeout in *err and ends the launch.
cudaError_t launch_msssp_loop(const MsArgs& a, uint32_t* const frontier[3], unsigned long long* changed,
                              uint64_t words, uint32_t max_steps, GridBar* bar, uint64_t timeout_ns, bool force,
                              uint32_t* err, uint32_t* steps_out, cudaStream_t s);
cudaError_t launch_msssp_init(uint32_t* dist, uint64_t n_vertices, const uint32_t* sources, uint32_t n_sources,
                              uint32_t* frontier, cudaStream_t s);
cudaError_t launch_popc(const uint32_t* bits, uint64_t words, unsigned long long* out, cudaStream_t s);
uint32_t msssp_grid(uint64_t units);

// sliced-ELL build on the device (sell_build.cu)
// The CSC a build reads: row v of the result is input row row_map[v] (or v),
// with its sources renumbered through src_map (or kept).
struct RowSource {
    const uint32_t* col_ptr;
    const uint32_t* src;
    const uint32_t* w;          // nullptr: unweighted
    const uint32_t* row_map;    // nullptr: identity
    const uint32_t* src_map;    // nullptr: identity
};
// rows of col_ptr (the result's offsets) sorted by source into ssrc / sw
// (rows of up to 256 edges by (source, weight), longer ones stably by
// source); sources are below n_src
cudaError_t launch_sort_rows(const uint32_t* col_ptr, uint32_t n, const RowSource& in, uint32_t n_src,
                             uint32_t* ssrc, uint32_t* sw, uint2* scratch_runs, uint32_t* scratch_cnt,
                             cudaStream_t s);   // scratch_runs: n + n_edges / 2048 + 1 entries
cudaError_t launch_sell_windows(const uint32_t* col_ptr, uint32_t n, uint32_t H, uint32_t* rows_out,
                                uint32_t* hub_out, uint32_t* nonhub_cnt, uint32_t* hub_cnt, cudaStream_t s);
cudaError_t launch_sell_slices(const uint32_t* col_ptr, uint32_t n, const uint32_t* rows_out,
                               const uint32_t* nonhub_cnt, const uint32_t* slice_base, uint32_t* perm,
                               uint32_t* width, uint64_t* off, uint32_t n_slices, bool g4, cudaStream_t s);
cudaError_t launch_sell_fill(const uint32_t* col_ptr, const uint32_t* ssrc, const uint32_t* sw, const uint32_t* perm,
                             const uint32_t* width, const uint64_t* off, uint32_t n_slices, uint32_t part,
                             uint32_t pad_id, bool g4, uint32_t* sell_src, uint32_t* sell_w, SellSlice* desc,
                             cudaStream_t s);
cudaError_t launch_hub_rows(const uint32_t* col_ptr, uint32_t n, const uint32_t* hub_out, const uint32_t* hub_cnt,
                            const uint32_t* hub_base, uint32_t* hub_list, uint32_t n_hub_rows, uint32_t T,
                            uint32_t* part_off, cudaStream_t s);
cudaError_t launch_hub_parts(const uint32_t* col_ptr, const uint32_t* hub_list, const uint32_t* part_off,
                             uint32_t n_hub_rows, uint32_t T, uint32_t part, uint32_t part_base, HubPart* hubs,
                             cudaStream_t s);
// slices by decreasing width (stable); afterwards scratch[0] holds the number
// of slices wider than 0 (the first offset of the last bin, width 0)
cudaError_t launch_order_slices(const SellSlice* in, uint32_t n, SellSlice* out, uint32_t* scratch, cudaStream_t s);
size_t order_slices_scratch_bytes(uint32_t n);

// vertex relabelling by decreasing in-degree (sell_build.cu): new2old / old2new
// and the renumbered offsets rcol[n + 1]; scratch: relabel_scratch_bytes
size_t relabel_scratch_bytes(uint32_t n);
cudaError_t launch_relabel(const uint32_t* col_ptr, uint32_t n, uint32_t* new2old, uint32_t* old2new, uint32_t* rcol,
                           uint32_t* scratch, cudaStream_t s);
// out[v] = in[map[v]] (gather) or out[map[v]] = in[v] (scatter)
cudaError_t launch_permute_u32(const uint32_t* in, const uint32_t* map, uint32_t n, uint32_t* out, bool scatter,
                               cudaStream_t s);

// serving (serve.cu): 64-slot personalized PageRank and slot management
cudaError_t launch_ppr_superstep(const PprArgs& a, cudaStream_t s);
uint32_t serve_grid(uint64_t warp_items);   // short-lived blocks for lanes sharing the GPU
// slots in `mask` start a new query: PPR columns get the messages of
// r_0 = e_src and its exact dangling mass; slot_source holds the sources
cudaError_t launch_ppr_slots_init(float* msg_cur, const float* inv_outdeg, uint64_t n_vertices, uint64_t mask,
                                  const uint32_t* slot_source, unsigned long long* dang_cur, cudaStream_t s);
// SSSP columns in `mask` get d = INF except d[src] = 0; sources join the frontier
cudaError_t launch_sssp_slots_init(uint32_t* dist, uint64_t n_vertices, uint64_t mask, const uint32_t* slot_source,
                                   uint32_t* frontier, cudaStream_t s);
// column slot[j] of mat[V][64] -> out[j][0..V) for j < n (row-tile transpose)
cudaError_t launch_gather_columns(const uint32_t* mat, uint64_t n_vertices, const GatherList& list, cudaStream_t s);

// Fixed point -> double (exact for sums below 2^53 units, else rounded once).
__host__ __device__ inline double fx_to_double(unsigned long long v) {
    return (double)v * (1.0 / (double)(1ULL << kFxShift));
}

// Fixed point (2^-60) -> fp32, from its two 32-bit halves (no FP64).
__host__ __device__ inline float fx_to_float(unsigned long long v) {
    const float hi = (float)(uint32_t)(v >> 32), lo = (float)(uint32_t)v;
    return fmaf(hi, 0x1p-28f, lo * 0x1p-60f);
}

// The base terms of a PageRank superstep from the exact dangling mass D of
// its input ranks (fixed point), for damping d and 1 / N: PageRank spreads
// (1-d) + d*D evenly, (1-d)/N + d*D/N to every vertex; personalized PageRank
// returns all of it to the source vertex (base_pr = 0 elsewhere).
// In fp32 only (the FP64 pipe of this GPU is narrow and every warp of the
// superstep forms these terms).
__host__ __device__ inline void pagerank_base(unsigned long long dangling_fx, float d, float inv_n, bool personalized,
                                              float* base_pr, float* base_src) {
    const float mass = fx_to_float(dangling_fx);   // D
    const float spread = fmaf(d, mass, 1.0f - d);
    if (!personalized) {
        *base_pr = *base_src = spread * inv_n;
    } else {
        *base_pr = 0.0f;
        *base_src = spread;
    }
}

#ifdef __CUDACC__
// x >= 0 (fp32) -> x * 2^60 truncated to an integer, exactly, with integer
// operations only; values below 2^-126 count as 0. For x <= 2 the result is
// below 2^62, so sums of up to 2 units of mass cannot overflow.
__device__ __forceinline__ unsigned long long fx_of(float x) {
    const uint32_t b = __float_as_uint(x);
    const int e = (int)((b >> 23) & 0xFFu);
    if (e == 0) return 0ull;
    const unsigned long long m = (unsigned long long)((b & 0x7FFFFFu) | 0x800000u);
    const int sh = e - 150 + kFxShift;
    if (sh >= 0) return m << sh;
    return (-sh) >= 64 ? 0ull : (m >> (-sh));
}
#endif

}  // namespace gxp
