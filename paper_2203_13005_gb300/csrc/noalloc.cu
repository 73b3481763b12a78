// gxp_superstep_min_noalloc: one SSSP or CC superstep over a CSC held in the
// caller's device memory, using no device allocation at all.
//
// Who needs it: callers that cannot call cudaMalloc — e.g. code whose device
// memory is entirely owned by another allocator (a framework's caching pool
// that has reserved the GPU), or latency-sensitive callers that cannot accept
// cudaMalloc's implicit device-wide synchronisation. The regular path
// (gxp_init / gxp_load_partition) allocates its own buffers; this entry point
// instead takes every input and output from the caller and keeps its
// internal scratch (edge-block descriptors, hub partials and counters, the
// statistics slot and the error word) in one fixed-size file-scope
// __device__ array.
//
// The array is a property of the loaded library: every GPU that loads it
// holds kNoAllocScratchBytes of device memory until the process exits. All
// calls on a device share the array and it keeps the last call's contents;
// the regions that must start at zero are cleared on every call. Calls that
// overlap on the GPU (e.g. issued to different streams without ordering) race
// on the array and must not be made.
#include <mutex>

#include "fault.hpp"
#include "gxp_internal.hpp"

namespace gxp {
namespace {

constexpr uint32_t kNoAllocTileItems = 2048;
constexpr uint32_t kNoAllocHubItems = 512;
constexpr uint64_t kNoAllocMaxTiles = 131072;   // 4 * n_vertices + n_edges <= 2^28
constexpr uint64_t kHeaderBytes = 4096;          // stats slot, error word, partition view
constexpr uint64_t kNoAllocScratchBytes =
    kHeaderBytes + kNoAllocMaxTiles * (4 + 4 + 4 + sizeof(Tile)) + 8 * (kNoAllocMaxTiles + 2);

static_assert(sizeof(StepStats) + sizeof(PartDev) + 16 <= kHeaderBytes, "header too small");

// The scratch. Host code must not take its address directly (that would be a
// host-side stand-in); it asks the runtime for the device address once per
// device.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

std::mutex g_mu;
constexpr int kMaxDevices = 64;
unsigned char* g_scratch_ptr[kMaxDevices] = {};

struct Layout {
    StepStats* stats;
    uint32_t* err;
    PartDev* part;
    uint32_t* hub_cnt;
    uint32_t* part_head;
    uint32_t* part_tail;
    uint64_t* cuts;
    Tile* tiles;
};

Layout layout_of(unsigned char* base) {
    Layout L;
    L.stats = reinterpret_cast<StepStats*>(base);
    L.err = reinterpret_cast<uint32_t*>(base + sizeof(StepStats));
    L.part = reinterpret_cast<PartDev*>(base + ((sizeof(StepStats) + 4 + 15) & ~size_t(15)));
    unsigned char* p = base + kHeaderBytes;
    L.hub_cnt = reinterpret_cast<uint32_t*>(p);
    p += 4 * kNoAllocMaxTiles;
    L.part_head = reinterpret_cast<uint32_t*>(p);
    p += 4 * kNoAllocMaxTiles;
    L.part_tail = reinterpret_cast<uint32_t*>(p);
    p += 4 * kNoAllocMaxTiles;
    L.cuts = reinterpret_cast<uint64_t*>(p);
    p += 8 * (kNoAllocMaxTiles + 2);
    L.tiles = reinterpret_cast<Tile*>(p);
    return L;
}

// Device address of the scratch on the current device (set-up on first use).
gxp_status scratch_for_current_device(unsigned char** out) {
    int dev = -1;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GXP_E_CUDA;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void* ptr = nullptr;
        if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || ptr == nullptr) {
            cudaGetLastError();
            return GXP_E_CUDA;
        }
        g_scratch_ptr[dev] = static_cast<unsigned char*>(ptr);
    }
    *out = g_scratch_ptr[dev];
    return GXP_OK;
}

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

bool overlap(const void* a, const void* b, size_t bytes) {
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + bytes && y < x + bytes;
}

// Read the scratch's error word (enqueued after the kernels that set it) and
// wait for the stream.
gxp_status read_error(const Layout& L, cudaStream_t s, uint32_t* err) {
    if (cudaMemcpyAsync(err, L.err, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return GXP_E_CUDA;
    return GXP_OK;
}

}  // namespace
}  // namespace gxp

extern "C" GXP_API gxp_status gxp_superstep_min_noalloc(gxp_algo algo, uint32_t n_vertices, uint64_t n_edges,
                                                        const uint32_t* d_col_ptr, const uint32_t* d_src,
                                                        const uint32_t* d_w, const uint32_t* d_cur,
                                                        uint32_t* d_next, uint64_t* n_changed, void* stream) {
    using namespace gxp;
    if (algo != GXP_ALGO_SSSP && algo != GXP_ALGO_CC) return GXP_E_UNSUPPORTED;
    if (n_vertices == 0 || n_vertices >= 0xFFFFFFFFu || n_edges > 0xFFFFFFFFull) return GXP_E_INVAL;
    if (!d_col_ptr || !d_cur || !d_next || (n_edges && !d_src) || (algo == GXP_ALGO_SSSP && n_edges && !d_w))
        return GXP_E_INVAL;
    if (!aligned16(d_col_ptr) || !aligned16(d_cur) || (d_src && !aligned16(d_src)) || (d_w && !aligned16(d_w)))
        return GXP_E_INVAL;
    if (overlap(d_cur, d_next, 4ull * n_vertices)) return GXP_E_INVAL;   // Jacobi: two distinct buffers
    const uint32_t n_tiles = tile_count(n_vertices, n_edges, kNoAllocTileItems);
    if ((uint64_t)n_tiles > kNoAllocMaxTiles) return GXP_E_INVAL;   // beyond the scratch's fixed size
    unsigned char* base = nullptr;
    gxp_status st = scratch_for_current_device(&base);
    if (st != GXP_OK) return st;
    const Layout L = layout_of(base);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    const Algo a = algo == GXP_ALGO_SSSP ? Algo::SSSP : Algo::CC;

    // clear what must start at zero: stats slot, error word, hub arrival counters
    if (cudaMemsetAsync(base, 0, sizeof(StepStats) + 4, s) != cudaSuccess) return GXP_E_CUDA;
    if (n_tiles && cudaMemsetAsync(L.hub_cnt, 0, 4ull * n_tiles, s) != cudaSuccess) return GXP_E_CUDA;
    const PartDev pd{d_col_ptr, d_src, algo == GXP_ALGO_SSSP ? d_w : nullptr, n_vertices, 0u, 0u, 0u, n_edges};
    if (cudaMemcpyAsync(L.part, &pd, sizeof(pd), cudaMemcpyHostToDevice, s) != cudaSuccess) return GXP_E_CUDA;
    // The tiles are cut from the offsets and the kernel stages them with bulk
    // copies sized from those cuts: check the CSC before either runs.
    uint32_t err = 0;
    if (launch_validate_csc(d_col_ptr, n_vertices, d_src, n_edges, n_vertices, L.err, s) != cudaSuccess)
        return GXP_E_CUDA;
    if ((st = read_error(L, s, &err)) != GXP_OK) return st;
    if (err & kErrInput) return GXP_E_INVAL;
    if (err & kErrBounds) return GXP_E_BOUNDS;
    if (launch_build_tiles(d_col_ptr, n_vertices, (uint32_t)n_edges, kNoAllocTileItems, kNoAllocHubItems, 0u, 0u,
                           n_tiles, L.tiles, L.cuts, s) != cudaSuccess)
        return GXP_E_CUDA;
    SuperstepArgs args{};
    args.tiles = L.tiles;
    args.parts = L.part;
    args.n_tiles = n_tiles;
    args.own_cur = d_cur;
    args.own_nxt = d_next;
    args.ghost = nullptr;
    args.changed_bits = nullptr;
    args.part_head = L.part_head;
    args.part_tail = L.part_tail;
    args.hub_cnt = L.hub_cnt;
    args.stats_in = L.stats;
    args.stats_out = L.stats;
    args.stats_clear = nullptr;
    args.err = L.err;
    args.timeout_ns = 2000000000ull;
    args.force_timeout = fault_plan_from_env().timeout ? 1u : 0u;
    args.check_bounds = 1;
    args.max_items = kNoAllocTileItems + kNoAllocHubItems;
    if (launch_superstep(a, args, superstep_smem_bytes(a, args.max_items), s) != cudaSuccess) return GXP_E_CUDA;

    StepStats host_stats;
    if (cudaMemcpyAsync(&host_stats, L.stats, sizeof(host_stats), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        return GXP_E_CUDA;
    if ((st = read_error(L, s, &err)) != GXP_OK) return st;
    if (err & (kErrTimeout | kErrDrain)) return GXP_E_TIMEOUT;
    if (err & kErrBounds) return GXP_E_BOUNDS;
    if (n_changed) {
        unsigned long long c = 0;
        for (int i = 0; i < kStatLanes; ++i) c += host_stats.changed[i];
        *n_changed = c;
    }
    return GXP_OK;
}
