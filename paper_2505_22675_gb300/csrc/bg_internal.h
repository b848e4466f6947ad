// Internal types shared by the host side of libbathygrid and its kernels.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <nvtx3/nvToolsExt.h>

#include <atomic>
#include <mutex>
#include <string>
#include <vector>

#include "bathygrid.h"

namespace bg {

// ------------------------------------------------------------------ errors

void set_error(const std::string& msg);
bg_status cuda_fail(cudaError_t e, const char* what);

// Kernel launches made by this library since load (bg_launch_count).
extern std::atomic<uint64_t> g_launches;
inline void note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

#define BG_CUDA(call)                                      \
    do {                                                   \
        cudaError_t e_ = (call);                           \
        if (e_ != cudaSuccess) return bg::cuda_fail(e_, #call); \
    } while (0)

// -------------------------------------------------------------- device views

// Cell-sorted soundings plus the lookup tables of the uniform-cell hash.
// Passed by value to kernels.
struct HashView {
    const int4* rec;          // [n_valid] cell-sorted {x_cm, y_cm, z bits, upload index}
    const int4* orig;         // [n_total] upload order {x_cm, y_cm, z bits, valid}
    const int32_t* cell_start;// [ncx*ncy + 1] first record of each cell (row-major cells)
    const int32_t* sat;       // [(ncy+1)*(ncx+1)] summed-area table of per-cell counts
    int32_t hx0, hy0;         // hash origin (cm) = bbox min
    int32_t cs;               // cell side (cm)
    float inv_cs;             // 1 / cs
    int32_t ncx, ncy;
    int32_t n_valid;
    int32_t idx_bits;         // bits that hold an upload index in a packed key
    int32_t r0;               // first square half-width (cells) tried by the bound search
};

struct GridView {
    int32_t x0, y0, cell, nx, ny;
};

// A named range on the host timeline of a profiler (NVTX; header-only, a no-op
// unless a tool is attached): one per entry point that enqueues work.
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// IDW fused into a kriging pass: depth over the first k of the kriging's
// sorted neighbours, weights d^-power (out == nullptr: none).
struct IdwFuse {
    float* out = nullptr;
    float power = 2.0f;
    int k = 0;
};

// Host destinations of a grid call's outputs (page-locked; NULL: not copied):
// the rows of each chunk are copied on the stream cs once the chunk's kernels
// have finished on the caller's stream, so the copies overlap the next
// chunk's work; ev orders the two streams.
struct HostOut {
    float* idw = nullptr;
    float* depth = nullptr;
    float* var = nullptr;
    cudaStream_t cs = nullptr;
    cudaEvent_t ev = nullptr;
};

// Query points: m device coordinates (cm) in two arrays.
struct PointsView {
    const int32_t* x;
    const int32_t* y;
    int64_t m;
};

struct OkParams {
    int32_t model;
    float c0;      // nugget
    float c;       // partial sill = sill - nugget
    float sill;    // total sill
    float inv_a;   // 1 / range (1/m)
};

// ---------------------------------------------------------------- handles

struct Server;  // serving state of a context (serve.cu)

}  // namespace bg

// Per-context kernel timing (bg_profile_*): CUDA events recorded on the
// launch stream around each timed kernel, read back on request.
namespace bg {
struct ProfEntry {
    int stage;
    int64_t units;
    cudaEvent_t a, b;
};
struct Profiler {
    bool on = false;
    std::mutex mu;
    std::vector<ProfEntry> live;        // recorded, not yet read
    std::vector<cudaEvent_t> spare;     // reusable events
};
}  // namespace bg

struct bg_ctx_s {
    int device = 0;
    bg::Profiler prof;
    size_t budget = 0;                 // 0 = unlimited
    std::atomic<int64_t> in_use{0};
    std::mutex mu;
    cudaMemPool_t pool = nullptr;      // stream-ordered pool owned by the context
    std::mutex pin_mu;                 // guards h_pinned
    int32_t* h_pinned = nullptr;       // pinned host scratch for the bbox read-back
    int n_grids = 0, n_soundings = 0;
    bg::Server* server = nullptr;      // serving state (created by the first bg_submit)
    cudaStream_t copy_stream = nullptr;  // device-to-host copies that overlap later kernels
};

struct bg_grid_s {
    bg_ctx_s* ctx;
    bg::GridView g;
};

struct bg_soundings_s {
    bg_ctx_s* ctx;
    bg_soundings_info info;
    bg::HashView h;
    void* d_orig = nullptr;
    void* d_rec = nullptr;
    void* d_cell_start = nullptr;
    void* d_sat = nullptr;
    size_t bytes = 0;
};

namespace bg {

// Stage ids of the profiler.
enum ProfStage { kProfHash = 0, kProfIdw = 1, kProfKnnIds = 2, kProfSolve = 3, kProfStages = 4 };

// Scope that records events around the work it encloses when profiling is on.
struct ProfScope {
    bg_ctx_s* ctx;
    int stage;
    int64_t units;
    cudaStream_t st;
    cudaEvent_t a = nullptr, b = nullptr;
    ProfScope(bg_ctx_s* c, int stage_id, int64_t work_units, cudaStream_t s);
    ~ProfScope();
};

// Budgeted stream-ordered allocation (cudaMallocAsync) charged to a context.
bg_status dalloc(bg_ctx_s* ctx, void** p, size_t bytes, cudaStream_t st);
void dfree(bg_ctx_s* ctx, void* p, size_t bytes, cudaStream_t st);

// Bounding box and validity of soundings already scanned on the host.
struct HostBBox {
    int32_t x0, y0, x1, y1;   // min / max over valid soundings
    int64_t n_valid;
    int32_t out_of_range;     // valid soundings outside (-2^30, 2^30)
};

// Hash build: validate + pack + bbox, then counting sort and lookup tables.
// With `known`, the bounding box comes from the caller and the stream is
// never synchronized.
bg_status build_soundings(bg_ctx_s* ctx, const int32_t* x, const int32_t* y, const float* z,
                          int64_t n, int on_device, int32_t cell_hint, cudaStream_t st,
                          bg_soundings_s* s, const HostBBox* known = nullptr);

// Device bytes a hash build over n soundings (n_valid of them valid) may hold.
size_t soundings_bytes_estimate(int64_t n, int64_t n_valid);

// Free a soundings handle's device memory (stream-ordered on st).
void free_soundings(bg_soundings_s* s, cudaStream_t st);

// Start half-width (cells) for the k-NN bound search at this k.
int32_t start_halfwidth(const bg_soundings_s* s, int k);

// Device memory carved by the caller for a hash build that allocates nothing.
struct HashArena {
    int4* orig;          // n_max records
    int4* rec;           // n_max records
    int32_t* cell_start; // cells_max + 1
    int32_t* count;      // cells_max
    int32_t* sat;        // sat_max
    int32_t* bsum;       // bsum_max
    int32_t* csum;       // csum_max
    int32_t* acc;        // 8
    int64_t n_max, cells_max, sat_max, bsum_max, csum_max;
};

// The same hash build as build_soundings, into arena memory. Synchronizes the
// stream once (bounding box) through a pageable host buffer.
bg_status build_hash_in_arena(const int32_t* x, const int32_t* y, const float* z, int64_t n,
                              const HashArena& ar, cudaStream_t st, bg_soundings_s* s);

// Exclusive scan of n ints into out[0..n] (out[n] = total); out2 (may alias
// in) gets a copy of out[0..n). bsum: scan_blocks(n) + 1 ints of scratch.
int scan_blocks(int64_t n);
void launch_excl_scan(const int* in, int64_t n, int* out, int* out2, int* bsum, cudaStream_t st);

// IDW launch with a caller-provided device flag (one int) instead of an allocated one.
bg_status launch_idw_with_flag(const bg_soundings_s* s, const GridView& g, int k, float power,
                               float* depth, int32_t* nbr, int* d_flag, cudaStream_t st);

// Each call allocates (stream-ordered) a one-int flag that tells the wide-key
// pass whether the packed pass left nodes for it.
bg_status launch_idw(const bg_soundings_s* s, const GridView& g, int k, float power,
                     float* depth, int32_t* nbr, cudaStream_t st);
// fz: NULL, or an IDW to write in the same pass (fz->k <= k)
// ho: NULL, or host destinations that each row chunk's outputs are copied to
bg_status launch_okrige(const bg_soundings_s* s, const GridView& g, int k, const OkParams& p,
                        float* depth, float* var, int32_t* nbr, cudaStream_t st,
                        const IdwFuse* fz = nullptr, const HostOut* ho = nullptr);

// Gridded input (bilinear / Catmull-Rom) at query points or output-grid nodes;
// no allocation.
bg_status launch_resample_points(const float* src, const GridView& g, int method,
                                 const int32_t* qx, const int32_t* qy, int64_t m, float* out,
                                 int8_t* how, cudaStream_t st);
bg_status launch_resample_grid(const float* src, const GridView& g, int method, const GridView& o,
                               float* out, int8_t* how, cudaStream_t st);

// The same at a list of query points.
bg_status launch_idw_points(const bg_soundings_s* s, const PointsView& q, int k, float power,
                            float* depth, int32_t* nbr, cudaStream_t st);
bg_status launch_okrige_points(const bg_soundings_s* s, const PointsView& q, int k,
                               const OkParams& p, float* depth, float* var, int32_t* nbr,
                               cudaStream_t st);

}  // namespace bg
