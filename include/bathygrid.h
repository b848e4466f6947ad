/*
 * bathygrid — gridding scattered multibeam soundings on one GB300 GPU.
 *
 * C ABI of libbathygrid.so. Every entry point takes plain pointers and sizes,
 * returns a bg_status, and never throws. All coordinates are int32
 * centimetres, depths are float32 metres (positive down), and squared
 * distances are exact int64 cm^2.
 *
 * The method (arXiv 2505.22675, "Towards Real-Time Interpolation for
 * Enhanced AUV Deep Sea Mapping"):
 *   - each grid node gathers its nearest valid soundings (Sec. III-D: "nearest
 *     n valid candidate neighbors"; valid = depth not NaN, Sec. III-B);
 *   - from them it computes an inverse-distance-weighted estimate or an
 *     ordinary-kriging estimate (Sec. III-C: variogram equation, kriging
 *     system, estimate equation) with its kriging variance.
 * Neighbours are exact: the k smallest (d2, upload index) pairs, ties broken
 * by the lower upload index, returned in ascending order.
 *
 * Ownership: the library owns everything it allocates (sorted soundings,
 * spatial hash, queues); the caller owns input and output buffers. Errors:
 * outputs are undefined when a call fails; bg_last_error() gives a message
 * for the calling thread. Handles are thread-compatible (one thread at a time
 * per handle); the serving calls (bg_submit / bg_poll / bg_wait) are
 * thread-safe on one context.
 */
#ifndef BATHYGRID_H
#define BATHYGRID_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum bg_status {
    BG_OK = 0,
    BG_PENDING = 1,            /* bg_poll: the ticket has not finished yet */
    BG_ERR_INVALID_ARG = -1,   /* a null pointer, a size out of range, a bad handle */
    BG_ERR_OOM_BUDGET = -2,    /* the context's HBM budget would be exceeded */
    BG_ERR_CUDA = -3,          /* a CUDA runtime call failed (message in bg_last_error) */
    BG_ERR_TIMEOUT = -4,       /* bg_wait ran out of time, or a device wait gave up */
    BG_ERR_CANCELLED = -5,     /* the ticket was cancelled */
    BG_ERR_INTERNAL = -6,      /* a device-side check failed (message in bg_last_error) */
    BG_ERR_NOT_FOUND = -7      /* unknown ticket */
} bg_status;

typedef struct bg_ctx_s* bg_ctx_t;
typedef struct bg_grid_s* bg_grid_t;
typedef struct bg_soundings_s* bg_soundings_t;

/* Variogram models. Spherical: gamma(h) = c0 + c (1.5 h/a - 0.5 (h/a)^3) for
 * 0 < h <= a and c0 + c beyond. Exponential (the model printed in Sec. III-C,
 * variogram equation): gamma(h) = c0 + c (1 - exp(-h/a)). c0 = nugget,
 * c0 + c = sill (the TOTAL sill), a = range, h in metres. gamma(0) = 0 for a
 * sounding with itself and for a node on top of a sounding; two distinct
 * soundings at one position get c0. */
typedef enum bg_variogram_model {
    BG_VARIOGRAM_SPHERICAL = 0,
    BG_VARIOGRAM_EXPONENTIAL = 1
} bg_variogram_model;

typedef struct bg_variogram {
    int32_t model;     /* bg_variogram_model */
    float nugget_m2;   /* c0 >= 0 */
    float sill_m2;     /* total sill c0 + c, > c0 */
    float range_m;     /* a > 0 */
} bg_variogram;

typedef struct bg_soundings_info {
    int64_t n_total;        /* soundings passed to bg_soundings_upload */
    int64_t n_valid;        /* of them with a non-NaN depth */
    int32_t bbox_x0_cm, bbox_y0_cm;   /* min x, min y over valid soundings */
    int32_t bbox_x1_cm, bbox_y1_cm;   /* max x, max y over valid soundings (inclusive) */
    int32_t cell_cm;        /* spatial-hash cell side */
    int32_t ncx, ncy;       /* hash cells along x and y */
    int64_t device_bytes;   /* device memory held by this handle */
} bg_soundings_info;

/* ---------------------------------------------------------------- context */

/* Create a context on CUDA device `device` that may hold at most
 * `hbm_budget_bytes` of device memory (0 = no limit). Allocations that would
 * exceed the budget fail with BG_ERR_OOM_BUDGET. */
bg_status bg_ctx_create(int device, size_t hbm_budget_bytes, bg_ctx_t* out);

/* Destroy a context. Every grid and soundings handle made from it must have
 * been destroyed; pending serving tickets are cancelled and drained. */
bg_status bg_ctx_destroy(bg_ctx_t ctx);

/* Bytes of device memory the context holds now. */
bg_status bg_ctx_device_bytes(bg_ctx_t ctx, int64_t* out);

/* ------------------------------------------------------------------- grid */

/* Describe a regular output grid of nx * ny nodes. Node (i, j) sits at the
 * pixel centre (x0 + i*cell + cell/2, y0 + j*cell + cell/2) cm; outputs are
 * row-major, index j*nx + i. cell_cm must be even and > 0 so that node
 * coordinates are integers; every node coordinate must lie in
 * (-2^30, 2^30), and nx * ny <= 2^36. */
bg_status bg_grid_create(bg_ctx_t ctx, int32_t x0_cm, int32_t y0_cm, int32_t cell_cm,
                         int32_t nx, int32_t ny, bg_grid_t* out);
bg_status bg_grid_destroy(bg_grid_t grid);

/* -------------------------------------------------------------- soundings */

/* Upload n soundings and build the device spatial hash (a counting sort of
 * the valid soundings into uniform cells, Sec. III-D's neighbour helper made
 * exact).
 *   x_cm, y_cm, z_m: n values each; device pointers if on_device != 0, else
 *     host pointers (pageable or pinned), copied before the call returns.
 *     Soundings with NaN depth are dropped ("valid" neighbours, Sec. III-B).
 *     Valid coordinates must lie in (-2^30, 2^30); n < 2^31 - 1.
 *   cell_cm_hint: hash cell side in cm; 0 picks one from the data density.
 *     Results do not depend on it (neighbour search is exact), only speed.
 *   cuda_stream: cudaStream_t (NULL = legacy default stream). The call
 *     synchronizes this stream once to read the bounding box; the rest of
 *     the build is enqueued on it.
 * The handle keeps its own copy; the input buffers may be reused on return. */
bg_status bg_soundings_upload(bg_ctx_t ctx, const int32_t* x_cm, const int32_t* y_cm,
                              const float* z_m, int64_t n, int on_device, int32_t cell_cm_hint,
                              void* cuda_stream, bg_soundings_t* out);
bg_status bg_soundings_info_get(bg_soundings_t s, bg_soundings_info* out);
bg_status bg_soundings_destroy(bg_soundings_t s);

/* --------------------------------------------------------- interpolation */

/* Inverse-distance weighting over the k nearest valid soundings:
 * zhat = sum w_i z_i / sum w_i, w_i = d_i^-power. A node on top of a
 * sounding returns that sounding's depth (lowest upload index first). With
 * k_eff = min(k, n_valid) neighbours; no valid sounding gives NaN.
 *   k in [1, 32]; power > 0.
 *   depth_out: device, nx*ny float32, row-major.
 *   nbr_out: NULL or device nx*ny*k int32: the neighbours' upload indices in
 *     ascending (d2, index) order, -1 beyond k_eff.
 * Asynchronous on cuda_stream; the caller synchronizes. */
bg_status bg_interp_idw(bg_soundings_t s, bg_grid_t grid, int k, float power,
                        float* depth_out, int32_t* nbr_out, void* cuda_stream);

/* Local ordinary kriging over the k nearest valid soundings (Sec. III-C):
 * solves [Gamma 1; 1^T 0][lambda; mu] = [gamma_0; 1], returns
 * zhat = sum lambda_i z_i (Sec. III-C, estimate equation) and the kriging
 * variance sigma^2 = sum lambda_i gamma_i0 + mu. The system is reduced to a
 * symmetric positive definite one (lambda_0 and mu eliminated), factored by
 * Cholesky in FP32, and refined once: the residual b - A x is formed exactly
 * (A as 30-bit and x as 24-bit fixed point, products summed in 64-bit
 * integers, i.e. wider than FP64 would give). The weight sum closes in FP64.
 *   k in [1, 32]; v: variogram (see bg_variogram).
 *   depth_out, var_out: device, nx*ny float32 each (var_out may be NULL).
 *   nbr_out: as for bg_interp_idw.
 * A node with no valid sounding gets NaN. Asynchronous on cuda_stream. */
bg_status bg_interp_okrige(bg_soundings_t s, bg_grid_t grid, int k, const bg_variogram* v,
                           float* depth_out, float* var_out, int32_t* nbr_out,
                           void* cuda_stream);

/* IDW and ordinary kriging of the same grid in one pass: one exact k-NN search
 * of k_okrige neighbours per node feeds both, and the IDW takes the first
 * k_idw of them (the k_idw nearest, in the same (d2, index) order). Every
 * output is bitwise what bg_interp_idw and bg_interp_okrige give when called
 * one after the other; the k-NN search is not repeated. The paper runs its
 * methods separately; this entry point is for callers that want both grids.
 *   k_idw in [1, k_okrige], k_okrige in [1, 32]; power > 0; v as for
 *   bg_interp_okrige.
 *   idw_out, depth_out: device, nx*ny float32 each; var_out: device or NULL.
 * Asynchronous on cuda_stream. */
bg_status bg_interp_idw_okrige(bg_soundings_t s, bg_grid_t grid, int k_idw, float power,
                               int k_okrige, const bg_variogram* v, float* idw_out,
                               float* depth_out, float* var_out, void* cuda_stream);

/* bg_interp_idw_okrige with the three grids also delivered to host memory:
 * each row chunk's outputs are copied to idw_host / depth_host / var_host on
 * the context's copy stream as soon as that chunk's kernels have finished,
 * so the download overlaps the later chunks' work instead of following the
 * whole call. The device outputs are filled as by bg_interp_idw_okrige
 * (bitwise the same values).
 *   idw_out, depth_out, var_out, k_idw, power, k_okrige, v: as for
 *     bg_interp_idw_okrige.
 *   idw_host, depth_host, var_host: host, nx*ny float32 each, or NULL (that
 *     grid is not copied); var_host needs var_out. Page-locked memory
 *     (cudaMallocHost, cudaHostRegister) overlaps; pageable memory gives the
 *     same result without the overlap. The caller owns them.
 * Asynchronous on cuda_stream: later work on cuda_stream waits for the last
 * copy, so the host arrays are complete once cuda_stream is synchronized. */
bg_status bg_interp_idw_okrige_host(bg_soundings_t s, bg_grid_t grid, int k_idw, float power,
                                    int k_okrige, const bg_variogram* v, float* idw_out,
                                    float* depth_out, float* var_out, float* idw_host,
                                    float* depth_host, float* var_host, void* cuda_stream);

/* The same two methods at a list of query points instead of grid nodes: the
 * paper's hole filling interpolates the missing entries of a grid (Sec. IV,
 * Grid B) and its runtime tests interpolate batches of generated points
 * (Sec. IV, Grid A). Neighbours, weights and outputs follow the two calls
 * above exactly; a grid's nodes passed as points give bitwise the grid's
 * results.
 *   qx_cm, qy_cm: device, m int32 each: query coordinates in cm; a point
 *     outside (-2^30, 2^30) cm gets NaN outputs (and -1 neighbours). Points
 *     in scan order (each near the previous one) run fastest.
 *   m in [0, 2^40); outputs (device) have m entries (nbr_out m*k).
 * Asynchronous on cuda_stream; the caller synchronizes. */
bg_status bg_interp_idw_points(bg_soundings_t s, const int32_t* qx_cm, const int32_t* qy_cm,
                               int64_t m, int k, float power, float* depth_out, int32_t* nbr_out,
                               void* cuda_stream);
bg_status bg_interp_okrige_points(bg_soundings_t s, const int32_t* qx_cm, const int32_t* qy_cm,
                                  int64_t m, int k, const bg_variogram* v, float* depth_out,
                                  float* var_out, int32_t* nbr_out, void* cuda_stream);

/* ----------------------------------------------------------- gridded input */

/* Resampling of a regular grid (the paper's stencil methods on gridded data):
 *   BG_RESAMPLE_BILINEAR: the four nodes of the lattice cell that holds the
 *     query, weighted as in Sec. III-A;
 *   BG_RESAMPLE_CATMULL_ROM: the 4 x 4 nodes around that cell, the cubic C(t)
 *     of Sec. III-B along x on each row, then along y; stencil indices past
 *     the grid edge repeat the edge node.
 * A node is needed when its weight is not zero (a query on a node line
 * needs only that line). A needed NaN node (a missing value) gives NaN for
 * bilinear, which has no fallback (Sec. III-D), and makes Catmull-Rom fall
 * back to bilinear (Sec. III-B). A query outside the hull of the node
 * centres gets NaN. Arithmetic is FP32 on anomalies from one needed node.
 * No device memory is allocated; the calls are asynchronous on cuda_stream. */
typedef enum bg_resample_method {
    BG_RESAMPLE_BILINEAR = 0,
    BG_RESAMPLE_CATMULL_ROM = 1
} bg_resample_method;

/* src: device, nx*ny float32 node values, row-major, node (i, j) at
 *   (x0 + i*cell + cell/2, y0 + j*cell + cell/2) cm; cell even, nx, ny >= 2,
 *   nodes inside (-2^30, 2^30) cm.
 * qx_cm, qy_cm: device, m query coordinates (cm); out: device, m float32.
 * how_out: NULL or device m int8: 0 the method's value, 1 the bilinear
 *   fallback, 2 no value (NaN). */
bg_status bg_resample_points(const float* src, int32_t x0_cm, int32_t y0_cm, int32_t cell_cm,
                             int32_t nx, int32_t ny, int method, const int32_t* qx_cm,
                             const int32_t* qy_cm, int64_t m, float* out, int8_t* how_out,
                             void* cuda_stream);

/* The same at every node of an output grid (ox0, oy0, ocell even, onx, ony),
 * written row-major to out (device, onx*ony float32); how_out as above. The
 * paper's row-filling tests (Sec. IV, Grid A) are the output grid offset by
 * half a cell in y: the points halfway between successive rows. */
bg_status bg_resample_grid(const float* src, int32_t x0_cm, int32_t y0_cm, int32_t cell_cm,
                           int32_t nx, int32_t ny, int method, int32_t ox0_cm, int32_t oy0_cm,
                           int32_t ocell_cm, int32_t onx, int32_t ony, float* out,
                           int8_t* how_out, void* cuda_stream);

/* ---------------------------------------------------------------- serving */

/* A gridding request for bg_submit. Inputs and outputs are HOST memory; the
 * caller keeps them valid until the ticket completes. */
typedef struct bg_request {
    const int32_t* x_cm;       /* n soundings (host) */
    const int32_t* y_cm;
    const float* z_m;          /* NaN = invalid sounding */
    int64_t n;
    int32_t x0_cm, y0_cm, cell_cm, nx, ny;   /* output grid, as bg_grid_create */
    int32_t method;            /* 0 = IDW, 1 = ordinary kriging */
    int32_t k;                 /* neighbours, [1, 32] */
    float power;               /* IDW exponent (> 0) */
    bg_variogram variogram;    /* kriging model */
    float* depth_out;          /* host, nx*ny, row-major; contents unspecified
                                  until the ticket completes with BG_OK */
    float* var_out;            /* host, nx*ny kriging variance, or NULL */
} bg_request;

typedef struct bg_result {
    int32_t status;            /* bg_status of the request (BG_OK, BG_ERR_CANCELLED, ...) */
    int64_t nodes;             /* nx*ny */
    double t_submit_us;        /* context clock (microseconds): bg_submit */
    double t_start_us;         /* admission: the request's work was issued */
    double t_done_us;          /* its grids were in depth_out / var_out */
} bg_result;

/* Submit a request; returns with a ticket without waiting for any device
 * work. Requests are admitted in arrival order when one of the context's
 * stream slots is free and the context's HBM budget (bg_ctx_create) covers
 * the request's estimated device memory; admitted requests run concurrently
 * on the device (continuous batching). When nothing is queued ahead and a
 * slot is free, the calling thread issues the request itself (host copy into
 * pinned staging, asynchronous upload and kernel launches: tens of
 * microseconds for a typical tile) before returning; otherwise the request is
 * queued for the context's dispatcher thread. A request whose estimate alone
 * exceeds the budget is refused with BG_ERR_OOM_BUDGET. Thread-safe.
 * A context that serves runs a dispatcher thread, a completion thread and
 * three copy-out helper threads; the completion thread and the helpers spin
 * (yielding) while requests are in flight and sleep otherwise. */
bg_status bg_submit(bg_ctx_t ctx, const bg_request* req, uint64_t* ticket);

/* Never blocks. BG_PENDING while the ticket runs; otherwise BG_OK with *out
 * filled, and the ticket is released (do not poll it again). Unknown ticket:
 * BG_ERR_NOT_FOUND. */
bg_status bg_poll(bg_ctx_t ctx, uint64_t ticket, bg_result* out);

/* As bg_poll, but waits up to timeout_ms (< 0: no limit); BG_ERR_TIMEOUT when
 * the time runs out (the ticket stays valid). */
bg_status bg_wait(bg_ctx_t ctx, uint64_t ticket, int timeout_ms, bg_result* out);

/* Cancel a ticket that has not started; it completes with BG_ERR_CANCELLED.
 * A running ticket cannot be cancelled (BG_ERR_INVALID_ARG). */
bg_status bg_cancel(bg_ctx_t ctx, uint64_t ticket);

/* Requests waiting, requests on the device, and device bytes reserved by them. */
bg_status bg_serve_stats(bg_ctx_t ctx, int64_t* queued, int64_t* running, int64_t* reserved_bytes);

/* Stop serving: cancel queued tickets and wait for running ones (also done by
 * bg_ctx_destroy). */
bg_status bg_serve_shutdown(bg_ctx_t ctx);

/* ---------------------------------------------------------------- batches */

typedef struct bg_batch_s* bg_batch_t;

/* One tile of a batch: like bg_request, but inputs and outputs are DEVICE
 * pointers that stay valid (same addresses) for the life of the batch; their
 * contents may change between runs. */
typedef struct bg_tile {
    const int32_t* x_cm;       /* n soundings (device) */
    const int32_t* y_cm;
    const float* z_m;          /* NaN = invalid sounding */
    int64_t n;
    int32_t x0_cm, y0_cm, cell_cm, nx, ny;   /* output grid, as bg_grid_create */
    int32_t method;            /* 0 = IDW, 1 = ordinary kriging */
    int32_t k;                 /* neighbours, [1, 32] */
    float power;               /* IDW exponent (> 0) */
    bg_variogram variogram;    /* kriging model */
    float* depth_out;          /* device, nx*ny */
    float* var_out;            /* device, nx*ny kriging variance, or NULL */
} bg_tile;

/* Lay out a batch of tiles of uneven size: one set of device buffers for all
 * of them (charged to the context's budget), per-tile work descriptors on the
 * device, and the item lists of the persistent kernels. Results equal the
 * per-grid calls (bg_soundings_upload + bg_interp_idw / bg_interp_okrige)
 * bit for bit. The tiles array is copied. */
bg_status bg_batch_create(bg_ctx_t ctx, const bg_tile* tiles, int n_tiles, bg_batch_t* out);

/* Grid every tile of the batch, ordered after prior work on cuda_stream and
 * before later work on it. The first run records the launch sequence (hash
 * build for all tiles, one persistent k-NN/IDW kernel, one persistent solve
 * kernel per kriging system size) as a CUDA graph; later runs replay it, with
 * no host synchronization. */
bg_status bg_batch_run(bg_batch_t b, void* cuda_stream);

/* Hash cell side as a target number of soundings per cell (default 2); the
 * next run records a new graph. */
bg_status bg_batch_set_cell_target(bg_batch_t b, float soundings_per_cell);

/* Launch shape of the next runs (the next run records a new graph):
 *   knn_strip: grid nodes a k-NN thread takes one after another along x (1, 2
 *     or 4; from the second on, the previous node's k-th distance plus the
 *     step bounds the search), i.e. (16 knn_strip) x 8 nodes per k-NN item;
 *   solve_item: block batches of kriging systems per claimed solve item (1, 2,
 *     4, 8 or 16; 256 systems at K = 32 for 8, the default).
 * Results never depend on the shape. Other values: BG_ERR_INVALID_ARG. */
bg_status bg_batch_set_shape(bg_batch_t b, int knn_strip, int solve_item);

/* The batch's current cell target, k-NN strip length and solve item size
 * (any pointer may be NULL). */
bg_status bg_batch_get_config(bg_batch_t b, float* soundings_per_cell, int* knn_strip,
                              int* solve_item);

/* Autotune the cell target, the k-NN strip length and the solve item size by
 * coordinate descent: time each candidate of one knob on this batch with the
 * others at their best so far (every run is a real run, so outputs are
 * written) and keep the fastest. *best_out gets the cell target;
 * bg_batch_get_config gives all three. Results never depend on the choice. */
bg_status bg_batch_tune(bg_batch_t b, void* cuda_stream, float* best_out);

/* After the last run has finished: bit 0 = a tile had a coordinate outside
 * (-2^30, 2^30) and yields NaN; bit 1 = some node needed the wide-key pass. */
bg_status bg_batch_status(bg_batch_t b, int* flags);

bg_status bg_batch_destroy(bg_batch_t b);

/* ------------------------------------------------- allocation-free IDW */

/* IDW gridding that allocates no device memory, for callers that cannot call
 * cudaMalloc: processes that reserve all device memory up front, runtimes
 * whose allocator policy forbids device allocation on their worker threads,
 * and driver-owned threads that must not allocate. The paper has no
 * counterpart: this is a deployment variant of bg_soundings_upload +
 * bg_interp_idw with bitwise the same results.
 *   x_cm, y_cm, z_m: DEVICE pointers, n values each, n <= 262144 (larger n
 *     returns BG_ERR_INVALID_ARG before any device work).
 *   Grid (x0_cm, y0_cm, cell_cm, nx, ny), k, power, depth_out, nbr_out: as
 *     for bg_grid_create and bg_interp_idw; outputs are device pointers.
 *   cuda_stream: cudaStream_t; the call synchronizes it once (bounding box),
 *     so it must not be made inside stream capture, nor from a CUDA stream
 *     callback (where CUDA calls are not allowed).
 * Work space: one 16 MiB file-scope __device__ array that every device loading
 * the library holds until the process exits; each call looks up its device
 * address (cudaGetSymbolAddress) with the caller's device current. Every call
 * shares the array and clears what must start at zero; calls whose GPU work
 * overlaps race on it, so do not run two at once. No context is needed. */
bg_status bg_interp_idw_noalloc(const int32_t* x_cm, const int32_t* y_cm, const float* z_m,
                                int64_t n, int32_t x0_cm, int32_t y0_cm, int32_t cell_cm,
                                int32_t nx, int32_t ny, int k, float power, float* depth_out,
                                int32_t* nbr_out, void* cuda_stream);

/* ---------------------------------------------------------------- errors */

const char* bg_status_str(bg_status st);
/* Message for the last failed call on this thread ("" if none). */
const char* bg_last_error(void);
/* Library version string. */
const char* bg_version(void);
/* Number of CUDA kernels this library has launched since it was loaded
 * (all threads, all contexts); a diagnostic for benchmarks. */
bg_status bg_launch_count(uint64_t* out);

/* Kernel timing for benchmarks. While enabled, the context records CUDA
 * events on the launch stream around each interpolation kernel launch.
 * bg_profile_read waits for the recorded events and returns, per stage
 * (0 hash build, 1 IDW, 2 kriging k-NN ids, 3 kriging solve; n entries),
 * the summed milliseconds, the launch count and the grid nodes processed,
 * then clears the record. */
bg_status bg_profile_enable(bg_ctx_t ctx, int on);
bg_status bg_profile_read(bg_ctx_t ctx, double* ms, int64_t* launches, int64_t* units, int n);

/* Measured ALU peak of a GPU, for rooflines of kernels that no memory or
 * tensor-core bound describes. The paper has no counterpart: a measurement
 * helper. kind: 0 FP32 FMA (flop/s, an FMA counts 2), 1 INT32 multiply-add
 * (op/s), 2 INT32 add then xor (op/s, 2 per step), 3 FP64 FMA (flop/s). It
 * runs about 0.5 s of kernels of independent dependency chains on every SM of
 * `device` (CUDA events; best of three) and writes the rate to *ops_per_s
 * and the SM clock measured inside the kernel (clock64 ticks per globaltimer
 * ns) to *sm_mhz_out (may be NULL). Allocates a few KB of device memory. */
bg_status bg_alu_peak(int device, int kind, double* ops_per_s, double* sm_mhz_out);

#ifdef __cplusplus
}
#endif

#endif /* BATHYGRID_H */
