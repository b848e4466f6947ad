// extern "C" entry points of libbathygrid.so (declared in include/bathygrid.h):
// argument checks, handle lifetimes, the HBM budget, and dispatch to kernels.
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>

#include "bg_internal.h"

namespace bg {

namespace {
thread_local std::string g_last_error;

bool finite_pos(float v) { return std::isfinite(v) && v > 0.0f; }

// Every node coordinate x0 + i*cell + cell/2 must stay inside (-2^30, 2^30).
bool grid_in_range(int64_t x0, int64_t y0, int64_t cell, int64_t nx, int64_t ny) {
    const int64_t lim = (int64_t)1 << 30;
    const int64_t xa = x0 + cell / 2, xb = x0 + (nx - 1) * cell + cell / 2;
    const int64_t ya = y0 + cell / 2, yb = y0 + (ny - 1) * cell + cell / 2;
    return xa > -lim && xb < lim && ya > -lim && yb < lim;
}

// RAII: make the context's device current for the duration of a call.
struct DeviceGuard {
    int prev = -1;
    bool ok = true;
    explicit DeviceGuard(int dev) {
        if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
        if (prev != dev) ok = cudaSetDevice(dev) == cudaSuccess;
    }
    ~DeviceGuard() {
        if (prev >= 0) cudaSetDevice(prev);
    }
};
}  // namespace

std::atomic<uint64_t> g_launches{0};

void set_error(const std::string& msg) { g_last_error = msg; }

bg_status cuda_fail(cudaError_t e, const char* what) {
    set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
    return BG_ERR_CUDA;
}

bg_status dalloc(bg_ctx_s* ctx, void** p, size_t bytes, cudaStream_t st) {
    *p = nullptr;
    if (bytes == 0) return BG_OK;
    const int64_t now = ctx->in_use.fetch_add((int64_t)bytes) + (int64_t)bytes;
    if (ctx->budget && now > (int64_t)ctx->budget) {
        ctx->in_use.fetch_sub((int64_t)bytes);
        set_error("HBM budget exceeded: need " + std::to_string(bytes) + " more bytes, " +
                  std::to_string(now - (int64_t)bytes) + " of " + std::to_string(ctx->budget) +
                  " in use");
        return BG_ERR_OOM_BUDGET;
    }
    const cudaError_t e = cudaMallocFromPoolAsync(p, bytes, ctx->pool, st);
    if (e != cudaSuccess) {
        ctx->in_use.fetch_sub((int64_t)bytes);
        *p = nullptr;
        return cuda_fail(e, "cudaMallocAsync");
    }
    return BG_OK;
}

void dfree(bg_ctx_s* ctx, void* p, size_t bytes, cudaStream_t st) {
    if (!p) return;
    cudaFreeAsync(p, st);
    ctx->in_use.fetch_sub((int64_t)bytes);
}

void free_soundings(bg_soundings_s* s, cudaStream_t st) {
    bg_ctx_s* ctx = s->ctx;
    const size_t ncells = (size_t)s->info.ncx * (size_t)s->info.ncy;
    dfree(ctx, s->d_orig, (size_t)s->info.n_total * 16, st);
    if (s->d_cell_start) dfree(ctx, s->d_cell_start, (ncells + 1) * 4, st);
    if (s->d_sat) dfree(ctx, s->d_sat, (size_t)(s->info.ncx + 1) * (s->info.ncy + 1) * 4, st);
    if (s->d_rec) dfree(ctx, s->d_rec, (size_t)s->info.n_valid * 16, st);
    s->d_orig = s->d_cell_start = s->d_sat = s->d_rec = nullptr;
}

static cudaEvent_t take_event(Profiler& pr) {
    cudaEvent_t e = nullptr;
    if (!pr.spare.empty()) {
        e = pr.spare.back();
        pr.spare.pop_back();
    } else if (cudaEventCreate(&e) != cudaSuccess) {
        e = nullptr;
    }
    return e;
}

ProfScope::ProfScope(bg_ctx_s* c, int stage_id, int64_t work_units, cudaStream_t s)
    : ctx(c), stage(stage_id), units(work_units), st(s) {
    if (!ctx || !ctx->prof.on) return;
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    a = take_event(ctx->prof);
    b = take_event(ctx->prof);
    if (a) cudaEventRecord(a, st);
}

ProfScope::~ProfScope() {
    if (!a || !b) return;
    cudaEventRecord(b, st);
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    ctx->prof.live.push_back(ProfEntry{stage, units, a, b});
}

size_t soundings_bytes_estimate(int64_t n, int64_t n_valid) {
    // records (2 x 16 B), cell tables (~2 soundings per cell: cell_start + SAT
    // + counts), host staging (12 B), small scratch
    return (size_t)n * 16 + (size_t)n_valid * 16 + (size_t)n * 12 + (size_t)n_valid * 8 +
           (size_t)(1 << 20);
}

}  // namespace bg

using namespace bg;

#define BG_REQUIRE(cond, msg)              \
    do {                                   \
        if (!(cond)) {                     \
            bg::set_error(msg);            \
            return BG_ERR_INVALID_ARG;     \
        }                                  \
    } while (0)

extern "C" {

const char* bg_version(void) { return "bathygrid 0.1.0 (sm_103a)"; }

const char* bg_last_error(void) { return bg::g_last_error.c_str(); }

bg_status bg_launch_count(uint64_t* out) {
    BG_REQUIRE(out, "out is NULL");
    *out = bg::g_launches.load();
    return BG_OK;
}

const char* bg_status_str(bg_status st) {
    switch (st) {
        case BG_OK: return "BG_OK";
        case BG_PENDING: return "BG_PENDING";
        case BG_ERR_INVALID_ARG: return "BG_ERR_INVALID_ARG";
        case BG_ERR_OOM_BUDGET: return "BG_ERR_OOM_BUDGET";
        case BG_ERR_CUDA: return "BG_ERR_CUDA";
        case BG_ERR_TIMEOUT: return "BG_ERR_TIMEOUT";
        case BG_ERR_CANCELLED: return "BG_ERR_CANCELLED";
        case BG_ERR_INTERNAL: return "BG_ERR_INTERNAL";
        case BG_ERR_NOT_FOUND: return "BG_ERR_NOT_FOUND";
    }
    return "BG_UNKNOWN";
}

bg_status bg_ctx_create(int device, size_t hbm_budget_bytes, bg_ctx_t* out) {
    BG_REQUIRE(out, "out is NULL");
    *out = nullptr;
    int ndev = 0;
    BG_CUDA(cudaGetDeviceCount(&ndev));
    BG_REQUIRE(device >= 0 && device < ndev, "device index out of range");
    DeviceGuard dg(device);
    if (!dg.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    bg_ctx_s* c = new (std::nothrow) bg_ctx_s();
    if (!c) return BG_ERR_INTERNAL;
    c->device = device;
    c->budget = hbm_budget_bytes;
    // the context's own pool keeps freed blocks for reuse (no release threshold),
    // so repeated uploads and calls do not map and unmap memory each time
    cudaMemPoolProps props{};
    props.allocType = cudaMemAllocationTypePinned;
    props.location.type = cudaMemLocationTypeDevice;
    props.location.id = device;
    cudaError_t e = cudaMemPoolCreate(&c->pool, &props);
    if (e == cudaSuccess) {
        uint64_t keep = UINT64_MAX;
        e = cudaMemPoolSetAttribute(c->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    if (e == cudaSuccess) e = cudaMallocHost((void**)&c->h_pinned, 64 * sizeof(int32_t));
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->copy_stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        if (c->h_pinned) cudaFreeHost(c->h_pinned);
        if (c->pool) cudaMemPoolDestroy(c->pool);
        delete c;
        return cuda_fail(e, "context set-up");
    }
    *out = c;
    return BG_OK;
}

bg_status bg_profile_enable(bg_ctx_t ctx, int on) {
    BG_REQUIRE(ctx, "ctx is NULL");
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    ctx->prof.on = on != 0;
    return BG_OK;
}

bg_status bg_profile_read(bg_ctx_t ctx, double* ms, int64_t* launches, int64_t* units, int n) {
    BG_REQUIRE(ctx && ms && launches && units && n > 0, "bad arguments");
    for (int i = 0; i < n; ++i) {
        ms[i] = 0.0;
        launches[i] = 0;
        units[i] = 0;
    }
    std::lock_guard<std::mutex> lk(ctx->prof.mu);
    for (const auto& e : ctx->prof.live) {
        cudaEventSynchronize(e.b);
        float t = 0.0f;
        cudaEventElapsedTime(&t, e.a, e.b);
        if (e.stage >= 0 && e.stage < n) {
            ms[e.stage] += t;
            launches[e.stage] += 1;
            units[e.stage] += e.units;
        }
        ctx->prof.spare.push_back(e.a);
        ctx->prof.spare.push_back(e.b);
    }
    ctx->prof.live.clear();
    return BG_OK;
}

bg_status bg_ctx_device_bytes(bg_ctx_t ctx, int64_t* out) {
    BG_REQUIRE(ctx && out, "NULL argument");
    *out = ctx->in_use.load();
    return BG_OK;
}

bg_status bg_ctx_destroy(bg_ctx_t ctx) {
    BG_REQUIRE(ctx, "ctx is NULL");
    BG_REQUIRE(ctx->n_grids == 0 && ctx->n_soundings == 0,
               "destroy every grid and soundings handle before the context");
    DeviceGuard dg(ctx->device);
    bg_serve_shutdown(ctx);
    cudaDeviceSynchronize();
    for (auto& e : ctx->prof.live) {
        cudaEventDestroy(e.a);
        cudaEventDestroy(e.b);
    }
    for (auto e : ctx->prof.spare) cudaEventDestroy(e);
    cudaStreamDestroy(ctx->copy_stream);
    cudaFreeHost(ctx->h_pinned);
    cudaMemPoolDestroy(ctx->pool);
    delete ctx;
    return BG_OK;
}

bg_status bg_grid_create(bg_ctx_t ctx, int32_t x0_cm, int32_t y0_cm, int32_t cell_cm, int32_t nx,
                         int32_t ny, bg_grid_t* out) {
    BG_REQUIRE(ctx && out, "NULL argument");
    *out = nullptr;
    BG_REQUIRE(cell_cm > 0 && cell_cm % 2 == 0, "cell_cm must be even and > 0");
    BG_REQUIRE(nx > 0 && ny > 0, "nx and ny must be > 0");
    BG_REQUIRE((int64_t)nx * ny <= ((int64_t)1 << 36), "grid too large (more than 2^36 nodes)");
    BG_REQUIRE(grid_in_range(x0_cm, y0_cm, cell_cm, nx, ny),
               "grid node coordinates must lie in (-2^30, 2^30) cm");
    bg_grid_s* g = new (std::nothrow) bg_grid_s();
    if (!g) return BG_ERR_INTERNAL;
    g->ctx = ctx;
    g->g = GridView{x0_cm, y0_cm, cell_cm, nx, ny};
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->n_grids++;
    }
    *out = g;
    return BG_OK;
}

bg_status bg_grid_destroy(bg_grid_t grid) {
    BG_REQUIRE(grid, "grid is NULL");
    {
        std::lock_guard<std::mutex> lk(grid->ctx->mu);
        grid->ctx->n_grids--;
    }
    delete grid;
    return BG_OK;
}

bg_status bg_soundings_upload(bg_ctx_t ctx, const int32_t* x_cm, const int32_t* y_cm,
                              const float* z_m, int64_t n, int on_device, int32_t cell_cm_hint,
                              void* cuda_stream, bg_soundings_t* out) {
    bg::NvtxRange nvtx("bg_soundings_upload");
    BG_REQUIRE(ctx && out, "NULL argument");
    *out = nullptr;
    BG_REQUIRE(n >= 0 && n < ((int64_t)1 << 31) - 1, "n must be in [0, 2^31 - 1)");
    BG_REQUIRE(n == 0 || (x_cm && y_cm && z_m), "NULL input pointer");
    BG_REQUIRE(cell_cm_hint >= 0, "cell_cm_hint must be >= 0");
    DeviceGuard dg(ctx->device);
    if (!dg.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    bg_soundings_s* s = new (std::nothrow) bg_soundings_s();
    if (!s) return BG_ERR_INTERNAL;
    s->ctx = ctx;
    const cudaStream_t st = (cudaStream_t)cuda_stream;
    const bg_status rc = build_soundings(ctx, x_cm, y_cm, z_m, n, on_device, cell_cm_hint, st, s);
    if (rc != BG_OK) {
        free_soundings(s, st);
        delete s;
        return rc;
    }
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->n_soundings++;
    }
    *out = s;
    return BG_OK;
}

bg_status bg_soundings_info_get(bg_soundings_t s, bg_soundings_info* out) {
    BG_REQUIRE(s && out, "NULL argument");
    *out = s->info;
    return BG_OK;
}

bg_status bg_soundings_destroy(bg_soundings_t s) {
    BG_REQUIRE(s, "soundings is NULL");
    bg_ctx_s* ctx = s->ctx;
    DeviceGuard dg(ctx->device);
    // stream-ordered frees on the legacy stream: work already queued on other
    // streams that reads this handle must be complete (the caller's contract)
    free_soundings(s, 0);
    {
        std::lock_guard<std::mutex> lk(ctx->mu);
        ctx->n_soundings--;
    }
    delete s;
    return BG_OK;
}

static bg_status check_interp(bg_soundings_t s, bg_grid_t grid, int k, float* depth) {
    BG_REQUIRE(s && grid, "NULL handle");
    BG_REQUIRE(s->ctx == grid->ctx, "soundings and grid belong to different contexts");
    BG_REQUIRE(depth, "depth_out is NULL");
    BG_REQUIRE(k >= 1 && k <= 32, "k must be in [1, 32]");
    return BG_OK;
}

bg_status bg_interp_idw(bg_soundings_t s, bg_grid_t grid, int k, float power, float* depth_out,
                        int32_t* nbr_out, void* cuda_stream) {
    bg::NvtxRange nvtx("bg_interp_idw");
    bg_status rc = check_interp(s, grid, k, depth_out);
    if (rc != BG_OK) return rc;
    BG_REQUIRE(finite_pos(power), "power must be finite and > 0");
    DeviceGuard dg(s->ctx->device);
    if (!dg.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    return launch_idw(s, grid->g, k, power, depth_out, nbr_out, (cudaStream_t)cuda_stream);
}

static bool okrige_params(const bg_variogram* v, OkParams* p) {
    if (!v) return set_error("variogram is NULL"), false;
    if (v->model != BG_VARIOGRAM_SPHERICAL && v->model != BG_VARIOGRAM_EXPONENTIAL)
        return set_error("unknown variogram model"), false;
    if (!(std::isfinite(v->nugget_m2) && v->nugget_m2 >= 0.0f))
        return set_error("nugget must be >= 0"), false;
    if (!(std::isfinite(v->sill_m2) && v->sill_m2 > v->nugget_m2))
        return set_error("sill must exceed the nugget"), false;
    if (!finite_pos(v->range_m)) return set_error("range must be > 0"), false;
    *p = OkParams{v->model, v->nugget_m2, v->sill_m2 - v->nugget_m2, v->sill_m2, 1.0f / v->range_m};
    return true;
}

bg_status bg_interp_okrige(bg_soundings_t s, bg_grid_t grid, int k, const bg_variogram* v,
                           float* depth_out, float* var_out, int32_t* nbr_out, void* cuda_stream) {
    bg::NvtxRange nvtx("bg_interp_okrige");
    bg_status rc = check_interp(s, grid, k, depth_out);
    if (rc != BG_OK) return rc;
    OkParams p;
    if (!okrige_params(v, &p)) return BG_ERR_INVALID_ARG;
    DeviceGuard dg(s->ctx->device);
    if (!dg.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    return launch_okrige(s, grid->g, k, p, depth_out, var_out, nbr_out, (cudaStream_t)cuda_stream);
}


bg_status bg_interp_idw_okrige(bg_soundings_t s, bg_grid_t grid, int k_idw, float power,
                               int k_okrige, const bg_variogram* v, float* idw_out,
                               float* depth_out, float* var_out, void* cuda_stream) {
    bg::NvtxRange nvtx("bg_interp_idw_okrige");
    bg_status rc = check_interp(s, grid, k_okrige, depth_out);
    if (rc != BG_OK) return rc;
    BG_REQUIRE(idw_out, "idw_out is NULL");
    BG_REQUIRE(k_idw >= 1 && k_idw <= k_okrige, "k_idw must be in [1, k_okrige]");
    BG_REQUIRE(finite_pos(power), "power must be finite and > 0");
    OkParams p;
    if (!okrige_params(v, &p)) return BG_ERR_INVALID_ARG;
    DeviceGuard dg(s->ctx->device);
    if (!dg.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    IdwFuse fz;
    fz.out = idw_out;
    fz.power = power;
    fz.k = k_idw;
    return launch_okrige(s, grid->g, k_okrige, p, depth_out, var_out, nullptr,
                         (cudaStream_t)cuda_stream, &fz);
}

bg_status bg_interp_idw_okrige_host(bg_soundings_t s, bg_grid_t grid, int k_idw, float power,
                                    int k_okrige, const bg_variogram* v, float* idw_out,
                                    float* depth_out, float* var_out, float* idw_host,
                                    float* depth_host, float* var_host, void* cuda_stream) {
    bg::NvtxRange nvtx("bg_interp_idw_okrige_host");
    bg_status rc = check_interp(s, grid, k_okrige, depth_out);
    if (rc != BG_OK) return rc;
    BG_REQUIRE(idw_out, "idw_out is NULL");
    BG_REQUIRE(!var_host || var_out, "var_host needs var_out");
    BG_REQUIRE(k_idw >= 1 && k_idw <= k_okrige, "k_idw must be in [1, k_okrige]");
    BG_REQUIRE(finite_pos(power), "power must be finite and > 0");
    OkParams p;
    if (!okrige_params(v, &p)) return BG_ERR_INVALID_ARG;
    DeviceGuard dg(s->ctx->device);
    if (!dg.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    IdwFuse fz;
    fz.out = idw_out;
    fz.power = power;
    fz.k = k_idw;
    HostOut ho;
    ho.idw = idw_host;
    ho.depth = depth_host;
    ho.var = var_host;
    ho.cs = s->ctx->copy_stream;
    BG_CUDA(cudaEventCreateWithFlags(&ho.ev, cudaEventDisableTiming));
    rc = launch_okrige(s, grid->g, k_okrige, p, depth_out, var_out, nullptr,
                       (cudaStream_t)cuda_stream, &fz, &ho);
    cudaEventDestroy(ho.ev);  // released once its last record completes
    return rc;
}

static bg_status check_points(bg_soundings_t s, const int32_t* qx, const int32_t* qy, int64_t m,
                              int k, float* depth) {
    BG_REQUIRE(s, "NULL handle");
    BG_REQUIRE(m >= 0 && m < ((int64_t)1 << 40), "m must be in [0, 2^40)");
    BG_REQUIRE(m == 0 || (qx && qy && depth), "NULL query or output pointer");
    BG_REQUIRE(k >= 1 && k <= 32, "k must be in [1, 32]");
    return BG_OK;
}


bg_status bg_interp_idw_points(bg_soundings_t s, const int32_t* qx_cm, const int32_t* qy_cm,
                               int64_t m, int k, float power, float* depth_out, int32_t* nbr_out,
                               void* cuda_stream) {
    bg::NvtxRange nvtx("bg_interp_idw_points");
    bg_status rc = check_points(s, qx_cm, qy_cm, m, k, depth_out);
    if (rc != BG_OK) return rc;
    BG_REQUIRE(finite_pos(power), "power must be finite and > 0");
    DeviceGuard dg(s->ctx->device);
    if (!dg.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    return launch_idw_points(s, PointsView{qx_cm, qy_cm, m}, k, power, depth_out, nbr_out,
                             (cudaStream_t)cuda_stream);
}

bg_status bg_interp_okrige_points(bg_soundings_t s, const int32_t* qx_cm, const int32_t* qy_cm,
                                  int64_t m, int k, const bg_variogram* v, float* depth_out,
                                  float* var_out, int32_t* nbr_out, void* cuda_stream) {
    bg::NvtxRange nvtx("bg_interp_okrige_points");
    bg_status rc = check_points(s, qx_cm, qy_cm, m, k, depth_out);
    if (rc != BG_OK) return rc;
    OkParams p;
    if (!okrige_params(v, &p)) return BG_ERR_INVALID_ARG;
    DeviceGuard dg(s->ctx->device);
    if (!dg.ok) return cuda_fail(cudaGetLastError(), "cudaSetDevice");
    return launch_okrige_points(s, PointsView{qx_cm, qy_cm, m}, k, p, depth_out, var_out, nbr_out,
                                (cudaStream_t)cuda_stream);
}

static bg_status check_source(const float* src, int32_t x0, int32_t y0, int32_t cell, int32_t nx,
                              int32_t ny, int method) {
    BG_REQUIRE(src, "src is NULL");
    BG_REQUIRE(cell > 0 && cell % 2 == 0, "cell_cm must be even and > 0");
    BG_REQUIRE(nx >= 2 && ny >= 2, "the source grid needs at least 2 x 2 nodes");
    BG_REQUIRE(grid_in_range(x0, y0, cell, nx, ny), "source nodes must lie in (-2^30, 2^30) cm");
    BG_REQUIRE(method == BG_RESAMPLE_BILINEAR || method == BG_RESAMPLE_CATMULL_ROM,
               "unknown resampling method");
    return BG_OK;
}

bg_status bg_resample_points(const float* src, int32_t x0_cm, int32_t y0_cm, int32_t cell_cm,
                             int32_t nx, int32_t ny, int method, const int32_t* qx_cm,
                             const int32_t* qy_cm, int64_t m, float* out, int8_t* how_out,
                             void* cuda_stream) {
    bg::NvtxRange nvtx("bg_resample_points");
    bg_status rc = check_source(src, x0_cm, y0_cm, cell_cm, nx, ny, method);
    if (rc != BG_OK) return rc;
    BG_REQUIRE(m >= 0 && m < ((int64_t)1 << 40), "m must be in [0, 2^40)");
    BG_REQUIRE(m == 0 || (qx_cm && qy_cm && out), "NULL query or output pointer");
    return launch_resample_points(src, GridView{x0_cm, y0_cm, cell_cm, nx, ny}, method, qx_cm,
                                  qy_cm, m, out, how_out, (cudaStream_t)cuda_stream);
}

bg_status bg_resample_grid(const float* src, int32_t x0_cm, int32_t y0_cm, int32_t cell_cm,
                           int32_t nx, int32_t ny, int method, int32_t ox0_cm, int32_t oy0_cm,
                           int32_t ocell_cm, int32_t onx, int32_t ony, float* out,
                           int8_t* how_out, void* cuda_stream) {
    bg::NvtxRange nvtx("bg_resample_grid");
    bg_status rc = check_source(src, x0_cm, y0_cm, cell_cm, nx, ny, method);
    if (rc != BG_OK) return rc;
    BG_REQUIRE(out, "out is NULL");
    BG_REQUIRE(ocell_cm > 0 && ocell_cm % 2 == 0, "output cell_cm must be even and > 0");
    BG_REQUIRE(onx > 0 && ony > 0, "output nx, ny must be > 0");
    BG_REQUIRE(grid_in_range(ox0_cm, oy0_cm, ocell_cm, onx, ony),
               "output nodes must lie in (-2^30, 2^30) cm");
    return launch_resample_grid(src, GridView{x0_cm, y0_cm, cell_cm, nx, ny}, method,
                                GridView{ox0_cm, oy0_cm, ocell_cm, onx, ony}, out, how_out,
                                (cudaStream_t)cuda_stream);
}

}  // extern "C"
