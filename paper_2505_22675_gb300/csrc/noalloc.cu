// bg_interp_idw_noalloc: IDW gridding for callers that cannot allocate device
// memory: a process that reserves all device memory up front, a runtime whose
// allocator policy forbids cudaMalloc on its worker threads, or code in a
// driver-owned thread that must not allocate. The work space that
// bg_soundings_upload and bg_interp_idw would allocate lives here in one
// file-scope __device__ array instead.
//
// The array is a fixed 16 MiB in every device that loads this library, held
// until the process exits. Every call shares it, and it keeps the last call's
// contents; the parts that must start at zero (cell counts, the bbox
// accumulator, the wide-pass flag) are cleared by each call. Two calls whose
// GPU work overlaps (on two streams, or from two host threads) race on the
// array: run them one after another.
//
// The call launches kernels and synchronizes its stream once, so it must not
// be made from a CUDA stream callback (cudaLaunchHostFunc; CUDA calls are not
// allowed there) or while the stream is being captured.
#include "bg_internal.h"

namespace {

constexpr int64_t kMaxSoundings = int64_t(1) << 18;   // 262,144
constexpr int64_t kMaxCells = int64_t(1) << 18;       // hash cells
constexpr size_t kScratchBytes = size_t(16) << 20;    // 16 MiB

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

size_t up256(size_t v) { return (v + 255) & ~size_t(255); }

// Device address of g_scratch on the current device. In host code the name
// g_scratch is only a host-side stand-in, so the address is looked up on
// every call: it is cheap, allocates nothing, and stays right after a
// cudaDeviceReset or a context re-creation.
bg_status scratch_address(unsigned char** out) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
    if (e != cudaSuccess) return bg::cuda_fail(e, "cudaGetSymbolAddress(g_scratch)");
    *out = static_cast<unsigned char*>(p);
    return BG_OK;
}

}  // namespace

extern "C" bg_status bg_interp_idw_noalloc(const int32_t* x_cm, const int32_t* y_cm,
                                           const float* z_m, int64_t n, int32_t x0_cm,
                                           int32_t y0_cm, int32_t cell_cm, int32_t nx, int32_t ny,
                                           int k, float power, float* depth_out,
                                           int32_t* nbr_out, void* cuda_stream) {
    using namespace bg;
    if (n < 0 || n > kMaxSoundings) {
        set_error("bg_interp_idw_noalloc takes at most 262144 soundings");
        return BG_ERR_INVALID_ARG;
    }
    if (n > 0 && !(x_cm && y_cm && z_m)) {
        set_error("NULL input pointer");
        return BG_ERR_INVALID_ARG;
    }
    if (!depth_out) {
        set_error("depth_out is NULL");
        return BG_ERR_INVALID_ARG;
    }
    if (k < 1 || k > 32) {
        set_error("k must be in [1, 32]");
        return BG_ERR_INVALID_ARG;
    }
    if (!(power > 0.0f) || !(power < 1e30f)) {
        set_error("power must be finite and > 0");
        return BG_ERR_INVALID_ARG;
    }
    if (cell_cm <= 0 || cell_cm % 2 != 0 || nx <= 0 || ny <= 0 ||
        (int64_t)nx * ny > (int64_t(1) << 36)) {
        set_error("bad grid: cell_cm must be even and > 0, nx and ny > 0, nx*ny <= 2^36");
        return BG_ERR_INVALID_ARG;
    }
    {
        const int64_t lim = int64_t(1) << 30;
        const int64_t xa = (int64_t)x0_cm + cell_cm / 2;
        const int64_t xb = (int64_t)x0_cm + (int64_t)(nx - 1) * cell_cm + cell_cm / 2;
        const int64_t ya = (int64_t)y0_cm + cell_cm / 2;
        const int64_t yb = (int64_t)y0_cm + (int64_t)(ny - 1) * cell_cm + cell_cm / 2;
        if (!(xa > -lim && xb < lim && ya > -lim && yb < lim)) {
            set_error("grid node coordinates must lie in (-2^30, 2^30) cm");
            return BG_ERR_INVALID_ARG;
        }
    }
    unsigned char* base = nullptr;
    const bg_status rc = scratch_address(&base);
    if (rc != BG_OK) return rc;

    // carve the array: records, cell tables, scan and SAT partial sums, flags
    HashArena ar{};
    size_t off = 0;
    auto take = [&](size_t bytes) {
        unsigned char* p = base + off;
        off += up256(bytes);
        return p;
    };
    ar.n_max = kMaxSoundings;
    ar.cells_max = kMaxCells;
    ar.sat_max = 3 * kMaxCells + 2;
    ar.bsum_max = kMaxCells / 4096 + 2;
    ar.csum_max = kMaxCells + 2;
    ar.orig = (int4*)take(size_t(ar.n_max) * 16);
    ar.rec = (int4*)take(size_t(ar.n_max) * 16);
    ar.cell_start = (int32_t*)take(size_t(ar.cells_max + 1) * 4);
    ar.count = (int32_t*)take(size_t(ar.cells_max) * 4);
    ar.sat = (int32_t*)take(size_t(ar.sat_max) * 4);
    ar.bsum = (int32_t*)take(size_t(ar.bsum_max) * 4);
    ar.csum = (int32_t*)take(size_t(ar.csum_max) * 4);
    ar.acc = (int32_t*)take(8 * 4);
    int* flag = (int*)take(4);
    if (off > kScratchBytes) {
        set_error("internal: scratch layout exceeds the static array");
        return BG_ERR_INTERNAL;
    }

    const cudaStream_t st = (cudaStream_t)cuda_stream;
    bg_soundings_s s{};
    bg_status r = build_hash_in_arena(x_cm, y_cm, z_m, n, ar, st, &s);
    if (r != BG_OK) return r;
    const GridView g{x0_cm, y0_cm, cell_cm, nx, ny};
    return launch_idw_with_flag(&s, g, k, power, depth_out, nbr_out, flag, st);
}
