// Device spatial hash over the valid soundings: a counting sort into uniform
// square cells, plus the two lookup tables the neighbour search reads.
//
//   K0 validate_pack : drop NaN depths (the paper's "valid" neighbours),
//                      pack upload-order records, reduce the bounding box
//   K1 cell_hist     : per-cell counts (global atomics; cells are many)
//   K2 scan          : exclusive scan of the counts -> cell_start
//   K3 scatter       : cell-sorted records {x, y, z bits, upload index}
//   K4 sat           : summed-area table of the counts (2-D prefix sums), so a
//                      rectangle of cells is counted with four loads
//
// All four passes stream through HBM; none has a data-dependent loop. An input
// of at most 65,536 soundings over at most 12,000 cells (a serving tile) takes
// them in one 1024-thread block instead (k_hash_small), with its counts in
// shared memory: one launch instead of eight.
#include <algorithm>
#include <climits>
#include <cmath>

#include "bg_internal.h"

namespace bg {
namespace {

constexpr int kThreads = 256;
constexpr int kScanItems = 16;                      // per thread
constexpr int kScanTile = kThreads * kScanItems;    // per block
constexpr int kSatRows = 32;                        // rows per SAT chunk (at least)
constexpr int32_t kCoordLimit = 1 << 30;

__global__ void k_bbox_init(int* acc) {
    if (threadIdx.x == 0) {
        acc[0] = INT_MAX;
        acc[1] = INT_MAX;
        acc[2] = INT_MIN;
        acc[3] = INT_MIN;
        acc[4] = 0;
        acc[5] = 0;
    }
}

__global__ void __launch_bounds__(kThreads) k_validate_pack(
    const int32_t* __restrict__ x, const int32_t* __restrict__ y, const float* __restrict__ z,
    int64_t n, int4* __restrict__ orig, int* __restrict__ acc) {
    int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN, cnt = 0, bad = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int xi = x[i], yi = y[i];
        const float zi = z[i];
        const int valid = isnan(zi) ? 0 : 1;
        orig[i] = make_int4(xi, yi, __float_as_int(zi), valid);
        if (valid) {
            mnx = min(mnx, xi);
            mny = min(mny, yi);
            mxx = max(mxx, xi);
            mxy = max(mxy, yi);
            ++cnt;
            bad += (xi <= -kCoordLimit || xi >= kCoordLimit || yi <= -kCoordLimit || yi >= kCoordLimit);
        }
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        mnx = min(mnx, __shfl_xor_sync(0xffffffffu, mnx, o));
        mny = min(mny, __shfl_xor_sync(0xffffffffu, mny, o));
        mxx = max(mxx, __shfl_xor_sync(0xffffffffu, mxx, o));
        mxy = max(mxy, __shfl_xor_sync(0xffffffffu, mxy, o));
        cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        bad += __shfl_xor_sync(0xffffffffu, bad, o);
    }
    __shared__ int sm[kThreads / 32][6];
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    if (l == 0) {
        sm[w][0] = mnx; sm[w][1] = mny; sm[w][2] = mxx; sm[w][3] = mxy; sm[w][4] = cnt; sm[w][5] = bad;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int i = 1; i < kThreads / 32; ++i) {
            mnx = min(mnx, sm[i][0]);
            mny = min(mny, sm[i][1]);
            mxx = max(mxx, sm[i][2]);
            mxy = max(mxy, sm[i][3]);
            cnt += sm[i][4];
            bad += sm[i][5];
        }
        if (cnt) {
            atomicMin(&acc[0], mnx);
            atomicMin(&acc[1], mny);
            atomicMax(&acc[2], mxx);
            atomicMax(&acc[3], mxy);
            atomicAdd(&acc[4], cnt);
            atomicAdd(&acc[5], bad);
        }
    }
}

struct CellGeom {
    int32_t hx0, hy0, cs, ncx, ncy;
};

__device__ __forceinline__ int cell_index(const CellGeom& g, int x, int y) {
    // x >= hx0 and y >= hy0 for every valid sounding (the origin is the bbox min)
    const int cx = (x - g.hx0) / g.cs;
    const int cy = (y - g.hy0) / g.cs;
    return cy * g.ncx + cx;
}

__global__ void __launch_bounds__(kThreads) k_cell_hist(const int4* __restrict__ orig, int64_t n,
                                                        CellGeom g, int* __restrict__ count) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int4 r = orig[i];
        if (r.w) atomicAdd(&count[cell_index(g, r.x, r.y)], 1);
    }
}

__global__ void __launch_bounds__(kThreads) k_scatter(const int4* __restrict__ orig, int64_t n,
                                                      CellGeom g, int* __restrict__ cursor,
                                                      int4* __restrict__ rec) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int4 r = orig[i];
        if (r.w) {
            const int pos = atomicAdd(&cursor[cell_index(g, r.x, r.y)], 1);
            rec[pos] = make_int4(r.x, r.y, r.z, (int)i);
        }
    }
}

// ------------------------------------------------------------ exclusive scan

__device__ __forceinline__ int warp_incl_scan(int v) {
    const int l = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int t = __shfl_up_sync(0xffffffffu, v, o);
        if (l >= o) v += t;
    }
    return v;
}

// Exclusive scan of the kThreads values of a block; returns this thread's prefix.
__device__ __forceinline__ int block_excl_scan(int v, int* sm /*kThreads/32 + 1*/) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int inc = warp_incl_scan(v);
    if (l == 31) sm[w] = inc;
    __syncthreads();
    if (w == 0) {
        int s = l < kThreads / 32 ? sm[l] : 0;
        const int si = warp_incl_scan(s);
        if (l < kThreads / 32) sm[l] = si - s;
        if (l == kThreads / 32 - 1) sm[kThreads / 32] = si;
    }
    __syncthreads();
    return sm[w] + inc - v;
}

__global__ void __launch_bounds__(kThreads) k_scan_reduce(const int* __restrict__ in, int64_t n,
                                                          int* __restrict__ bsum) {
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int64_t j = base + (int64_t)i * kThreads + threadIdx.x;
        if (j < n) s += in[j];
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    __shared__ int sm[kThreads / 32];
    if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
        for (int i = 0; i < kThreads / 32; ++i) t += sm[i];
        bsum[blockIdx.x] = t;
    }
}

// One block: exclusive scan of the block sums in place; total -> *total.
__global__ void __launch_bounds__(kThreads) k_scan_blocksums(int* __restrict__ bsum, int nb,
                                                             int* __restrict__ total) {
    __shared__ int sm[kThreads / 32 + 1];
    int carry = 0;
    for (int base = 0; base < nb; base += kThreads) {
        const int j = base + threadIdx.x;
        const int v = j < nb ? bsum[j] : 0;
        const int ex = block_excl_scan(v, sm);
        if (j < nb) bsum[j] = carry + ex;
        carry += sm[kThreads / 32];
        __syncthreads();
    }
    if (threadIdx.x == 0) *total = carry;
}

// out[j] = boff[block] + exclusive prefix within the tile; in may alias out2.
__global__ void __launch_bounds__(kThreads) k_scan_apply(const int* in, int64_t n,
                                                         const int* __restrict__ boff,
                                                         int* __restrict__ out, int* out2) {
    __shared__ int tile[kScanTile];
    __shared__ int sm[kThreads / 32 + 1];
    const int64_t base = (int64_t)blockIdx.x * kScanTile;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int t = i * kThreads + threadIdx.x;
        const int64_t j = base + t;
        tile[t] = j < n ? in[j] : 0;
    }
    __syncthreads();
    int v[kScanItems];
    int s = 0;
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        v[i] = tile[threadIdx.x * kScanItems + i];
        s += v[i];
    }
    int ex = block_excl_scan(s, sm) + boff[blockIdx.x];
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        tile[threadIdx.x * kScanItems + i] = ex;
        ex += v[i];
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < kScanItems; ++i) {
        const int t = i * kThreads + threadIdx.x;
        const int64_t j = base + t;
        if (j < n) {
            out[j] = tile[t];
            if (out2) out2[j] = tile[t];
        }
    }
}

// ----------------------------------------------------------- summed-area table
// sat[(y)*(ncx+1) + x] = number of soundings in cells [0, x) x [0, y).
// The row prefix of row r at column x is cell_start[r*ncx + x] - cell_start[r*ncx].

__global__ void k_sat_chunk(const int* __restrict__ cs, int ncx, int ncy, int rows,
                            int* __restrict__ csum) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.y;
    if (x > ncx) return;
    const int y0 = ch * rows, y1 = min(ncy, y0 + rows);
    int s = 0;
    for (int y = y0; y < y1; ++y) s += cs[(int64_t)y * ncx + x] - cs[(int64_t)y * ncx];
    csum[(int64_t)ch * (ncx + 1) + x] = s;
}

__global__ void k_sat_chunkscan(int* __restrict__ csum, int ncx, int nch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x > ncx) return;
    int run = 0;
    for (int ch = 0; ch < nch; ++ch) {
        const int t = csum[(int64_t)ch * (ncx + 1) + x];
        csum[(int64_t)ch * (ncx + 1) + x] = run;
        run += t;
    }
}

__global__ void k_sat_apply(const int* __restrict__ cs, const int* __restrict__ csum, int ncx,
                            int ncy, int rows, int* __restrict__ sat) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int ch = blockIdx.y;
    if (x > ncx) return;
    const int64_t W = ncx + 1;
    const int y0 = ch * rows, y1 = min(ncy, y0 + rows);
    int run = csum[(int64_t)ch * W + x];
    if (ch == 0) sat[x] = 0;
    for (int y = y0; y < y1; ++y) {
        run += cs[(int64_t)y * ncx + x] - cs[(int64_t)y * ncx];
        sat[(int64_t)(y + 1) * W + x] = run;
    }
}

// ------------------------------------------------------- small inputs, one block
// A tile of a few tens of thousands of soundings spends its build on eight
// launches of tiny kernels. One 1024-thread block does the same passes with
// the counts in shared memory: (pack,) count, exclusive scan, summed-area
// table, scatter. cell_start and the table are those of the multi-kernel
// passes; the order of records within a cell comes from shared-memory
// atomics instead of global ones (every search result is keyed by (d2,
// index), so no result depends on it).
constexpr int kSmallThreads = 1024;
constexpr int64_t kSmallN = 1 << 16;
constexpr int64_t kSmallCells = 12000;  // counts + scan sums within 48 KB

// Exclusive scan over the 1024 threads of a block; ws holds 33 ints, ws[32]
// the total on return.
__device__ __forceinline__ int block_excl_scan_1024(int v, int* ws) {
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    const int inc = warp_incl_scan(v);
    if (l == 31) ws[w] = inc;
    __syncthreads();
    if (w == 0) {
        const int s = ws[l];
        const int si = warp_incl_scan(s);
        ws[l] = si - s;
        if (l == 31) ws[32] = si;
    }
    __syncthreads();
    return ws[w] + inc - v;
}

// pack: also write the upload-order records (when no earlier pass did).
// Dynamic shared memory: (ncx * ncy + 34) ints.
__global__ void __launch_bounds__(kSmallThreads) k_hash_small(
    const int32_t* __restrict__ x, const int32_t* __restrict__ y, const float* __restrict__ z,
    int n, int pack, int4* __restrict__ orig, CellGeom g, int* __restrict__ cell_start,
    int4* __restrict__ rec, int* __restrict__ sat) {
    extern __shared__ int cnt[];  // ncells counts, then starts, then cursors; + total + 33
    const int ncells = g.ncx * g.ncy;
    int* ws = cnt + ncells + 1;
    for (int c = threadIdx.x; c < ncells; c += blockDim.x) cnt[c] = 0;
    __syncthreads();
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const int xi = x[i], yi = y[i];
        const float zi = z[i];
        const int valid = isnan(zi) ? 0 : 1;
        if (pack) orig[i] = make_int4(xi, yi, __float_as_int(zi), valid);
        if (valid) atomicAdd(&cnt[cell_index(g, xi, yi)], 1);
    }
    __syncthreads();
    // exclusive scan, thread t over the cells [t * per, (t + 1) * per)
    const int per = (ncells + kSmallThreads - 1) / kSmallThreads;
    const int c0 = min(ncells, (int)threadIdx.x * per), c1 = min(ncells, c0 + per);
    int s = 0;
    for (int c = c0; c < c1; ++c) s += cnt[c];
    int run = block_excl_scan_1024(s, ws);
    for (int c = c0; c < c1; ++c) {
        const int v = cnt[c];
        cnt[c] = run;
        cell_start[c] = run;
        run += v;
    }
    if (threadIdx.x == 0) {
        cnt[ncells] = ws[32];
        cell_start[ncells] = ws[32];
    }
    __syncthreads();
    // summed-area table: column xx walks the rows; the row prefix of row yy
    // at column xx is start[yy * ncx + xx] - start[yy * ncx]
    const int64_t W = g.ncx + 1;
    for (int xx = threadIdx.x; xx < W; xx += blockDim.x) {
        int col = 0;
        sat[xx] = 0;
        for (int yy = 0; yy < g.ncy; ++yy) {
            col += cnt[yy * g.ncx + xx] - cnt[yy * g.ncx];
            sat[(int64_t)(yy + 1) * W + xx] = col;
        }
    }
    __syncthreads();  // the starts become the scatter's cursors
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float zi = z[i];
        if (!isnan(zi)) {
            const int xi = x[i], yi = y[i];
            const int pos = atomicAdd(&cnt[cell_index(g, xi, yi)], 1);
            rec[pos] = make_int4(xi, yi, __float_as_int(zi), i);
        }
    }
}

int grid_for(int64_t n, int per_block, int cap) {
    int64_t b = (n + per_block - 1) / per_block;
    if (b < 1) b = 1;
    if (b > cap) b = cap;
    return (int)b;
}

}  // namespace

namespace {
// Stream-ordered scratch released on every exit path.
struct Scratch {
    bg_ctx_s* ctx;
    cudaStream_t st;
    void* p = nullptr;
    size_t bytes = 0;
    Scratch(bg_ctx_s* c, cudaStream_t s) : ctx(c), st(s) {}
    bg_status alloc(size_t b) {
        bytes = b;
        return dalloc(ctx, &p, b, st);
    }
    ~Scratch() {
        if (p) dfree(ctx, p, bytes, st);
    }
};
}  // namespace

namespace {
// The cell side for a bounding box a = (x0, y0, x1, y1) holding nvalid soundings:
// the caller's hint, else about four soundings per cell at the mean density of
// the box (measured on the swath: 2 or 8 per cell make the k-NN 3-6% slower),
// widened until the tables fit.
int64_t pick_cell_side(const int32_t* a, int64_t nvalid, int32_t cell_hint) {
    const int64_t W = (int64_t)a[2] - a[0] + 1, H = (int64_t)a[3] - a[1] + 1;
    int64_t cs = cell_hint;
    if (cs <= 0) {
        const double rho = (double)nvalid / ((double)W * (double)H);
        cs = (int64_t)std::ceil(std::sqrt(4.0 / rho));
    }
    if (cs < 1) cs = 1;
    if (cs > kCoordLimit) cs = kCoordLimit;
    const int64_t max_cells = std::min<int64_t>((int64_t)1 << 28, 16 * nvalid + 4096);
    for (;;) {
        const int64_t ncx = (W + cs - 1) / cs, ncy = (H + cs - 1) / cs;
        if (ncx * ncy <= max_cells && (ncx + 1) * (ncy + 1) < ((int64_t)1 << 31)) break;
        cs = cs + cs / 4 + 1;
    }
    return cs;
}

int64_t cells_of(const int32_t* a, int64_t cs) {
    const int64_t W = (int64_t)a[2] - a[0] + 1, H = (int64_t)a[3] - a[1] + 1;
    return ((W + cs - 1) / cs) * ((H + cs - 1) / cs);
}
}  // namespace

bg_status build_soundings(bg_ctx_s* ctx, const int32_t* x, const int32_t* y, const float* z,
                          int64_t n, int on_device, int32_t cell_hint, cudaStream_t st,
                          bg_soundings_s* s, const HostBBox* known) {
    bg_status rc = BG_OK;
    const int32_t *dx = x, *dy = y;
    const float* dz = z;
    Scratch staging(ctx, st), scratch(ctx, st), accbuf(ctx, st);

    s->info = bg_soundings_info{};
    s->info.n_total = n;
    s->h = HashView{};
    int bits = 1;
    while (bits < 62 && (int64_t(1) << bits) < n) ++bits;
    s->h.idx_bits = bits;

    if (n > 0 && !on_device) {
        if ((rc = staging.alloc((size_t)n * 12)) != BG_OK) return rc;
        int32_t* sx = (int32_t*)staging.p;
        int32_t* sy = sx + n;
        float* sz = (float*)(sy + n);
        BG_CUDA(cudaMemcpyAsync(sx, x, n * 4, cudaMemcpyHostToDevice, st));
        BG_CUDA(cudaMemcpyAsync(sy, y, n * 4, cudaMemcpyHostToDevice, st));
        BG_CUDA(cudaMemcpyAsync(sz, z, n * 4, cudaMemcpyHostToDevice, st));
        dx = sx;
        dy = sy;
        dz = sz;
    }
    if (n > 0) {
        if ((rc = dalloc(ctx, &s->d_orig, (size_t)n * 16, st)) != BG_OK) return rc;
        s->bytes += (size_t)n * 16;
        s->h.orig = (const int4*)s->d_orig;
    }
    // a small input whose bounding box the caller scanned on the host is packed
    // by the one-block build itself
    bool pack_small = false;
    if (known && n > 0 && n <= kSmallN && known->n_valid > 0 && known->out_of_range == 0) {
        const int32_t kb[4] = {known->x0, known->y0, known->x1, known->y1};
        pack_small = cells_of(kb, pick_cell_side(kb, known->n_valid, cell_hint)) <= kSmallCells;
    }
    int* acc = nullptr;
    if (!pack_small) {
        if ((rc = accbuf.alloc(8 * sizeof(int))) != BG_OK) return rc;
        acc = (int*)accbuf.p;  // min x, min y, max x, max y, valid count, out-of-range count
        k_bbox_init<<<1, 32, 0, st>>>(acc);
        note_launches(1);
        if (n > 0) {
            k_validate_pack<<<grid_for(n, kThreads * 4, 152 * 16), kThreads, 0, st>>>(
                dx, dy, dz, n, (int4*)s->d_orig, acc);
            note_launches(1);
        }
        BG_CUDA(cudaGetLastError());
    }
    int32_t a[6];
    if (known) {
        // the caller scanned the (host) input already: no device round trip
        a[0] = known->x0;
        a[1] = known->y0;
        a[2] = known->x1;
        a[3] = known->y1;
        a[4] = (int32_t)known->n_valid;
        a[5] = known->out_of_range;
    } else {
        std::lock_guard<std::mutex> lk(ctx->pin_mu);
        BG_CUDA(cudaMemcpyAsync(ctx->h_pinned, acc, 6 * sizeof(int), cudaMemcpyDeviceToHost, st));
        BG_CUDA(cudaStreamSynchronize(st));
        for (int i = 0; i < 6; ++i) a[i] = ctx->h_pinned[i];
    }
    const int64_t nvalid = a[4];
    s->info.n_valid = nvalid;
    s->info.device_bytes = (int64_t)s->bytes;
    if (a[5] != 0) {
        set_error("a valid sounding lies outside (-2^30, 2^30) cm");
        return BG_ERR_INVALID_ARG;
    }
    if (nvalid == 0) return BG_OK;  // every interpolation over this handle yields NaN

    const int64_t W = (int64_t)a[2] - a[0] + 1, H = (int64_t)a[3] - a[1] + 1;
    const int64_t cs = pick_cell_side(a, nvalid, cell_hint);
    const int32_t ncx = (int32_t)((W + cs - 1) / cs), ncy = (int32_t)((H + cs - 1) / cs);
    const int64_t ncells = (int64_t)ncx * ncy;
    s->info.bbox_x0_cm = a[0];
    s->info.bbox_y0_cm = a[1];
    s->info.bbox_x1_cm = a[2];
    s->info.bbox_y1_cm = a[3];
    s->info.cell_cm = (int32_t)cs;
    s->info.ncx = ncx;
    s->info.ncy = ncy;

    const size_t cs_bytes = (size_t)(ncells + 1) * 4;
    const size_t sat_bytes = (size_t)(ncx + 1) * (ncy + 1) * 4;
    const size_t rec_bytes = (size_t)nvalid * 16;
    if ((rc = dalloc(ctx, &s->d_cell_start, cs_bytes, st)) != BG_OK) return rc;
    s->bytes += cs_bytes;
    if ((rc = dalloc(ctx, &s->d_sat, sat_bytes, st)) != BG_OK) return rc;
    s->bytes += sat_bytes;
    if ((rc = dalloc(ctx, &s->d_rec, rec_bytes, st)) != BG_OK) return rc;
    s->bytes += rec_bytes;

    const CellGeom g{a[0], a[1], (int32_t)cs, ncx, ncy};
    int* cell_start = (int*)s->d_cell_start;
    if (n <= kSmallN && ncells <= kSmallCells) {
        k_hash_small<<<1, kSmallThreads, (size_t)(ncells + 34) * sizeof(int), st>>>(
            dx, dy, dz, (int)n, pack_small ? 1 : 0, (int4*)s->d_orig, g, cell_start,
            (int4*)s->d_rec, (int*)s->d_sat);
        note_launches(1);
        BG_CUDA(cudaGetLastError());
    } else {
        const int nb = (int)((ncells + kScanTile - 1) / kScanTile);
        // chunks of rows for the column prefix of the SAT (grid.y stays <= 65535)
        const int sat_rows = std::max(kSatRows, (ncy + 65534) / 65535);
        const int nch = (ncy + sat_rows - 1) / sat_rows;
        const size_t count_bytes = (size_t)ncells * 4;
        const size_t bsum_bytes = (size_t)(nb + 1) * 4;
        const size_t csum_bytes = (size_t)nch * (ncx + 1) * 4;
        if ((rc = scratch.alloc(count_bytes + bsum_bytes + csum_bytes + 64)) != BG_OK) return rc;
        int* count = (int*)scratch.p;
        int* bsum = count + ncells;
        int* csum = bsum + nb + 1;

        BG_CUDA(cudaMemsetAsync(count, 0, count_bytes, st));
        k_cell_hist<<<grid_for(n, kThreads * 4, 152 * 16), kThreads, 0, st>>>(
            (const int4*)s->d_orig, n, g, count);
        k_scan_reduce<<<nb, kThreads, 0, st>>>(count, ncells, bsum);
        k_scan_blocksums<<<1, kThreads, 0, st>>>(bsum, nb, cell_start + ncells);
        k_scan_apply<<<nb, kThreads, 0, st>>>(count, ncells, bsum, cell_start, count);
        k_scatter<<<grid_for(n, kThreads * 4, 152 * 16), kThreads, 0, st>>>(
            (const int4*)s->d_orig, n, g, count, (int4*)s->d_rec);
        const dim3 sg((ncx + 1 + 255) / 256, nch);
        k_sat_chunk<<<sg, 256, 0, st>>>(cell_start, ncx, ncy, sat_rows, csum);
        k_sat_chunkscan<<<(ncx + 1 + 255) / 256, 256, 0, st>>>(csum, ncx, nch);
        k_sat_apply<<<sg, 256, 0, st>>>(cell_start, csum, ncx, ncy, sat_rows, (int*)s->d_sat);
        note_launches(8);
        BG_CUDA(cudaGetLastError());
    }

    s->h.rec = (const int4*)s->d_rec;
    s->h.cell_start = cell_start;
    s->h.sat = (const int32_t*)s->d_sat;
    s->h.hx0 = a[0];
    s->h.hy0 = a[1];
    s->h.cs = (int32_t)cs;
    s->h.inv_cs = 1.0f / (float)cs;
    s->h.ncx = ncx;
    s->h.ncy = ncy;
    s->h.n_valid = (int32_t)nvalid;
    s->info.device_bytes = (int64_t)s->bytes;
    return BG_OK;
}

int32_t start_halfwidth(const bg_soundings_s* s, int k) {
    const double ncells = (double)s->info.ncx * (double)s->info.ncy;
    if (s->info.n_valid <= 0 || ncells <= 0) return 0;
    const double per_cell = (double)s->info.n_valid / ncells;
    // smallest R with (2R+1)^2 cells holding k soundings at the mean density
    const double side = std::sqrt((double)k / per_cell);
    int32_t r = (int32_t)std::ceil((side - 1.0) * 0.5);
    if (r < 0) r = 0;
    const int32_t rmax = std::max(s->info.ncx, s->info.ncy);
    return r > rmax ? rmax : r;
}

bg_status build_hash_in_arena(const int32_t* x, const int32_t* y, const float* z, int64_t n,
                              const HashArena& ar, cudaStream_t st, bg_soundings_s* s) {
    s->info = bg_soundings_info{};
    s->info.n_total = n;
    s->h = HashView{};
    int bits = 1;
    while (bits < 62 && (int64_t(1) << bits) < n) ++bits;
    s->h.idx_bits = bits;
    if (n > ar.n_max) {
        set_error("too many soundings for the arena");
        return BG_ERR_INVALID_ARG;
    }
    s->h.orig = ar.orig;
    k_bbox_init<<<1, 32, 0, st>>>(ar.acc);
    note_launches(1);
    if (n > 0) {
        k_validate_pack<<<grid_for(n, kThreads * 4, 152 * 16), kThreads, 0, st>>>(x, y, z, n,
                                                                                ar.orig, ar.acc);
        note_launches(1);
    }
    BG_CUDA(cudaGetLastError());
    int32_t a[8];
    BG_CUDA(cudaMemcpyAsync(a, ar.acc, 6 * sizeof(int), cudaMemcpyDeviceToHost, st));
    BG_CUDA(cudaStreamSynchronize(st));
    const int64_t nvalid = a[4];
    s->info.n_valid = nvalid;
    if (a[5] != 0) {
        set_error("a valid sounding lies outside (-2^30, 2^30) cm");
        return BG_ERR_INVALID_ARG;
    }
    if (nvalid == 0) return BG_OK;

    const int64_t W = (int64_t)a[2] - a[0] + 1, H = (int64_t)a[3] - a[1] + 1;
    const double rho = (double)nvalid / ((double)W * (double)H);
    int64_t cs = (int64_t)std::ceil(std::sqrt(4.0 / rho));
    if (cs < 1) cs = 1;
    if (cs > kCoordLimit) cs = kCoordLimit;
    int64_t ncx = 0, ncy = 0, nb = 0, nch = 0, sat_rows = kSatRows;
    for (;;) {
        ncx = (W + cs - 1) / cs;
        ncy = (H + cs - 1) / cs;
        sat_rows = std::max<int64_t>(kSatRows, (ncy + 65534) / 65535);
        nch = (ncy + sat_rows - 1) / sat_rows;
        nb = (ncx * ncy + kScanTile - 1) / kScanTile;
        if (ncx * ncy <= ar.cells_max && (ncx + 1) * (ncy + 1) <= ar.sat_max &&
            nb + 1 <= ar.bsum_max && nch * (ncx + 1) <= ar.csum_max)
            break;
        cs = cs + cs / 4 + 1;
    }
    const int64_t ncells = ncx * ncy;
    s->info.bbox_x0_cm = a[0];
    s->info.bbox_y0_cm = a[1];
    s->info.bbox_x1_cm = a[2];
    s->info.bbox_y1_cm = a[3];
    s->info.cell_cm = (int32_t)cs;
    s->info.ncx = (int32_t)ncx;
    s->info.ncy = (int32_t)ncy;

    const CellGeom g{a[0], a[1], (int32_t)cs, (int32_t)ncx, (int32_t)ncy};
    BG_CUDA(cudaMemsetAsync(ar.count, 0, (size_t)ncells * 4, st));
    k_cell_hist<<<grid_for(n, kThreads * 4, 152 * 16), kThreads, 0, st>>>(ar.orig, n, g, ar.count);
    k_scan_reduce<<<(unsigned)nb, kThreads, 0, st>>>(ar.count, ncells, ar.bsum);
    k_scan_blocksums<<<1, kThreads, 0, st>>>(ar.bsum, (int)nb, ar.cell_start + ncells);
    k_scan_apply<<<(unsigned)nb, kThreads, 0, st>>>(ar.count, ncells, ar.bsum, ar.cell_start,
                                                    ar.count);
    k_scatter<<<grid_for(n, kThreads * 4, 152 * 16), kThreads, 0, st>>>(ar.orig, n, g, ar.count,
                                                                        ar.rec);
    const dim3 sg((unsigned)((ncx + 1 + 255) / 256), (unsigned)nch);
    k_sat_chunk<<<sg, 256, 0, st>>>(ar.cell_start, (int)ncx, (int)ncy, (int)sat_rows, ar.csum);
    k_sat_chunkscan<<<(unsigned)((ncx + 1 + 255) / 256), 256, 0, st>>>(ar.csum, (int)ncx, (int)nch);
    k_sat_apply<<<sg, 256, 0, st>>>(ar.cell_start, ar.csum, (int)ncx, (int)ncy, (int)sat_rows,
                                    ar.sat);
    note_launches(8);
    BG_CUDA(cudaGetLastError());

    s->h.rec = ar.rec;
    s->h.cell_start = ar.cell_start;
    s->h.sat = ar.sat;
    s->h.hx0 = a[0];
    s->h.hy0 = a[1];
    s->h.cs = (int32_t)cs;
    s->h.inv_cs = 1.0f / (float)cs;
    s->h.ncx = (int32_t)ncx;
    s->h.ncy = (int32_t)ncy;
    s->h.n_valid = (int32_t)nvalid;
    return BG_OK;
}

int scan_blocks(int64_t n) { return (int)((n + kScanTile - 1) / kScanTile); }

void launch_excl_scan(const int* in, int64_t n, int* out, int* out2, int* bsum, cudaStream_t st) {
    const int nb = scan_blocks(n);
    k_scan_reduce<<<nb, kThreads, 0, st>>>(in, n, bsum);
    k_scan_blocksums<<<1, kThreads, 0, st>>>(bsum, nb, out + n);
    k_scan_apply<<<nb, kThreads, 0, st>>>(in, n, bsum, out, out2);
    note_launches(3);
}

}  // namespace bg
