// Batched gridding: many tiles of uneven size in a fixed sequence of launches.
//
// All tiles share one set of device buffers laid out at bg_batch_create:
// soundings and cells are concatenated tile after tile, every tile with a
// fixed capacity of cells. A run is one CUDA graph, captured on the first
// bg_batch_run and replayed after (no host synchronization inside):
//   1. validate + pack all soundings, per-tile bounding boxes (block
//      reductions per tile segment of each block's chunk);
//   2. per-tile hash geometry on the device (cell side for about `ppc`
//      soundings per cell, grown until the tile's cells fit its capacity);
//   3. one counting sort over the concatenated cells: histogram, one
//      exclusive scan, scatter (cell_start holds positions in the shared
//      record array, so each tile's hash is a window of it);
//   4. per-tile summed-area tables (one block per tile);
//   5. a persistent kernel drains (tile, 16 S x 8 node patch) items, a thread
//      gridding S consecutive nodes along x (S = 1, 2 or 4: the strip
//      length; from the second node on, the previous node's K-th distance
//      plus the step bounds the search): IDW tiles are gridded in place,
//      kriging tiles get their neighbour ids;
//   6. a persistent kernel per kriging system size drains (tile, nb x 16
//      warps' systems) items (okrige_solve_block), nb block batches per
//      claimed item;
//   7. a wide-key pass, which returns at once unless a node's bound needed
//      more than the packed key's bits.
// Items are claimed with a global atomic counter, so uneven tiles balance
// across the SMs. Results are bitwise those of the per-grid calls, whatever
// the cell target, strip length and solve item size (bg_batch_tune picks
// those three by timing runs).
#include <algorithm>
#include <cmath>
#include <new>
#include <vector>

#include "bathygrid.h"
#include "idw_dev.cuh"
#include "okrige_dev.cuh"

namespace bg {

// One tile of a batch as the kernels see it.
struct TileDesc {
    HashView h;          // geometry fields written on the device each run
    GridView g;
    const int32_t* x;    // inputs (device)
    const int32_t* y;
    const float* z;
    float* depth;        // outputs (device)
    float* var;
    int32_t* ids;        // kriging: nx*ny*k neighbour ids
    OkParams p;
    float power;
    int32_t method, k, K;  // K: kriging system size (4/8/16/32)
    int32_t gx;          // node patches along x
    int64_t soff, n;     // soundings in the concatenation
    int64_t coff, cap;   // cells
    int64_t satoff, satcap;
};

namespace {

constexpr int kChunk = 4096;      // soundings per block in the per-sounding kernels
constexpr int kBT = 256;          // threads of those kernels
constexpr int kItemThreads = 128;
constexpr int kKnnThreads = 64;  // k-NN blocks: a 16 KB heap, 13 blocks (26 warps) per SM
constexpr int kBatchSolveBlocks = 8;  // default block batches per claimed item (256 systems at K = 32)
constexpr int kStrips[3] = {1, 2, 4};  // k-NN strip lengths the batch offers
// The persistent solve runs 8-warp blocks, 2 per SM (128 registers, dynamic
// shared memory), like the per-grid kernels: two blocks in different phases
// of the long unrolled solve wait far less for instruction fetch than 3 or 4
// smaller ones (measured 291 ms per batch against 325 ms for 3 x 4 warps).
constexpr int kBatchSolveWarps = 8;
constexpr int kBatchSolveBlocksPerSM = 2;

__device__ __forceinline__ int upper_tile(const int64_t* off, int T, int64_t v) {
    // largest t with off[t] <= v  (off ascending, off[0] = 0)
    int lo = 0, hi = T;
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= v)
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

__global__ void k_batch_init(int* acc, int T) {
    for (int t = blockIdx.x * blockDim.x + threadIdx.x; t < T; t += gridDim.x * blockDim.x) {
        int* a = acc + 8 * t;
        a[0] = INT_MAX;
        a[1] = INT_MAX;
        a[2] = INT_MIN;
        a[3] = INT_MIN;
        a[4] = 0;
        a[5] = 0;
    }
}

__device__ __forceinline__ int block_reduce(int v, int op, int* sm) {
    // op 0: min, 1: max, 2: sum; every thread of the block calls it
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        const int u = __shfl_xor_sync(0xffffffffu, v, o);
        v = op == 0 ? min(v, u) : op == 1 ? max(v, u) : v + u;
    }
    const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
    __syncthreads();
    if (l == 0) sm[w] = v;
    __syncthreads();
    if (threadIdx.x == 0)
        for (int i = 1; i < (int)(blockDim.x >> 5); ++i)
            v = op == 0 ? min(v, sm[i]) : op == 1 ? max(v, sm[i]) : v + sm[i];
    return v;
}

// 1. validate + pack, per-tile bounding box
__global__ void __launch_bounds__(kBT) k_batch_validate(const TileDesc* __restrict__ td, int T,
                                                        const int64_t* __restrict__ soff,
                                                        int64_t total, int4* __restrict__ orig,
                                                        int* __restrict__ acc) {
    __shared__ int sm[kBT / 32];
    int64_t beg = (int64_t)blockIdx.x * kChunk;
    const int64_t end = min(total, beg + kChunk);
    int t = upper_tile(soff, T + 1, beg);
    while (beg < end && t < T) {
        const int64_t tend = min(end, __ldg(soff + t + 1));
        const int32_t* x = td[t].x;
        const int32_t* y = td[t].y;
        const float* z = td[t].z;
        const int64_t base = __ldg(soff + t);
        int mnx = INT_MAX, mny = INT_MAX, mxx = INT_MIN, mxy = INT_MIN, cnt = 0, bad = 0;
        for (int64_t i = beg + threadIdx.x; i < tend; i += blockDim.x) {
            const int64_t li = i - base;
            const int xi = x[li], yi = y[li];
            const float zi = z[li];
            const int valid = isnan(zi) ? 0 : 1;
            orig[i] = make_int4(xi, yi, __float_as_int(zi), valid);
            if (valid) {
                mnx = min(mnx, xi);
                mny = min(mny, yi);
                mxx = max(mxx, xi);
                mxy = max(mxy, yi);
                ++cnt;
                bad += (xi <= -(1 << 30) || xi >= (1 << 30) || yi <= -(1 << 30) || yi >= (1 << 30));
            }
        }
        mnx = block_reduce(mnx, 0, sm);
        mny = block_reduce(mny, 0, sm);
        mxx = block_reduce(mxx, 1, sm);
        mxy = block_reduce(mxy, 1, sm);
        cnt = block_reduce(cnt, 2, sm);
        bad = block_reduce(bad, 2, sm);
        if (threadIdx.x == 0 && cnt) {
            int* a = acc + 8 * t;
            atomicMin(a + 0, mnx);
            atomicMin(a + 1, mny);
            atomicMax(a + 2, mxx);
            atomicMax(a + 3, mxy);
            atomicAdd(a + 4, cnt);
            atomicAdd(a + 5, bad);
        }
        beg = tend;
        ++t;
    }
}

// 2. per-tile hash geometry (one thread per tile)
__global__ void k_batch_geom(TileDesc* td, int T, const int* __restrict__ acc, float ppc,
                             int* __restrict__ status) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= T) return;
    TileDesc& d = td[t];
    const int* a = acc + 8 * t;
    HashView& h = d.h;
    h.n_valid = a[4];
    if (a[5] != 0) {
        atomicOr(status, 1);  // a coordinate outside (-2^30, 2^30): the tile yields NaN
        h.n_valid = 0;
    }
    if (h.n_valid == 0) {
        h.ncx = h.ncy = 0;
        return;
    }
    const int64_t W = (int64_t)a[2] - a[0] + 1, H = (int64_t)a[3] - a[1] + 1;
    const double rho = (double)h.n_valid / ((double)W * (double)H);
    int64_t cs = (int64_t)ceil(sqrt((double)ppc / rho));
    if (cs < 1) cs = 1;
    for (;;) {
        const int64_t ncx = (W + cs - 1) / cs, ncy = (H + cs - 1) / cs;
        if (ncx * ncy <= d.cap && (ncx + 1) * (ncy + 1) <= d.satcap) break;
        cs = cs + cs / 4 + 1;
    }
    h.hx0 = a[0];
    h.hy0 = a[1];
    h.cs = (int32_t)cs;
    h.inv_cs = 1.0f / (float)cs;
    h.ncx = (int32_t)((W + cs - 1) / cs);
    h.ncy = (int32_t)((H + cs - 1) / cs);
    // first square half-width tried by the bound search, for this tile's k
    const int kq = d.method == 0 ? d.k : d.K;
    const double per_cell = (double)h.n_valid / ((double)h.ncx * h.ncy);
    int r = (int)ceil((sqrt((double)kq / per_cell) - 1.0) * 0.5);
    h.r0 = max(0, min(r, max(h.ncx, h.ncy)));
}

// 3a/3c. histogram and scatter over the concatenated soundings
template <bool kScatter>
__global__ void __launch_bounds__(kBT) k_batch_cells(const TileDesc* __restrict__ td, int T,
                                                     const int64_t* __restrict__ soff,
                                                     int64_t total, const int4* __restrict__ orig,
                                                     int* __restrict__ count,
                                                     int4* __restrict__ rec) {
    int64_t beg = (int64_t)blockIdx.x * kChunk;
    const int64_t end = min(total, beg + kChunk);
    int t = upper_tile(soff, T + 1, beg);
    while (beg < end && t < T) {
        const int64_t tend = min(end, __ldg(soff + t + 1));
        const HashView& h = td[t].h;
        const int hx0 = h.hx0, hy0 = h.hy0, cs = h.cs, ncx = h.ncx;
        const int64_t coff = td[t].coff, base = __ldg(soff + t);
        if (td[t].h.n_valid > 0) {
            for (int64_t i = beg + threadIdx.x; i < tend; i += blockDim.x) {
                const int4 r = orig[i];
                if (!r.w) continue;
                const int cell = ((r.y - hy0) / cs) * ncx + (r.x - hx0) / cs;
                if (kScatter) {
                    const int pos = atomicAdd(&count[coff + cell], 1);
                    rec[pos] = make_int4(r.x, r.y, r.z, (int)(i - base));
                } else {
                    atomicAdd(&count[coff + cell], 1);
                }
            }
        }
        beg = tend;
        ++t;
    }
}

// 4. per-tile summed-area table, one block per tile
__global__ void k_batch_sat(const TileDesc* __restrict__ td, const int* __restrict__ cell_start,
                            int* __restrict__ sat) {
    const TileDesc& d = td[blockIdx.x];
    const int ncx = d.h.ncx, ncy = d.h.ncy;
    if (d.h.n_valid == 0) return;
    const int* cs = cell_start + d.coff;
    int* s = sat + d.satoff;
    const int64_t W = ncx + 1;
    for (int x = threadIdx.x; x <= ncx; x += blockDim.x) {
        int run = 0;
        s[x] = 0;
        for (int y = 0; y < ncy; ++y) {
            run += cs[(int64_t)y * ncx + x] - cs[(int64_t)y * ncx];
            s[(int64_t)(y + 1) * W + x] = run;
        }
    }
}

// the tile's hash view with pointers into the shared buffers
__device__ __forceinline__ HashView tile_view(const TileDesc& d, const int4* orig, const int4* rec,
                                              const int* cell_start, const int* sat) {
    HashView h = d.h;
    h.orig = orig + d.soff;
    h.rec = rec;
    h.cell_start = cell_start + d.coff;
    h.sat = sat + d.satoff;
    return h;
}

// 5. persistent k-NN items: IDW in place, kriging ids. An item is a
// (16 kS) x 8 node patch of one tile; warp w covers its (8 kS) x 4 quarter,
// each thread a strip of kS nodes along x.
template <int kS>
__global__ void __launch_bounds__(kKnnThreads) k_batch_knn(
    const TileDesc* __restrict__ td, int T, const int64_t* __restrict__ item_off, int64_t items,
    unsigned long long* __restrict__ ctr, const int4* __restrict__ orig,
    const int4* __restrict__ rec, const int* __restrict__ cell_start, const int* __restrict__ sat,
    int* __restrict__ wide) {
    __shared__ uint64_t heap[32 * kKnnThreads];
    __shared__ long long s_item;
    __shared__ int s_tile;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint64_t* hp = heap + threadIdx.x;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = (long long)atomicAdd(ctr, 1ull);
            s_tile = s_item < items ? upper_tile(item_off, T + 1, s_item) : 0;
        }
        __syncthreads();
        const long long item = s_item;
        const int t = s_tile;
        __syncthreads();
        if (item >= items) break;
        const TileDesc& d = td[t];
        const HashView h = tile_view(d, orig, rec, cell_start, sat);
        const GridView g = d.g;
        const int gx = (g.nx + 16 * kS - 1) / (16 * kS);
        const int64_t patch = item - __ldg(item_off + t);
        const int px = (int)(patch % gx), py = (int)(patch / gx);
        const int k = d.k, kc = d.method == 0 ? k : d.K;
        const int bits = h.idx_bits;
        const uint64_t mask = (1ull << bits) - 1;
        // the node's neighbours, sorted ascending in hp[0 .. cnt)
        auto emit = [&](int i, int cnt, int j) {
            const int64_t node = (int64_t)j * g.nx + i;
            const int keff = min(cnt, k);
            if (d.method == 0) {
                d.depth[node] = idw_from(h, keff, d.power, [&](int q, uint64_t& dd, int& ii) {
                    const uint64_t key = hp[q * kKnnThreads];
                    dd = key >> bits;
                    ii = (int)(key & mask);
                });
            } else {
                emit_ids<kKnnThreads>(d.ids + node * k, hp, k, keff, mask);
            }
        };
        // the (16 kS) x 8 patch in two halves of (16 kS) x 4 (two warps each)
        for (int half = 0; half < 2; ++half) {
            const int w = warp + 2 * half;
            const int i0 = px * 16 * kS + (w & 1) * 8 * kS + (lane & 7) * kS;
            const int j = py * 8 + (w >> 1) * 4 + (lane >> 3);
            if (i0 >= g.nx || j >= g.ny) continue;
            if (h.n_valid == 0) {
                for (int i = i0; i < min(i0 + kS, g.nx); ++i) emit(i, 0, j);
                continue;
            }
            auto emit_j = [&](int i, int cnt) { emit(i, cnt, j); };
            knn_strip<kKnnThreads, decltype(emit_j), true, kS>(h, g, kc, i0, j, hp, wide, emit_j);
        }
    }
}

// 6. persistent kriging solves for the tiles of one system size K; the tile's
// descriptor is staged in shared memory so its fields are read where needed
// instead of being held in registers across the solve
template <int K>
__global__ void __launch_bounds__(kBatchSolveWarps * 32, kBatchSolveBlocksPerSM) k_batch_solve(
    const TileDesc* __restrict__ td, const int* __restrict__ tiles, int nt,
    const int64_t* __restrict__ off, int64_t items, unsigned long long* __restrict__ ctr,
    const int4* __restrict__ orig, const int4* __restrict__ rec, const int* __restrict__ cell_start,
    const int* __restrict__ sat, int nb) {
    extern __shared__ __align__(16) float smem[];
    __shared__ long long s_item;
    __shared__ int s_j;
    __shared__ HashView s_h;
    __shared__ GridView s_g;
    __shared__ OkParams s_p;
    __shared__ int s_k;
    __shared__ float* s_depth;
    __shared__ float* s_var;
    __shared__ const int32_t* s_ids;
    for (;;) {
        if (threadIdx.x == 0) {
            s_item = (long long)atomicAdd(ctr, 1ull);
            s_j = s_item < items ? upper_tile(off, nt + 1, s_item) : 0;
            if (s_item < items) {
                const TileDesc& d = td[__ldg(tiles + s_j)];
                s_h = tile_view(d, orig, rec, cell_start, sat);
                s_g = d.g;
                s_p = d.p;
                s_k = d.k;
                s_depth = d.depth;
                s_var = d.var;
                s_ids = d.ids;
            }
        }
        __syncthreads();
        const long long item = s_item;
        if (item >= items) break;
        const int64_t b0 = (item - __ldg(off + s_j)) * nb;
        for (int b = 0; b < nb; ++b)
            okrige_solve_block<K, false, false, kBatchSolveWarps>(
                s_h, s_g, s_k, s_p, 0, (int64_t)s_g.nx * s_g.ny, s_ids, s_depth, s_var, b0 + b, smem);
        __syncthreads();  // the next item overwrites the staged descriptor
    }
}

// 7. wide-key pass over every item of every tile; returns at once unless flagged
template <int K>
__device__ __forceinline__ void wide_node(const TileDesc& d, const HashView& h, NodeIdx nd) {
    const GridView& g = d.g;
    if (nd.i >= g.nx || nd.j >= g.ny || h.n_valid == 0) return;
    const int64_t node = (int64_t)nd.j * g.nx + nd.i;
    const int qx = g.x0 + nd.i * g.cell + g.cell / 2;
    const int qy = g.y0 + nd.j * g.cell + g.cell / 2;
    const int kq = d.method == 0 ? d.k : d.K;
    const Bound b = knn_bound_rt(h, qx, qy, kq);
    if (packed_fits(h, b.tau0)) return;
    uint64_t d2[K];
    int id[K];
    // the bound above used kq <= K soundings; the K-slot scan keeps the kq nearest in front
    const int keff = min(knn_scan<K, true>(h, qx, qy, b, d2, id), d.k);
    if (d.method == 0) {
        d.depth[node] = idw_from(h, keff, d.power, [&](int i, uint64_t& dd, int& ii) {
            dd = d2[i];
            ii = id[i];
        });
    } else {
        int32_t* o = d.ids + node * d.k;
        for (int i = 0; i < d.k; ++i) o[i] = i < keff ? id[i] : -1;
    }
}

__global__ void __launch_bounds__(kItemThreads) k_batch_wide(
    const TileDesc* __restrict__ td, int T, const int64_t* __restrict__ item_off, int64_t items,
    const int4* __restrict__ orig, const int4* __restrict__ rec, const int* __restrict__ cell_start,
    const int* __restrict__ sat, const int* __restrict__ wide) {
    if (*(volatile const int*)wide == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t item = blockIdx.x; item < items; item += gridDim.x) {
        const int t = upper_tile(item_off, T + 1, item);
        const TileDesc& d = td[t];
        const HashView h = tile_view(d, orig, rec, cell_start, sat);
        const int64_t patch = item - __ldg(item_off + t);
        const NodeIdx nd = patch_node((int)(patch % d.gx), (int)(patch / d.gx), warp, lane);
        const int kq = d.method == 0 ? d.k : d.K;
        if (kq <= 8)
            wide_node<8>(d, h, nd);
        else if (kq <= 16)
            wide_node<16>(d, h, nd);
        else
            wide_node<32>(d, h, nd);
    }
}

int grid_items(int64_t n, int per) { return (int)std::max<int64_t>(1, (n + per - 1) / per); }

}  // namespace
}  // namespace bg

struct bg_batch_s {
    bg_ctx_s* ctx = nullptr;
    int T = 0;
    float ppc = 2.0f;                      // soundings per hash cell (tuned)
    int strip = 1;                         // k-NN nodes per thread along x (tuned)
    int solve_nb = bg::kBatchSolveBlocks;  // solve block batches per claimed item (tuned)
    int off_nb = 0;                        // solve_nb the groups' item offsets hold
    std::vector<bg::TileDesc> host_desc;
    int64_t total_n = 0, total_cells = 0, total_sat = 0, total_ids = 0;
    int64_t knn_items = 0;                 // 16 x 8 patches (wide pass)
    int64_t knn_items_s[3] = {0, 0, 0};    // k-NN items per strip length 1, 2, 4
    struct Group {
        int K;
        int nt;
        int64_t items;
        int* tiles;       // device: tile indices
        int64_t* off;     // device: item prefix (nt + 1)
        std::vector<int64_t> nodes;  // host: nodes of each tile of the group
    };
    std::vector<Group> groups;
    // device buffers (one allocation, carved)
    void* mem = nullptr;
    size_t mem_bytes = 0;
    bg::TileDesc* d_desc = nullptr;
    int64_t* d_soff = nullptr;
    int64_t* d_item_off = nullptr;         // 16 x 8 patch prefix (wide pass)
    int64_t* d_item_off_s[3] = {nullptr, nullptr, nullptr};  // k-NN item prefix per strip
    int4* d_orig = nullptr;
    int4* d_rec = nullptr;
    int* d_cell_start = nullptr;
    int* d_count = nullptr;
    int* d_sat = nullptr;
    int* d_bsum = nullptr;
    int* d_acc = nullptr;
    int* d_flags = nullptr;                // [0] wide, [1] status
    unsigned long long* d_ctr = nullptr;   // item counters: [0] k-NN, [1 + g] solve groups
    int32_t* d_ids = nullptr;
    cudaStream_t stream = nullptr;
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int kernels_per_run = 0;               // kernel nodes of the captured graph
};

namespace bg {
namespace {

void enqueue_batch(bg_batch_s* b, cudaStream_t st) {
    const int T = b->T;
    const int64_t n = b->total_n;
    const int ng = (int)b->groups.size();
    cudaMemsetAsync(b->d_count, 0, (size_t)b->total_cells * 4, st);
    cudaMemsetAsync(b->d_flags, 0, 2 * sizeof(int), st);
    cudaMemsetAsync(b->d_ctr, 0, (size_t)(1 + ng) * sizeof(unsigned long long), st);
    k_batch_init<<<grid_items(T, 128), 128, 0, st>>>(b->d_acc, T);
    const int cb = grid_items(n, kChunk);
    if (n > 0)
        k_batch_validate<<<cb, kBT, 0, st>>>(b->d_desc, T, b->d_soff, n, b->d_orig, b->d_acc);
    k_batch_geom<<<grid_items(T, 64), 64, 0, st>>>(b->d_desc, T, b->d_acc, b->ppc, b->d_flags + 1);
    if (n > 0)
        k_batch_cells<false><<<cb, kBT, 0, st>>>(b->d_desc, T, b->d_soff, n, b->d_orig, b->d_count,
                                                 nullptr);
    launch_excl_scan(b->d_count, b->total_cells, b->d_cell_start, b->d_count, b->d_bsum, st);
    if (n > 0)
        k_batch_cells<true><<<cb, kBT, 0, st>>>(b->d_desc, T, b->d_soff, n, b->d_orig, b->d_count,
                                                b->d_rec);
    k_batch_sat<<<T, 128, 0, st>>>(b->d_desc, b->d_cell_start, b->d_sat);
    note_launches(6 + (n > 0 ? 3 : 0));
    // persistent kernels: as many blocks as an SM keeps resident drain the item lists
    if (b->knn_items > 0) {
        const int si = b->strip == 4 ? 2 : b->strip == 2 ? 1 : 0;
        const int64_t ki = b->knn_items_s[si];
        const unsigned kg = (unsigned)std::min<int64_t>(ki, 152 * 13);
#define BG_KNN(SS)                                                                               \
    k_batch_knn<SS><<<kg, kKnnThreads, 0, st>>>(b->d_desc, T, b->d_item_off_s[si], ki, b->d_ctr, \
                                                b->d_orig, b->d_rec, b->d_cell_start, b->d_sat,  \
                                                b->d_flags)
        if (b->strip == 4)
            BG_KNN(4);
        else if (b->strip == 2)
            BG_KNN(2);
        else
            BG_KNN(1);
#undef BG_KNN
        k_batch_wide<<<(unsigned)std::min<int64_t>(b->knn_items, 152 * 4), kItemThreads, 0, st>>>(
            b->d_desc, T, b->d_item_off, b->knn_items, b->d_orig, b->d_rec, b->d_cell_start,
            b->d_sat, b->d_flags);
        note_launches(2);
    }
    for (int gi = 0; gi < ng; ++gi) {
        const auto& G = b->groups[gi];
        if (G.items == 0) continue;
        const unsigned grid = (unsigned)std::min<int64_t>(G.items, 152 * kBatchSolveBlocksPerSM);
        unsigned long long* ctr = b->d_ctr + 1 + gi;
#define BG_SOLVE(KK)                                                                              \
    k_batch_solve<KK><<<grid, kBatchSolveWarps * 32, kBatchSolveWarps * Geo<KK>::WARP_FLOATS * 4, st>>>(b->d_desc, G.tiles, G.nt, G.off, G.items, \
                                                        ctr, b->d_orig, b->d_rec,                 \
                                                        b->d_cell_start, b->d_sat, b->solve_nb)
        switch (G.K) {
            case 4: BG_SOLVE(4); break;
            case 8: BG_SOLVE(8); break;
            case 16: BG_SOLVE(16); break;
            default: BG_SOLVE(32); break;
        }
#undef BG_SOLVE
        note_launches(1);
    }
}

cudaError_t set_batch_solve_smem() {
    cudaError_t e = cudaSuccess;
#define BG_SMEM(KK)                                                                          \
    if (e == cudaSuccess)                                                                    \
        e = cudaFuncSetAttribute(k_batch_solve<KK>, cudaFuncAttributeMaxDynamicSharedMemorySize, \
                                 kBatchSolveWarps * Geo<KK>::WARP_FLOATS * 4);
    BG_SMEM(4) BG_SMEM(8) BG_SMEM(16) BG_SMEM(32)
#undef BG_SMEM
    return e;
}

// The solve groups' item prefixes for the current solve item size: a tile of m
// nodes needs ceil(m / systems per item) items. Synchronous (never during
// capture); no graph may be running that reads the old offsets.
bg_status set_solve_offsets(bg_batch_s* b) {
    if (b->off_nb == b->solve_nb) return BG_OK;
    for (auto& G : b->groups) {
        const int sys_per_item = kBatchSolveWarps * (32 / (G.K / kR)) * kRounds * b->solve_nb;
        std::vector<int64_t> go(G.nodes.size() + 1, 0);
        for (size_t j = 0; j < G.nodes.size(); ++j)
            go[j + 1] = go[j] + (G.nodes[j] + sys_per_item - 1) / sys_per_item;
        G.items = go.back();
        const cudaError_t e = cudaMemcpy(G.off, go.data(), 8 * go.size(), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) return cuda_fail(e, "solve item offsets");
    }
    b->off_nb = b->solve_nb;
    return BG_OK;
}

bg_status drop_graph(bg_batch_s* b) {
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->exec = nullptr;
    b->graph = nullptr;
    return BG_OK;
}

}  // namespace
}  // namespace bg

using namespace bg;

extern "C" {

bg_status bg_batch_create(bg_ctx_t ctx, const bg_tile* tiles, int n_tiles, bg_batch_t* out) {
    if (!ctx || !out || (n_tiles > 0 && !tiles) || n_tiles < 0 || n_tiles > (1 << 20)) {
        set_error("bad arguments");
        return BG_ERR_INVALID_ARG;
    }
    *out = nullptr;
    for (int t = 0; t < n_tiles; ++t) {
        const bg_tile& r = tiles[t];
        const char* bad = nullptr;
        if (r.n < 0 || r.n >= ((int64_t)1 << 31) - 1) bad = "n out of range";
        else if (r.n > 0 && (!r.x_cm || !r.y_cm || !r.z_m)) bad = "NULL input pointer";
        else if (r.cell_cm <= 0 || r.cell_cm % 2 || r.nx <= 0 || r.ny <= 0) bad = "bad grid";
        else if ((int64_t)r.nx * r.ny > ((int64_t)1 << 36)) bad = "grid too large";
        else if (!r.depth_out) bad = "depth_out is NULL";
        else if (r.method != 0 && r.method != 1) bad = "method must be 0 (IDW) or 1 (kriging)";
        else if (r.k < 1 || r.k > 32) bad = "k must be in [1, 32]";
        else if (r.method == 0 && !(r.power > 0.0f && std::isfinite(r.power))) bad = "power must be > 0";
        else if (r.method == 1 && (!(r.variogram.model == 0 || r.variogram.model == 1) ||
                                   !(r.variogram.nugget_m2 >= 0.0f) ||
                                   !(r.variogram.sill_m2 > r.variogram.nugget_m2) ||
                                   !(r.variogram.range_m > 0.0f)))
            bad = "bad variogram";
        const int64_t lim = (int64_t)1 << 30;
        if (!bad && !((int64_t)r.x0_cm + r.cell_cm / 2 > -lim &&
                      (int64_t)r.x0_cm + (int64_t)(r.nx - 1) * r.cell_cm + r.cell_cm / 2 < lim &&
                      (int64_t)r.y0_cm + r.cell_cm / 2 > -lim &&
                      (int64_t)r.y0_cm + (int64_t)(r.ny - 1) * r.cell_cm + r.cell_cm / 2 < lim))
            bad = "grid node coordinates must lie in (-2^30, 2^30) cm";
        if (bad) {
            set_error(std::string("tile ") + std::to_string(t) + ": " + bad);
            return BG_ERR_INVALID_ARG;
        }
    }
    bg_batch_s* b = new (std::nothrow) bg_batch_s();
    if (!b) return BG_ERR_INTERNAL;
    b->ctx = ctx;
    b->T = n_tiles;
    b->host_desc.resize(n_tiles);
    std::vector<int64_t> soff(n_tiles + 1, 0), item_off(n_tiles + 1, 0);
    std::vector<std::vector<int64_t>> item_off_s(3, std::vector<int64_t>(n_tiles + 1, 0));
    const int Ks[4] = {4, 8, 16, 32};
    std::vector<std::vector<int>> gt(4);
    for (int t = 0; t < n_tiles; ++t) {
        const bg_tile& r = tiles[t];
        TileDesc& d = b->host_desc[t];
        d = TileDesc{};
        d.g = GridView{r.x0_cm, r.y0_cm, r.cell_cm, r.nx, r.ny};
        d.x = r.x_cm;
        d.y = r.y_cm;
        d.z = r.z_m;
        d.depth = r.depth_out;
        d.var = r.var_out;
        d.method = r.method;
        d.k = r.k;
        d.K = r.k <= 4 ? 4 : r.k <= 8 ? 8 : r.k <= 16 ? 16 : 32;
        d.power = r.power;
        const bg_variogram& v = r.variogram;
        if (r.method == 1)
            d.p = OkParams{v.model, v.nugget_m2, v.sill_m2 - v.nugget_m2, v.sill_m2, 1.0f / v.range_m};
        d.gx = (r.nx + 15) / 16;
        d.soff = b->total_n;
        d.n = r.n;
        d.cap = 4 * r.n + 4096;
        d.coff = b->total_cells;
        d.satcap = 2 * d.cap + 64;
        d.satoff = b->total_sat;
        int bits = 1;
        while (bits < 62 && (int64_t(1) << bits) < r.n) ++bits;
        d.h.idx_bits = bits;
        b->total_n += r.n;
        b->total_cells += d.cap;
        b->total_sat += d.satcap;
        soff[t + 1] = b->total_n;
        const int64_t m = (int64_t)r.nx * r.ny;
        item_off[t + 1] = item_off[t] + (int64_t)d.gx * ((r.ny + 7) / 8);
        for (int si = 0; si < 3; ++si)
            item_off_s[si][t + 1] = item_off_s[si][t] + (int64_t)((r.nx + 16 * kStrips[si] - 1) /
                                                                  (16 * kStrips[si])) *
                                                        ((r.ny + 7) / 8);
        if (r.method == 1) {
            b->total_ids += m * r.k;
            for (int q = 0; q < 4; ++q)
                if (Ks[q] == d.K) gt[q].push_back(t);
        }
    }
    b->knn_items = item_off[n_tiles];
    for (int si = 0; si < 3; ++si) b->knn_items_s[si] = item_off_s[si][n_tiles];
    // carve one allocation
    size_t off = 0;
    auto take = [&](size_t bytes) {
        const size_t o = off;
        off += (bytes + 255) & ~size_t(255);
        return o;
    };
    const size_t o_desc = take(sizeof(TileDesc) * std::max(1, n_tiles));
    const size_t o_soff = take(8 * (n_tiles + 1));
    const size_t o_item = take(8 * (n_tiles + 1));
    size_t o_item_s[3];
    for (int si = 0; si < 3; ++si) o_item_s[si] = take(8 * (n_tiles + 1));
    const size_t o_orig = take(16 * (size_t)b->total_n);
    const size_t o_rec = take(16 * (size_t)b->total_n);
    const size_t o_cs = take(4 * (size_t)(b->total_cells + 1));
    const size_t o_count = take(4 * (size_t)b->total_cells);
    const size_t o_sat = take(4 * (size_t)b->total_sat);
    const size_t o_bsum = take(4 * (size_t)(scan_blocks(b->total_cells) + 1));
    const size_t o_acc = take(32 * (size_t)std::max(1, n_tiles));
    const size_t o_flags = take(16);
    const size_t o_ctr = take(8 * 16);  // [0] k-NN items, [1 + g] solve groups
    const size_t o_ids = take(4 * (size_t)b->total_ids);
    std::vector<size_t> o_gt, o_go;
    for (int q = 0; q < 4; ++q) {
        o_gt.push_back(take(4 * (gt[q].size() + 1)));
        o_go.push_back(take(8 * (gt[q].size() + 1)));
    }
    b->mem_bytes = off;
    cudaStream_t st = nullptr;
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(ctx->device);
    cudaError_t e = set_batch_solve_smem();
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming);
    st = b->stream;
    bg_status rc = e == cudaSuccess ? BG_OK : cuda_fail(e, "batch stream");
    if (rc == BG_OK) rc = dalloc(ctx, &b->mem, b->mem_bytes, st);
    if (rc != BG_OK) {
        cudaSetDevice(prev);
        bg_batch_destroy(b);
        return rc;
    }
    char* base = (char*)b->mem;
    b->d_desc = (TileDesc*)(base + o_desc);
    b->d_soff = (int64_t*)(base + o_soff);
    b->d_item_off = (int64_t*)(base + o_item);
    for (int si = 0; si < 3; ++si) b->d_item_off_s[si] = (int64_t*)(base + o_item_s[si]);
    b->d_orig = (int4*)(base + o_orig);
    b->d_rec = (int4*)(base + o_rec);
    b->d_cell_start = (int*)(base + o_cs);
    b->d_count = (int*)(base + o_count);
    b->d_sat = (int*)(base + o_sat);
    b->d_bsum = (int*)(base + o_bsum);
    b->d_acc = (int*)(base + o_acc);
    b->d_flags = (int*)(base + o_flags);
    b->d_ctr = (unsigned long long*)(base + o_ctr);
    b->d_ids = (int32_t*)(base + o_ids);
    int64_t ids_at = 0;
    for (int t = 0; t < n_tiles; ++t) {
        TileDesc& d = b->host_desc[t];
        if (d.method == 1) {
            d.ids = b->d_ids + ids_at;
            ids_at += (int64_t)d.g.nx * d.g.ny * d.k;
        }
    }
    for (int q = 0; q < 4; ++q) {
        if (gt[q].empty()) continue;
        bg_batch_s::Group G{Ks[q], (int)gt[q].size(), 0, (int*)(base + o_gt[q]),
                            (int64_t*)(base + o_go[q]), {}};
        for (int t : gt[q])
            G.nodes.push_back((int64_t)b->host_desc[t].g.nx * b->host_desc[t].g.ny);
        e = cudaMemcpyAsync(G.tiles, gt[q].data(), 4 * gt[q].size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) break;
        b->groups.push_back(std::move(G));
        e = cudaStreamSynchronize(st);  // the host vectors go out of scope
        if (e != cudaSuccess) break;
    }
    if (e == cudaSuccess && set_solve_offsets(b) != BG_OK) e = cudaErrorUnknown;
    for (int si = 0; si < 3 && e == cudaSuccess; ++si)
        e = cudaMemcpyAsync(b->d_item_off_s[si], item_off_s[si].data(), 8 * (n_tiles + 1),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess && n_tiles > 0)
        e = cudaMemcpyAsync(b->d_desc, b->host_desc.data(), sizeof(TileDesc) * n_tiles,
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_soff, soff.data(), 8 * soff.size(), cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess)
        e = cudaMemcpyAsync(b->d_item_off, item_off.data(), 8 * item_off.size(),
                            cudaMemcpyHostToDevice, st);
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    cudaSetDevice(prev);
    if (e != cudaSuccess) {
        rc = cuda_fail(e, "batch set-up");
        bg_batch_destroy(b);
        return rc;
    }
    *out = b;
    return BG_OK;
}

bg_status bg_batch_run(bg_batch_t b, void* cuda_stream) {
    bg::NvtxRange nvtx("bg_batch_run");
    if (!b) {
        set_error("batch is NULL");
        return BG_ERR_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->ctx->device);
    const cudaStream_t user = (cudaStream_t)cuda_stream;
    cudaError_t e = cudaEventRecord(b->ev_in, user);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(b->stream, b->ev_in, 0);
    if (e == cudaSuccess && !b->exec) {
        if (b->off_nb != b->solve_nb) {
            // no replay of the previous graph may still read the offsets
            e = cudaStreamSynchronize(b->stream);
            if (e == cudaSuccess && set_solve_offsets(b) != BG_OK) e = cudaErrorUnknown;
        }
    }
    if (e == cudaSuccess && !b->exec) {
        const uint64_t before = g_launches.load();
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            enqueue_batch(b, b->stream);
            e = cudaStreamEndCapture(b->stream, &b->graph);
        }
        // kernels are counted when the graph runs, not when it is recorded
        b->kernels_per_run = (int)(g_launches.load() - before);
        g_launches.fetch_sub((uint64_t)b->kernels_per_run);
        if (e == cudaSuccess) e = cudaGraphInstantiate(&b->exec, b->graph, 0);
        if (e != cudaSuccess) drop_graph(b);
    }
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec, b->stream);
    if (e == cudaSuccess) note_launches(b->kernels_per_run);
    if (e == cudaSuccess) e = cudaEventRecord(b->ev_out, b->stream);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(user, b->ev_out, 0);
    cudaSetDevice(prev);
    return e == cudaSuccess ? BG_OK : cuda_fail(e, "bg_batch_run");
}

bg_status bg_batch_set_cell_target(bg_batch_t b, float soundings_per_cell) {
    if (!b || !(soundings_per_cell > 0.0f) || !(soundings_per_cell < 1e6f)) {
        set_error("bad arguments");
        return BG_ERR_INVALID_ARG;
    }
    if (soundings_per_cell != b->ppc) {
        b->ppc = soundings_per_cell;
        drop_graph(b);  // the next run captures a graph with the new target
    }
    return BG_OK;
}

bg_status bg_batch_set_shape(bg_batch_t b, int knn_strip, int solve_item) {
    if (!b || !(knn_strip == 1 || knn_strip == 2 || knn_strip == 4) ||
        !(solve_item == 1 || solve_item == 2 || solve_item == 4 || solve_item == 8 ||
          solve_item == 16)) {
        set_error("knn_strip must be 1, 2 or 4 and solve_item 1, 2, 4, 8 or 16");
        return BG_ERR_INVALID_ARG;
    }
    if (knn_strip != b->strip || solve_item != b->solve_nb) {
        b->strip = knn_strip;
        b->solve_nb = solve_item;
        drop_graph(b);  // the next run captures a graph with the new shape
    }
    return BG_OK;
}

bg_status bg_batch_get_config(bg_batch_t b, float* soundings_per_cell, int* knn_strip,
                              int* solve_item) {
    if (!b) {
        set_error("batch is NULL");
        return BG_ERR_INVALID_ARG;
    }
    if (soundings_per_cell) *soundings_per_cell = b->ppc;
    if (knn_strip) *knn_strip = b->strip;
    if (solve_item) *solve_item = b->solve_nb;
    return BG_OK;
}

bg_status bg_batch_tune(bg_batch_t b, void* cuda_stream, float* best_out) {
    if (!b) {
        set_error("batch is NULL");
        return BG_ERR_INVALID_ARG;
    }
    const cudaStream_t user = (cudaStream_t)cuda_stream;
    cudaEvent_t e0, e1;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    bg_status rc = BG_OK;
    // one configuration: capture + warm-up run, then two timed replays
    auto time_cfg = [&](float* ms) {
        if ((rc = bg_batch_run(b, user)) != BG_OK) return false;
        cudaEventRecord(e0, user);
        for (int i = 0; i < 2 && rc == BG_OK; ++i) rc = bg_batch_run(b, user);
        cudaEventRecord(e1, user);
        if (rc != BG_OK) return false;
        if (cudaEventSynchronize(e1) != cudaSuccess) {
            rc = cuda_fail(cudaGetLastError(), "tune");
            return false;
        }
        cudaEventElapsedTime(ms, e0, e1);
        return true;
    };
    // coordinate descent: the cell target, then the k-NN strip length, then
    // the solve item size, each with the others at their best so far
    const float cells[4] = {1.0f, 2.0f, 3.0f, 5.0f};
    const int strips[3] = {1, 2, 4}, items[4] = {2, 4, 8, 16};
    float best_ppc = b->ppc, best_ms = 1e30f, ms = 0.0f;
    int best_strip = b->strip, best_nb = b->solve_nb;
    for (float c : cells) {
        bg_batch_set_cell_target(b, c);
        if (!time_cfg(&ms)) break;
        if (ms < best_ms) {
            best_ms = ms;
            best_ppc = c;
        }
    }
    bg_batch_set_cell_target(b, best_ppc);
    for (int sv : strips) {
        if (rc != BG_OK) break;
        bg_batch_set_shape(b, sv, best_nb);
        if (!time_cfg(&ms)) break;
        if (ms < best_ms) {
            best_ms = ms;
            best_strip = sv;
        }
    }
    for (int nb : items) {
        if (rc != BG_OK) break;
        bg_batch_set_shape(b, best_strip, nb);
        if (!time_cfg(&ms)) break;
        if (ms < best_ms) {
            best_ms = ms;
            best_nb = nb;
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    bg_batch_set_cell_target(b, best_ppc);
    bg_batch_set_shape(b, best_strip, best_nb);
    if (best_out) *best_out = best_ppc;
    return rc;
}

bg_status bg_batch_status(bg_batch_t b, int* flags) {
    if (!b || !flags) {
        set_error("bad arguments");
        return BG_ERR_INVALID_ARG;
    }
    int h[2] = {0, 0};
    const cudaError_t e = cudaMemcpy(h, b->d_flags, sizeof(h), cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(e, "bg_batch_status");
    *flags = (h[1] ? 1 : 0) | (h[0] ? 2 : 0);
    return BG_OK;
}

bg_status bg_batch_destroy(bg_batch_t b) {
    if (!b) {
        set_error("batch is NULL");
        return BG_ERR_INVALID_ARG;
    }
    int prev = 0;
    cudaGetDevice(&prev);
    cudaSetDevice(b->ctx->device);
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graph(b);
    if (b->mem) dfree(b->ctx, b->mem, b->mem_bytes, b->stream);
    if (b->stream) {
        cudaStreamSynchronize(b->stream);
        cudaStreamDestroy(b->stream);
    }
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    cudaSetDevice(prev);
    delete b;
    return BG_OK;
}

}  // extern "C"
