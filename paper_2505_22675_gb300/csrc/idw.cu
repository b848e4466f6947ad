// Fused exact k-NN + inverse-distance weighting: per-grid kernels and launchers.
// The device code is in idw_dev.cuh.
#include <algorithm>

#include "idw_dev.cuh"

namespace bg {
namespace {

// Packed pass: one (16 * kLen) x 8 node patch per block, a strip of kLen
// nodes per thread (strip_len_for).
template <int K, int kLen>
__global__ void __launch_bounds__(128) k_idw(HashView h, GridView g, int k, float power,
                                             float* __restrict__ depth,
                                             int32_t* __restrict__ nbr, int* __restrict__ flag) {
    __shared__ uint64_t heap[K * 128];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gx = (g.nx + 16 * kLen - 1) / (16 * kLen);
    const NodeIdx o = strip_origin<kLen>(blockIdx.x % gx, blockIdx.x / gx, warp, lane);
    if (o.j >= g.ny) return;
    uint64_t* hp = heap + threadIdx.x;
    const int64_t row = (int64_t)o.j * g.nx;
    if (h.n_valid == 0) {
        for (int i = o.i; i < min(o.i + kLen, g.nx); ++i) {
            depth[row + i] = __int_as_float(0x7fc00000);
            if (nbr)
                for (int q = 0; q < k; ++q) nbr[(row + i) * k + q] = -1;
        }
        return;
    }
    const int bits = h.idx_bits;
    const uint64_t mask = (1ull << bits) - 1;
    auto emit = [&](int i, int cnt) {
        const int keff = min(cnt, k);
        depth[row + i] = idw_from(h, keff, power, [&](int q, uint64_t& dd, int& ii) {
            const uint64_t key = hp[q * 128];
            dd = key >> bits;
            ii = (int)(key & mask);
        });
        if (nbr) emit_ids<128>(nbr + (row + i) * k, hp, k, keff, mask);
    };
    knn_strip<128, decltype(emit), true, kLen>(h, g, K, o.i, o.j, hp, flag, emit);
}

// Wide-key pass over the nodes the packed pass could not take; it returns at
// once when the packed pass flagged none.
template <int K>
__global__ void __launch_bounds__(128) k_idw_wide(HashView h, GridView g, int k, float power,
                                                  float* __restrict__ depth,
                                                  int32_t* __restrict__ nbr, int* __restrict__ flag) {
    if (*(volatile int*)flag == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gx = (g.nx + 15) / 16;
    const int64_t nb = (int64_t)gx * ((g.ny + 7) / 8);
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x)
        idw_node<K, true>(h, g, k, power, depth, nbr, flag,
                          patch_node((int)(b % gx), (int)(b / gx), warp, lane), nullptr);
}

template <int K>
bg_status launch_k(const HashView& h, const GridView& g, int k, float power, float* depth,
                   int32_t* nbr, int* d_flag, cudaStream_t st, bg_ctx_s* prof_ctx) {
    const int64_t nb = (int64_t)((g.nx + 15) / 16) * ((g.ny + 7) / 8);
    const int len = strip_len_for((int64_t)g.nx * g.ny);
    const int64_t nbs = (int64_t)((g.nx + 16 * len - 1) / (16 * len)) * ((g.ny + 7) / 8);
    BG_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
    {
        ProfScope ps(prof_ctx, kProfIdw, (int64_t)g.nx * g.ny, st);
        if (len == 1)
            k_idw<K, 1><<<(unsigned)nbs, 128, 0, st>>>(h, g, k, power, depth, nbr, d_flag);
        else if (len == 2)
            k_idw<K, 2><<<(unsigned)nbs, 128, 0, st>>>(h, g, k, power, depth, nbr, d_flag);
        else
            k_idw<K, 4><<<(unsigned)nbs, 128, 0, st>>>(h, g, k, power, depth, nbr, d_flag);
    }
    k_idw_wide<K><<<(unsigned)std::min<int64_t>(nb, 152 * 4), 128, 0, st>>>(h, g, k, power, depth,
                                                                        nbr, d_flag);
    note_launches(2);
    BG_CUDA(cudaGetLastError());
    return BG_OK;
}

// Query points: kLen consecutive points per thread (knn_chain).
template <int K, int kLen>
__global__ void __launch_bounds__(128) k_idw_pts(HashView h, PointsView q, int k, float power,
                                                 float* __restrict__ depth,
                                                 int32_t* __restrict__ nbr, int* __restrict__ flag) {
    __shared__ uint64_t heap[K * 128];
    const int64_t p0 = ((int64_t)blockIdx.x * 128 + threadIdx.x) * kLen;
    if (p0 >= q.m) return;
    uint64_t* hp = heap + threadIdx.x;
    const int bits = h.idx_bits;
    const uint64_t mask = (1ull << bits) - 1;
    auto none = [&](int64_t p) {
        depth[p] = __int_as_float(0x7fc00000);
        if (nbr)
            for (int i = 0; i < k; ++i) nbr[p * k + i] = -1;
    };
    if (h.n_valid == 0) {
        for (int64_t p = p0; p < min(p0 + kLen, q.m); ++p) none(p);
        return;
    }
    auto emit = [&](int64_t p, int cnt) {
        if (cnt < 0) {
            none(p);
            return;
        }
        const int keff = min(cnt, k);
        depth[p] = idw_from(h, keff, power, [&](int i, uint64_t& dd, int& ii) {
            const uint64_t key = hp[i * 128];
            dd = key >> bits;
            ii = (int)(key & mask);
        });
        if (nbr) emit_ids<128>(nbr + p * k, hp, k, keff, mask);
    };
    knn_chain<128, decltype(emit), kLen>(h, q.x, q.y, p0, q.m, K, hp, flag, emit);
}

template <int K>
__global__ void __launch_bounds__(128) k_idw_pts_wide(HashView h, PointsView q, int k, float power,
                                                      float* __restrict__ depth,
                                                      int32_t* __restrict__ nbr,
                                                      int* __restrict__ flag) {
    if (*(volatile int*)flag == 0) return;
    for (int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < q.m;
         p += (int64_t)gridDim.x * blockDim.x)
        idw_point_wide<K>(h, __ldg(q.x + p), __ldg(q.y + p), k, power, depth + p,
                          nbr ? nbr + p * k : nullptr);
}

template <int K>
bg_status launch_pts_k(const HashView& h, const PointsView& q, int k, float power, float* depth,
                       int32_t* nbr, int* d_flag, cudaStream_t st, bg_ctx_s* prof_ctx) {
    const int len = strip_len_for(q.m);
    const int64_t threads = (q.m + len - 1) / len;
    const int64_t nb = (threads + 127) / 128;
    BG_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
    {
        ProfScope ps(prof_ctx, kProfIdw, q.m, st);
        if (len == 1)
            k_idw_pts<K, 1><<<(unsigned)nb, 128, 0, st>>>(h, q, k, power, depth, nbr, d_flag);
        else if (len == 2)
            k_idw_pts<K, 2><<<(unsigned)nb, 128, 0, st>>>(h, q, k, power, depth, nbr, d_flag);
        else
            k_idw_pts<K, 4><<<(unsigned)nb, 128, 0, st>>>(h, q, k, power, depth, nbr, d_flag);
    }
    k_idw_pts_wide<K><<<(unsigned)std::min<int64_t>((q.m + 127) / 128, 152 * 4), 128, 0, st>>>(
        h, q, k, power, depth, nbr, d_flag);
    note_launches(2);
    BG_CUDA(cudaGetLastError());
    return BG_OK;
}

}  // namespace

bg_status launch_idw_points(const bg_soundings_s* s, const PointsView& q, int k, float power,
                            float* depth, int32_t* nbr, cudaStream_t st) {
    if (q.m == 0) return BG_OK;
    HashView h = s->h;
    const int K = k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
    h.r0 = start_halfwidth(s, K);
    int* flag = nullptr;
    bg_status rc = dalloc(s->ctx, (void**)&flag, sizeof(int), st);
    if (rc != BG_OK) return rc;
    switch (K) {
        case 4: rc = launch_pts_k<4>(h, q, k, power, depth, nbr, flag, st, s->ctx); break;
        case 8: rc = launch_pts_k<8>(h, q, k, power, depth, nbr, flag, st, s->ctx); break;
        case 16: rc = launch_pts_k<16>(h, q, k, power, depth, nbr, flag, st, s->ctx); break;
        default: rc = launch_pts_k<32>(h, q, k, power, depth, nbr, flag, st, s->ctx); break;
    }
    dfree(s->ctx, flag, sizeof(int), st);
    return rc;
}

bg_status launch_idw(const bg_soundings_s* s, const GridView& g, int k, float power,
                     float* depth, int32_t* nbr, cudaStream_t st) {
    HashView h = s->h;
    const int K = k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
    h.r0 = start_halfwidth(s, K);
    int* flag = nullptr;
    bg_status rc = dalloc(s->ctx, (void**)&flag, sizeof(int), st);
    if (rc != BG_OK) return rc;
    switch (K) {
        case 4: rc = launch_k<4>(h, g, k, power, depth, nbr, flag, st, s->ctx); break;
        case 8: rc = launch_k<8>(h, g, k, power, depth, nbr, flag, st, s->ctx); break;
        case 16: rc = launch_k<16>(h, g, k, power, depth, nbr, flag, st, s->ctx); break;
        default: rc = launch_k<32>(h, g, k, power, depth, nbr, flag, st, s->ctx); break;
    }
    dfree(s->ctx, flag, sizeof(int), st);
    return rc;
}

bg_status launch_idw_with_flag(const bg_soundings_s* s, const GridView& g, int k, float power,
                               float* depth, int32_t* nbr, int* d_flag, cudaStream_t st) {
    HashView h = s->h;
    const int K = k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
    h.r0 = start_halfwidth(s, K);
    switch (K) {
        case 4: return launch_k<4>(h, g, k, power, depth, nbr, d_flag, st, s->ctx);
        case 8: return launch_k<8>(h, g, k, power, depth, nbr, d_flag, st, s->ctx);
        case 16: return launch_k<16>(h, g, k, power, depth, nbr, d_flag, st, s->ctx);
        default: return launch_k<32>(h, g, k, power, depth, nbr, d_flag, st, s->ctx);
    }
}

}  // namespace bg
