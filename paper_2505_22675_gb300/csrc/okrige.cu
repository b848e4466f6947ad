// Local ordinary kriging (Sec. III-C): the per-grid kernels and their launcher.
// The device code (k-NN to ids, reduced-system assembly, Cholesky, refinement)
// is in okrige_dev.cuh; see there for the formulation.
#include <algorithm>

#include "okrige_dev.cuh"

namespace bg {
namespace {

// grid rows [j0, j1); j0 is a multiple of 8; a strip of kLen nodes per thread
// (strip_len_for). 64-thread blocks: the 16 KB heap (K = 32) plus the
// per-block reserve lets 13 blocks (26 warps) share an SM, against 6 blocks
// (24 warps) of 128.
template <int K, int kLen>
__global__ void __launch_bounds__(64) k_knn_ids(HashView h, GridView g, int k, int j0, int j1,
                                                int32_t* __restrict__ ids, int* __restrict__ flag) {
    __shared__ uint64_t heap[K * 64];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gx = (g.nx + 16 * kLen - 1) / (16 * kLen);
    // (16 * kLen) x 4 node patches: warp w covers columns w * 8 * kLen ..
    const int px = blockIdx.x % gx, py = j0 / 4 + blockIdx.x / gx;
    const NodeIdx o{px * 16 * kLen + warp * 8 * kLen + (lane & 7) * kLen, py * 4 + (lane >> 3)};
    if (o.j >= j1) return;
    uint64_t* hp = heap + threadIdx.x;
    int32_t* base = ids + ((int64_t)(o.j - j0) * g.nx) * k;
    if (h.n_valid == 0) {
        for (int i = o.i; i < min(o.i + kLen, g.nx); ++i)
            for (int q = 0; q < k; ++q) base[(int64_t)i * k + q] = -1;
        return;
    }
    const uint64_t mask = (1ull << h.idx_bits) - 1;
    // k == K (a multiple of 4) puts every node's ids on a 16-byte boundary when
    // the buffer is aligned: a full heap is then drained straight into them,
    // four ids per store; otherwise it is sorted in place and copied out
    const bool vec = k == K && K % 4 == 0 && (reinterpret_cast<uintptr_t>(ids) & 15) == 0;
    auto emit = [&](int i, int cnt) {
        int32_t* out = base + (int64_t)i * k;
        if (vec && cnt == K) {
            drain_ids<K, 64>(out, hp, mask);
            return;
        }
        for (int e = cnt - 1; e > 0; --e) {  // heapsort of a partial heap
            const uint64_t v = hp[e * 64];
            hp[e * 64] = hp[0];
            heap_sift_down<64>(hp, 0, e, v);
        }
        emit_ids<64>(out, hp, k, cnt, mask);
    };
    knn_strip<64, decltype(emit), false, kLen>(h, g, K, o.i, o.j, hp, flag, emit);
}

template <int K>
__global__ void __launch_bounds__(128) k_knn_ids_wide(HashView h, GridView g, int k, int j0,
                                                      int j1, int32_t* __restrict__ ids,
                                                      int* __restrict__ flag) {
    if (*(volatile int*)flag == 0) return;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gx = (g.nx + 15) / 16;
    const int64_t nb = (int64_t)gx * ((j1 - j0 + 7) / 8);
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x)
        knn_ids_node<K, true>(h, g, k, (int64_t)j0 * g.nx, ids, flag,
                              patch_node((int)(b % gx), j0 / 8 + (int)(b / gx), warp, lane), j1,
                              nullptr);
}

// dynamic shared memory: kGridSolveWarps * Geo<K>::WARP_FLOATS floats
template <int K, bool kIdw>
__global__ void __launch_bounds__(kGridSolveWarps * 32, kGridSolveBlocksPerSM) k_okrige_solve(
    HashView h, GridView g, int k, OkParams p, int64_t node0, int64_t nodes,
    const int32_t* __restrict__ ids, float* __restrict__ depth, float* __restrict__ var,
    IdwFuse fz) {
    extern __shared__ __align__(16) float smem[];
    // the ids of a block two waves on (2 blocks per SM): the k-NN kernel wrote
    // them a launch ago and they have left L2 since
    prefetch_ids_l2(ids, nodes, k, (int64_t)blockIdx.x + kIdsPrefetchBlocks,
                    kGridSolveWarps * Geo<K>::SYS * kRounds);
    okrige_solve_block<K, false, kIdw, kGridSolveWarps>(h, g, k, p, node0, nodes, ids, depth, var,
                                                        blockIdx.x, smem, nullptr, nullptr, fz);
}

// Copy rows [off, off + n) of the outputs to their host destinations on
// ho->cs, after the work enqueued so far on st.
bg_status copy_rows_to_host(const HostOut* ho, int64_t off, int64_t n, const float* idw,
                            const float* depth, const float* var, cudaStream_t st) {
    cudaError_t e = cudaEventRecord(ho->ev, st);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(ho->cs, ho->ev, 0);
    const size_t bytes = (size_t)n * sizeof(float);
    if (e == cudaSuccess && ho->idw && idw)
        e = cudaMemcpyAsync(ho->idw + off, idw + off, bytes, cudaMemcpyDeviceToHost, ho->cs);
    if (e == cudaSuccess && ho->depth)
        e = cudaMemcpyAsync(ho->depth + off, depth + off, bytes, cudaMemcpyDeviceToHost, ho->cs);
    if (e == cudaSuccess && ho->var && var)
        e = cudaMemcpyAsync(ho->var + off, var + off, bytes, cudaMemcpyDeviceToHost, ho->cs);
    return e == cudaSuccess ? BG_OK : cuda_fail(e, "device-to-host copy");
}

template <int K>
bg_status launch_k(const HashView& h, const GridView& g, int k, const OkParams& p, float* depth,
                   float* var, int32_t* nbr, bg_ctx_s* ctx, cudaStream_t st, const IdwFuse* fz,
                   const HostOut* ho) {
    using Gm = Geo<K>;
    // grid rows per chunk: the id buffer stays near 1 GiB unless the caller
    // passed nbr_out, which then holds all ids
    int64_t rows = g.ny;
    if (!nbr) rows = std::max<int64_t>(8, ((((int64_t)1 << 28) / ((int64_t)k * g.nx)) / 8) * 8);
    if (rows > g.ny) rows = g.ny;
    const size_t flag_bytes = 256;
    const size_t id_bytes = nbr ? 0 : (size_t)rows * g.nx * k * sizeof(int32_t);
    void* scratch = nullptr;
    bg_status rc = dalloc(ctx, &scratch, flag_bytes + id_bytes, st);
    if (rc != BG_OK) return rc;
    int* flag = (int*)scratch;
    const int gx = (g.nx + 15) / 16;
    const int64_t sys_per_block = (int64_t)kGridSolveWarps * Gm::SYS * kRounds;
    const int smem_bytes = kGridSolveWarps * Gm::WARP_FLOATS * (int)sizeof(float);
    cudaError_t ea = cudaFuncSetAttribute(k_okrige_solve<K, false>,
                                          cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if constexpr (K == 32)
        if (ea == cudaSuccess)
            ea = cudaFuncSetAttribute(k_okrige_solve<K, true>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (ea != cudaSuccess) {
        dfree(ctx, scratch, flag_bytes + id_bytes, st);
        return cuda_fail(ea, "solve shared-memory size");
    }
    for (int64_t j0 = 0; j0 < g.ny; j0 += rows) {
        const int64_t j1 = std::min<int64_t>(g.ny, j0 + rows);
        const int64_t nb = (int64_t)gx * ((j1 - j0 + 7) / 8);
        const int len = strip_len_for((j1 - j0) * (int64_t)g.nx);
        const int64_t nbs = (int64_t)((g.nx + 16 * len - 1) / (16 * len)) * ((j1 - j0 + 3) / 4);
        int32_t* chunk_ids = nbr ? nbr + j0 * g.nx * k : (int32_t*)((char*)scratch + flag_bytes);
        cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "memset");
            break;
        }
        const int64_t nodes = (j1 - j0) * g.nx;
        {
            ProfScope ps(ctx, kProfKnnIds, nodes, st);
            if (len == 1)
                k_knn_ids<K, 1><<<(unsigned)nbs, 64, 0, st>>>(h, g, k, (int)j0, (int)j1, chunk_ids, flag);
            else if (len == 2)
                k_knn_ids<K, 2><<<(unsigned)nbs, 64, 0, st>>>(h, g, k, (int)j0, (int)j1, chunk_ids, flag);
            else
                k_knn_ids<K, 4><<<(unsigned)nbs, 64, 0, st>>>(h, g, k, (int)j0, (int)j1, chunk_ids, flag);
        }
        k_knn_ids_wide<K><<<(unsigned)std::min<int64_t>(nb, 152 * 4), 128, 0, st>>>(
            h, g, k, (int)j0, (int)j1, chunk_ids, flag);
        const int64_t sb = (nodes + sys_per_block - 1) / sys_per_block;
        {
            ProfScope ps(ctx, kProfSolve, nodes, st);
            bool fused = false;
            if constexpr (K == 32) {  // the fused IDW runs with 8 threads per system
                if (fz) {
                    k_okrige_solve<K, true><<<(unsigned)sb, kGridSolveWarps * 32, smem_bytes, st>>>(
                        h, g, k, p, j0 * g.nx, nodes, chunk_ids, depth, var, *fz);
                    fused = true;
                }
            }
            if (!fused)
                k_okrige_solve<K, false><<<(unsigned)sb, kGridSolveWarps * 32, smem_bytes, st>>>(
                    h, g, k, p, j0 * g.nx, nodes, chunk_ids, depth, var, IdwFuse{});
        }
        note_launches(3);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "kriging launch");
            break;
        }
        if (ho) {
            rc = copy_rows_to_host(ho, j0 * g.nx, nodes, fz ? fz->out : nullptr, depth, var, st);
            if (rc != BG_OK) break;
        }
    }
    if (ho && rc == BG_OK) {  // later work on st waits for the last copy
        cudaError_t e = cudaEventRecord(ho->ev, ho->cs);
        if (e == cudaSuccess) e = cudaStreamWaitEvent(st, ho->ev, 0);
        if (e != cudaSuccess) rc = cuda_fail(e, "copy-stream join");
    }
    dfree(ctx, scratch, flag_bytes + id_bytes, st);
    return rc;
}

// ------------------------------------------------------------ query points

// points [p0, p1), kLen consecutive points per thread (strip_len_for)
template <int K, int kLen>
__global__ void __launch_bounds__(128) k_knn_ids_pts(HashView h, PointsView q, int k, int64_t p0,
                                                     int64_t p1, int32_t* __restrict__ ids,
                                                     int* __restrict__ flag) {
    __shared__ uint64_t heap[K * 128];
    const int64_t a = p0 + ((int64_t)blockIdx.x * 128 + threadIdx.x) * kLen;
    if (a >= p1) return;
    uint64_t* hp = heap + threadIdx.x;
    if (h.n_valid == 0) {
        for (int64_t p = a; p < min(a + kLen, p1); ++p)
            for (int i = 0; i < k; ++i) ids[(p - p0) * k + i] = -1;
        return;
    }
    const uint64_t mask = (1ull << h.idx_bits) - 1;
    auto emit = [&](int64_t p, int cnt) { emit_ids<128>(ids + (p - p0) * k, hp, k, cnt, mask); };
    knn_chain<128, decltype(emit), kLen>(h, q.x, q.y, a, p1, K, hp, flag, emit);
}

template <int K>
__global__ void __launch_bounds__(128) k_knn_ids_pts_wide(HashView h, PointsView q, int k,
                                                          int64_t p0, int64_t p1,
                                                          int32_t* __restrict__ ids,
                                                          int* __restrict__ flag) {
    if (*(volatile int*)flag == 0) return;
    for (int64_t p = p0 + (int64_t)blockIdx.x * blockDim.x + threadIdx.x; p < p1;
         p += (int64_t)gridDim.x * blockDim.x)
        knn_ids_point_wide<K>(h, __ldg(q.x + p), __ldg(q.y + p), k, ids + (p - p0) * k);
}

// dynamic shared memory: kGridSolveWarps * Geo<K>::WARP_FLOATS floats
template <int K>
__global__ void __launch_bounds__(kGridSolveWarps * 32, kGridSolveBlocksPerSM) k_okrige_solve_pts(
    HashView h, PointsView q, int k, OkParams p, int64_t p0, int64_t nodes,
    const int32_t* __restrict__ ids, float* __restrict__ depth, float* __restrict__ var) {
    extern __shared__ __align__(16) float smem[];
    prefetch_ids_l2(ids, nodes, k, (int64_t)blockIdx.x + kIdsPrefetchBlocks,
                    kGridSolveWarps * Geo<K>::SYS * kRounds);
    okrige_solve_block<K, true, false, kGridSolveWarps>(h, GridView{}, k, p, p0, nodes, ids, depth,
                                                        var, blockIdx.x, smem, q.x, q.y);
}

template <int K>
bg_status launch_pts_k(const HashView& h, const PointsView& q, int k, const OkParams& p,
                       float* depth, float* var, int32_t* nbr, bg_ctx_s* ctx, cudaStream_t st) {
    using Gm = Geo<K>;
    // points per chunk: the id buffer stays near 1 GiB unless the caller
    // passed nbr_out, which then holds all ids
    int64_t per = q.m;
    if (!nbr) per = std::min<int64_t>(q.m, std::max<int64_t>(4096, ((int64_t)1 << 28) / k));
    const size_t flag_bytes = 256;
    const size_t id_bytes = nbr ? 0 : (size_t)per * k * sizeof(int32_t);
    void* scratch = nullptr;
    bg_status rc = dalloc(ctx, &scratch, flag_bytes + id_bytes, st);
    if (rc != BG_OK) return rc;
    int* flag = (int*)scratch;
    const int64_t sys_per_block = (int64_t)kGridSolveWarps * Gm::SYS * kRounds;
    const int smem_bytes = kGridSolveWarps * Gm::WARP_FLOATS * (int)sizeof(float);
    const cudaError_t ea = cudaFuncSetAttribute(
        k_okrige_solve_pts<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem_bytes);
    if (ea != cudaSuccess) {
        dfree(ctx, scratch, flag_bytes + id_bytes, st);
        return cuda_fail(ea, "solve shared-memory size");
    }
    for (int64_t p0 = 0; p0 < q.m; p0 += per) {
        const int64_t p1 = std::min<int64_t>(q.m, p0 + per);
        const int64_t n = p1 - p0;
        int32_t* chunk_ids = nbr ? nbr + p0 * k : (int32_t*)((char*)scratch + flag_bytes);
        cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "memset");
            break;
        }
        const int len = strip_len_for(n);
        const int64_t nb = ((n + len - 1) / len + 127) / 128;
        {
            ProfScope ps(ctx, kProfKnnIds, n, st);
            if (len == 1)
                k_knn_ids_pts<K, 1><<<(unsigned)nb, 128, 0, st>>>(h, q, k, p0, p1, chunk_ids, flag);
            else if (len == 2)
                k_knn_ids_pts<K, 2><<<(unsigned)nb, 128, 0, st>>>(h, q, k, p0, p1, chunk_ids, flag);
            else
                k_knn_ids_pts<K, 4><<<(unsigned)nb, 128, 0, st>>>(h, q, k, p0, p1, chunk_ids, flag);
        }
        k_knn_ids_pts_wide<K><<<(unsigned)std::min<int64_t>((n + 127) / 128, 152 * 4), 128, 0, st>>>(
            h, q, k, p0, p1, chunk_ids, flag);
        const int64_t sb = (n + sys_per_block - 1) / sys_per_block;
        {
            ProfScope ps(ctx, kProfSolve, n, st);
            k_okrige_solve_pts<K><<<(unsigned)sb, kGridSolveWarps * 32, smem_bytes, st>>>(
                h, q, k, p, p0, n, chunk_ids, depth, var);
        }
        note_launches(3);
        e = cudaGetLastError();
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "kriging launch");
            break;
        }
    }
    dfree(ctx, scratch, flag_bytes + id_bytes, st);
    return rc;
}

}  // namespace

bg_status launch_okrige_points(const bg_soundings_s* s, const PointsView& q, int k,
                               const OkParams& p, float* depth, float* var, int32_t* nbr,
                               cudaStream_t st) {
    if (q.m == 0) return BG_OK;
    HashView h = s->h;
    const int K = k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
    h.r0 = start_halfwidth(s, K);
    switch (K) {
        case 4: return launch_pts_k<4>(h, q, k, p, depth, var, nbr, s->ctx, st);
        case 8: return launch_pts_k<8>(h, q, k, p, depth, var, nbr, s->ctx, st);
        case 16: return launch_pts_k<16>(h, q, k, p, depth, var, nbr, s->ctx, st);
        default: return launch_pts_k<32>(h, q, k, p, depth, var, nbr, s->ctx, st);
    }
}

bg_status launch_okrige(const bg_soundings_s* s, const GridView& g, int k, const OkParams& p,
                        float* depth, float* var, int32_t* nbr, cudaStream_t st,
                        const IdwFuse* fz, const HostOut* ho) {
    HashView h = s->h;
    const int K = k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
    if (fz && K != 32) {
        // smaller systems run 2 or 4 threads each: the IDW takes its own pass
        // (the same depths: idw_from sums in the same fixed order)
        bg_status rc = launch_idw(s, g, fz->k, fz->power, fz->out, nullptr, st);
        if (rc != BG_OK) return rc;
        if (ho && ho->idw) {  // the whole IDW grid is done: copy it now
            HostOut only_idw = *ho;
            only_idw.depth = only_idw.var = nullptr;
            rc = copy_rows_to_host(&only_idw, 0, (int64_t)g.nx * g.ny, fz->out, nullptr, nullptr, st);
            if (rc != BG_OK) return rc;
        }
        fz = nullptr;
    }
    h.r0 = start_halfwidth(s, K);
    switch (K) {
        case 4: return launch_k<4>(h, g, k, p, depth, var, nbr, s->ctx, st, fz, ho);
        case 8: return launch_k<8>(h, g, k, p, depth, var, nbr, s->ctx, st, fz, ho);
        case 16: return launch_k<16>(h, g, k, p, depth, var, nbr, s->ctx, st, fz, ho);
        default: return launch_k<32>(h, g, k, p, depth, var, nbr, s->ctx, st, fz, ho);
    }
}

}  // namespace bg
