// Fused exact k-NN + local ordinary kriging (Sec. III-C), one warp per system.
//
// Each thread first finds the k nearest soundings of its own node (the
// search of knn.cuh); the warp then solves its 32 nodes' kriging systems one
// after another, lane a holding neighbour a.
//
// The bordered variogram system [Gamma 1; 1^T 0][lambda; mu] = [gamma_0; 1]
// is reduced with the constraint sum(lambda) = 1: eliminating lambda_0 (the
// nearest neighbour) and mu leaves, for a, c = 1..k-1,
//     A[a][c] = Gamma_a0 + Gamma_c0 - Gamma_ac,   b_a = Gamma_a0 + gamma_00 - gamma_a0,
//     A lambda' = b,   lambda_0 = 1 - sum(lambda'),   mu = gamma_00 - sum_a Gamma_0a lambda_a.
// A is symmetric positive definite for a valid variogram (one that is
// conditionally negative definite), so it is factored by Cholesky in FP32.
// One step of iterative refinement follows: the residual b - A lambda' is
// accumulated in FP64 (every FP32 x FP32 product is exact in FP64), and the
// correction reuses the factor. lambda_0 = 1 - sum(lambda') is accumulated in
// FP64, which closes the weight sum. Outputs:
//     zhat    = z_0 + sum_a lambda_a (z_a - z_0)            (= sum lambda_i z_i)
//     sigma^2 = lambda_0 gamma_00 + sum_a lambda_a gamma_a0 + mu.
// Unused rows (lane 0, lanes >= k_eff) are identity rows with a zero right-hand
// side, so every system has the same fixed shape and the loops fully unroll.
#include <cmath>

#include "bg_internal.h"
#include "knn.cuh"

namespace bg {
namespace {

constexpr int kWarps = 4;

__device__ __forceinline__ float variogram(const OkParams& p, float h_m) {
    if (p.model == BG_VARIOGRAM_SPHERICAL) {
        const float t = h_m * p.inv_a;
        if (t >= 1.0f) return p.sill;
        return fmaf(p.c * t, fmaf(-0.5f * t, t, 1.5f), p.c0);
    }
    return fmaf(p.c, 1.0f - expf(-h_m * p.inv_a), p.c0);
}

// gamma between two soundings (dx, dy in cm); distinct soundings at one position get c0
__device__ __forceinline__ float gamma_pair(const OkParams& p, int dx, int dy) {
    if (dx == 0 && dy == 0) return p.c0;
    const float fx = (float)dx, fy = (float)dy;
    return variogram(p, sqrtf(fmaf(fx, fx, fy * fy)) * 0.01f);
}

// gamma between the node and a sounding; 0 when the node sits on it
__device__ __forceinline__ float gamma_node(const OkParams& p, int dx, int dy) {
    if (dx == 0 && dy == 0) return 0.0f;
    const float fx = (float)dx, fy = (float)dy;
    return variogram(p, sqrtf(fmaf(fx, fx, fy * fy)) * 0.01f);
}

__device__ __forceinline__ float warp_sum(float v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
    return v;
}

// Solve L L^T x = rhs with L held as rows in registers (Lr, lane a = row a)
// and in shared memory (sL, for the transposed sweep). dinv[j] = 1 / L[j][j].
template <int K>
__device__ __forceinline__ float chol_solve(const float (&Lr)[K], const float* sL,
                                            const float (&dinv)[K], float rhs, int a) {
    float y = rhs;
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float yj = __shfl_sync(kFull, y, j) * dinv[j];
        if (a == j)
            y = yj;
        else if (a > j)
            y = fmaf(-Lr[j], yj, y);
    }
    float x = y;
#pragma unroll
    for (int j = K - 1; j >= 0; --j) {
        const float xj = __shfl_sync(kFull, x, j) * dinv[j];
        if (a == j)
            x = xj;
        else if (a < j)
            x = fmaf(-sL[j * (K + 1) + a], xj, x);
    }
    return x;
}

// One kriging system, solved by the whole warp. ids: the node's neighbours
// (shared memory, ascending), ke: how many of them to use (1..K).
template <int K>
__device__ __forceinline__ void solve_system(const HashView& h, const OkParams& p, int qx, int qy,
                                             const int* ids, int ke, float* sL, int64_t node,
                                             float* __restrict__ depth, float* __restrict__ var) {
    const int a = threadIdx.x & 31;
    const bool real = a < ke;
    int4 r = make_int4(0, 0, 0, 0);
    if (real) r = __ldg(h.orig + ids[a]);
    const int xa = r.x, ya = r.y;
    const float za = __int_as_float(r.z);
    const float ga0 = real ? gamma_node(p, xa - qx, ya - qy) : 0.0f;  // gamma(node, a)
    const int x0 = __shfl_sync(kFull, xa, 0), y0 = __shfl_sync(kFull, ya, 0);
    const float z0 = __shfl_sync(kFull, za, 0);
    const float g00 = __shfl_sync(kFull, ga0, 0);
    const float Ga0 = (a == 0) ? 0.0f : gamma_pair(p, xa - x0, ya - y0);  // Gamma(a, 0)
    const bool row = real && a >= 1;

    // assemble the reduced system, row a on lane a
    float A[K];
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const int xc = __shfl_sync(kFull, xa, c), yc = __shfl_sync(kFull, ya, c);
        const float Gc0 = __shfl_sync(kFull, Ga0, c);
        const float Gac = (a == c) ? 0.0f : gamma_pair(p, xa - xc, ya - yc);
        const bool col = c >= 1 && c < ke;
        A[c] = row ? (col ? (Ga0 + Gc0) - Gac : 0.0f) : (a == c ? 1.0f : 0.0f);
    }
    const float b = row ? (Ga0 + g00) - ga0 : 0.0f;
    float A0[K];
#pragma unroll
    for (int c = 0; c < K; ++c) A0[c] = A[c];

    // Cholesky, right-looking: column j is scaled by 1/L[j][j], then the
    // trailing rows are updated with column j broadcast lane by lane
    float dinv[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
        const float ljj = sqrtf(__shfl_sync(kFull, A[j], j));
        const float inv = 1.0f / ljj;
        dinv[j] = inv;
        const float laj = (a > j) ? A[j] * inv : (a == j ? ljj : A[j]);
        A[j] = laj;
#pragma unroll
        for (int c = j + 1; c < K; ++c) {
            const float lcj = __shfl_sync(kFull, laj, c);
            A[c] = fmaf(-laj, lcj, A[c]);  // lanes a < c touch only their unused upper part
        }
    }
    if (a < K) {  // lanes beyond K (K < 32) hold no row
#pragma unroll
        for (int c = 0; c < K; ++c) sL[a * (K + 1) + c] = A[c];
    }
    __syncwarp();

    float x = chol_solve<K>(A, sL, dinv, b, a);

    // one refinement step: residual in FP64, correction with the FP32 factor
    double res = (double)b;
#pragma unroll
    for (int c = 0; c < K; ++c) {
        const float xc = __shfl_sync(kFull, x, c);
        res = fma(-(double)A0[c], (double)xc, res);
    }
    x += chol_solve<K>(A, sL, dinv, (float)res, a);
    __syncwarp();  // sL is rewritten by the next system

    const float lam = row ? x : 0.0f;
    const double wsum = warp_sum(row ? (double)x : 0.0);
    const float lam0 = (float)(1.0 - wsum);
    const float zsum = warp_sum(lam * (za - z0));
    const float vsum = warp_sum(lam * (ga0 - Ga0));
    if (a == 0) {
        depth[node] = z0 + zsum;
        if (var) var[node] = fmaf(lam0, g00, g00 + vsum);
    }
}

template <int K, bool kWide>
__device__ __forceinline__ void okrige_patch(const HashView& h, const GridView& g, int k,
                                             const OkParams& p, float* __restrict__ depth,
                                             float* __restrict__ var, int32_t* __restrict__ nbr,
                                             int* __restrict__ flag, int px, int py, int* s_ids,
                                             int* s_keff, float* sL) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const NodeIdx nd = patch_node(px, py, warp, lane);
    int keff = -1;  // -1: this pass writes nothing for the node
    if (nd.i < g.nx && nd.j < g.ny) {
        const int qx = g.x0 + nd.i * g.cell + g.cell / 2;
        const int qy = g.y0 + nd.j * g.cell + g.cell / 2;
        uint64_t d2[K];
        int id[K];
        if (h.n_valid > 0) {
            const Bound b = knn_bound<K>(h, qx, qy);
            const bool fits = packed_fits(h, b.tau0);
            if (!kWide && !fits) {
                *flag = 1;
            } else if (!kWide || !fits) {
                keff = min(knn_scan<K, kWide>(h, qx, qy, b, d2, id), k);
#pragma unroll
                for (int i = 0; i < K; ++i) s_ids[lane * K + i] = i < keff ? id[i] : -1;
            }
        } else if (!kWide) {
            keff = 0;
        }
        if (keff >= 0 && nbr) {
            const int64_t node = (int64_t)nd.j * g.nx + nd.i;
            for (int i = 0; i < k; ++i) nbr[node * k + i] = i < keff ? s_ids[lane * K + i] : -1;
        }
    }
    s_keff[lane] = keff;
    __syncwarp();
    for (int t = 0; t < 32; ++t) {
        const int ke = s_keff[t];
        if (ke < 0) continue;
        const NodeIdx nt = patch_node(px, py, warp, t);
        const int64_t node = (int64_t)nt.j * g.nx + nt.i;
        if (ke == 0) {
            if (lane == 0) {
                depth[node] = __int_as_float(0x7fc00000);
                if (var) var[node] = __int_as_float(0x7fc00000);
            }
            continue;
        }
        const int qx = g.x0 + nt.i * g.cell + g.cell / 2;
        const int qy = g.y0 + nt.j * g.cell + g.cell / 2;
        solve_system<K>(h, p, qx, qy, s_ids + t * K, ke, sL, node, depth, var);
    }
    __syncwarp();
}

template <int K>
__global__ void __launch_bounds__(kWarps * 32) k_okrige(HashView h, GridView g, int k, OkParams p,
                                                        float* __restrict__ depth,
                                                        float* __restrict__ var,
                                                        int32_t* __restrict__ nbr,
                                                        int* __restrict__ flag) {
    __shared__ int s_ids[kWarps][32 * K];
    __shared__ int s_keff[kWarps][32];
    __shared__ float s_L[kWarps][K * (K + 1)];
    const int warp = threadIdx.x >> 5;
    const int gx = (g.nx + 15) / 16;
    okrige_patch<K, false>(h, g, k, p, depth, var, nbr, flag, blockIdx.x % gx, blockIdx.x / gx,
                           s_ids[warp], s_keff[warp], s_L[warp]);
}

template <int K>
__global__ void __launch_bounds__(kWarps * 32) k_okrige_wide(HashView h, GridView g, int k,
                                                             OkParams p, float* __restrict__ depth,
                                                             float* __restrict__ var,
                                                             int32_t* __restrict__ nbr,
                                                             int* __restrict__ flag) {
    if (*(volatile int*)flag == 0) return;
    __shared__ int s_ids[kWarps][32 * K];
    __shared__ int s_keff[kWarps][32];
    __shared__ float s_L[kWarps][K * (K + 1)];
    const int warp = threadIdx.x >> 5;
    const int gx = (g.nx + 15) / 16;
    const int64_t nb = (int64_t)gx * ((g.ny + 7) / 8);
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x)
        okrige_patch<K, true>(h, g, k, p, depth, var, nbr, flag, (int)(b % gx), (int)(b / gx),
                              s_ids[warp], s_keff[warp], s_L[warp]);
}

template <int K>
bg_status launch_k(const HashView& h, const GridView& g, int k, const OkParams& p, float* depth,
                   float* var, int32_t* nbr, int* d_flag, cudaStream_t st) {
    const int64_t nb = (int64_t)((g.nx + 15) / 16) * ((g.ny + 7) / 8);
    BG_CUDA(cudaMemsetAsync(d_flag, 0, sizeof(int), st));
    k_okrige<K><<<(unsigned)nb, kWarps * 32, 0, st>>>(h, g, k, p, depth, var, nbr, d_flag);
    k_okrige_wide<K><<<(unsigned)(nb < 152 * 4 ? nb : 152 * 4), kWarps * 32, 0, st>>>(
        h, g, k, p, depth, var, nbr, d_flag);
    note_launches(2);
    BG_CUDA(cudaGetLastError());
    return BG_OK;
}

}  // namespace

bg_status launch_okrige(const bg_soundings_s* s, const GridView& g, int k, const OkParams& p,
                        float* depth, float* var, int32_t* nbr, cudaStream_t st) {
    HashView h = s->h;
    const int K = k <= 8 ? 8 : k <= 16 ? 16 : 32;
    h.r0 = start_halfwidth(s, K);
    int* flag = nullptr;
    bg_status rc = dalloc(s->ctx, (void**)&flag, sizeof(int), st);
    if (rc != BG_OK) return rc;
    switch (K) {
        case 8: rc = launch_k<8>(h, g, k, p, depth, var, nbr, flag, st); break;
        case 16: rc = launch_k<16>(h, g, k, p, depth, var, nbr, flag, st); break;
        default: rc = launch_k<32>(h, g, k, p, depth, var, nbr, flag, st); break;
    }
    dfree(s->ctx, flag, sizeof(int), st);
    return rc;
}

}  // namespace bg
