// Local ordinary kriging (Sec. III-C) over the exact k nearest soundings.
//
// Two kernels per chunk of grid rows:
//   k_knn_ids<K>      one thread per node: exact k-NN (knn.cuh), writes the
//                     neighbours' upload indices (ascending) to an id buffer;
//   k_okrige_solve<K> G = K/4 threads per kriging system, 32/G systems per
//                     warp: each thread owns R = 4 rows of its system.
//
// The bordered variogram system [Gamma 1; 1^T 0][lambda; mu] = [gamma_0; 1]
// is reduced with sum(lambda) = 1 by eliminating lambda_0 (the nearest
// neighbour) and mu. For reduced rows r, c (neighbours r+1, c+1):
//     A[r][c] = Gamma_r0 + Gamma_c0 - Gamma_rc,   b_r = Gamma_r0 + gamma_00 - gamma_r0,
//     A lambda' = b,  lambda_0 = 1 - sum(lambda'),  mu = gamma_00 - sum_a Gamma_0a lambda_a.
// A is symmetric positive definite for a conditionally negative definite
// variogram (spherical and exponential are, in 2-D). It is factored by
// Cholesky in FP32 with the lower triangle in registers (thread t, slot s
// holds row G*s + t, columns 0 .. G*(s+1)-1); pivots and column entries move
// between the G threads of a system by warp shuffles. One refinement step
// follows: the residual b - A lambda' is accumulated from exact products
// (FMA error terms) and error-free sums as an FP32 double-word (about 48
// significant bits) against the original A kept in shared memory, and the
// correction reuses the factor. The weight sum closes in FP64:
// lambda_0 = 1 - sum(lambda'). Outputs:
//     zhat    = z_0 + sum_a lambda_a (z_a - z_0)          (= sum lambda_i z_i)
//     sigma^2 = lambda_0 gamma_00 + sum_a lambda_a gamma_a0 + mu.
// Rows beyond k_eff - 1 are identity rows with zero right-hand side, so every
// system has the fixed size K and all loops over rows and columns unroll.
#include <algorithm>
#include <cmath>
#include <utility>

#include "bg_internal.h"
#include "knn.cuh"

namespace bg {
namespace {

constexpr int kR = 4;            // rows per thread
constexpr int kSolveWarps = 2;   // warps per solve block
constexpr int kRounds = 8;       // system batches per warp

template <int K>
struct Geo {
    static constexpr int G = K / kR;                      // threads per system
    static constexpr int SYS = 32 / G;                    // systems per warp
    static constexpr int LEN = G * kR * (kR + 1) / 2;     // register floats of L
    static constexpr int ROW = K + 1;                     // smem row stride of A
    // per-system smem floats, padded to G (mod 32) so that the systems of a
    // warp read distinct banks
    static constexpr int MAT = K * ROW + ((G - (K * ROW) % 32) + 32) % 32;
    static constexpr int TAB = K + 1;                     // neighbour table stride
    static constexpr int WARP_FLOATS = SYS * (MAT + 4 * TAB);
    static __host__ __device__ constexpr int off(int s) { return G * s * (s + 1) / 2; }
};

__device__ __forceinline__ float variogram(const OkParams& p, float h_m) {
    if (p.model == BG_VARIOGRAM_SPHERICAL) {
        const float t = h_m * p.inv_a;
        if (t >= 1.0f) return p.sill;
        return fmaf(p.c * t, fmaf(-0.5f * t, t, 1.5f), p.c0);
    }
    return fmaf(p.c, 1.0f - __expf(-h_m * p.inv_a), p.c0);
}

// gamma from a separation in cm; zero separation gives `at_zero`
__device__ __forceinline__ float gamma_cm(const OkParams& p, int dx, int dy, float at_zero) {
    if ((dx | dy) == 0) return at_zero;
    const float fx = (float)dx, fy = (float)dy;
    const float d2 = fmaf(fx, fx, fy * fy);
    return variogram(p, d2 * rsqrtf(d2) * 0.01f);
}

// ------------------------------------------------------------ k-NN -> ids

template <int K, bool kWide>
__device__ __forceinline__ void knn_ids_node(const HashView& h, const GridView& g, int k,
                                             int64_t node0, int32_t* __restrict__ ids,
                                             int* __restrict__ flag, NodeIdx nd, int j1) {
    if (nd.i >= g.nx || nd.j >= j1) return;
    const int64_t node = (int64_t)nd.j * g.nx + nd.i;
    const int qx = g.x0 + nd.i * g.cell + g.cell / 2;
    const int qy = g.y0 + nd.j * g.cell + g.cell / 2;
    uint64_t d2[K];
    int id[K];
    int keff = 0;
    if (h.n_valid > 0) {
        const Bound b = knn_bound<K>(h, qx, qy);
        const bool fits = packed_fits(h, b.tau0);
        if (kWide) {
            if (fits) return;
        } else if (!fits) {
            *flag = 1;
            return;
        }
        keff = knn_scan<K, kWide>(h, qx, qy, b, d2, id);
    } else if (kWide) {
        return;
    }
    int32_t* o = ids + (node - node0) * k;
#pragma unroll
    for (int i = 0; i < K; ++i)
        if (i < k) o[i] = i < keff ? id[i] : -1;
}

// grid rows [j0, j1); j0 is a multiple of 8
template <int K>
__global__ void __launch_bounds__(128) k_knn_ids(HashView h, GridView g, int k, int j0, int j1,
                                                 int32_t* __restrict__ ids, int* __restrict__ flag) {
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int gx = (g.nx + 15) / 16;
    const int px = blockIdx.x % gx, py = j0 / 8 + blockIdx.x / gx;
    knn_ids_node<K, false>(h, g, k, (int64_t)j0 * g.nx, ids, flag,
                           patch_node(px, py, warp, lane), j1);
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
                              patch_node((int)(b % gx), j0 / 8 + (int)(b / gx), warp, lane), j1);
}

// ---------------------------------------------------------------- solve

// error-free transformation: a + b = s + e exactly
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
    s = a + b;
    const float bb = s - a;
    e = (a - (s - bb)) + (b - bb);
}

// The factor and solve sweeps below are written as one function per column
// j, expanded over j = 0..K-1 with an integer_sequence, so that every index
// into the register arrays is a compile-time constant (a plain nested
// #pragma unroll over the triangle is too large for the unroller, which then
// leaves the arrays in local memory).

// Cholesky column j: scale by the pivot, then update the trailing rows with
// column j broadcast within the group.
template <int K, int J>
__device__ __forceinline__ void chol_column(float (&L)[Geo<K>::LEN], float (&dinv)[kR], int t,
                                            int gbase) {
    using Gm = Geo<K>;
    constexpr int G = Gm::G;
    constexpr int SJ = J / G;
    const float d = __shfl_sync(kFull, L[Gm::off(SJ) + J], gbase + J % G);
    const float inv = rsqrtf(d);
#pragma unroll
    for (int s = 0; s < kR; ++s) {
        if (G * (s + 1) - 1 >= J) {
            const int r = G * s + t;
            if (r > J) L[Gm::off(s) + J] *= inv;
            if (r == J) {
                L[Gm::off(s) + J] = d * inv;
                dinv[s] = inv;
            }
        }
    }
#pragma unroll
    for (int c = J + 1; c < K; ++c) {
        const float lcj = __shfl_sync(kFull, L[Gm::off(c / G) + J], gbase + c % G);
#pragma unroll
        for (int s = 0; s < kR; ++s)
            if (G * (s + 1) - 1 >= c) L[Gm::off(s) + c] = fmaf(-L[Gm::off(s) + J], lcj, L[Gm::off(s) + c]);
    }
}

template <int K, int... J>
__device__ __forceinline__ void chol_factor(float (&L)[Geo<K>::LEN], float (&dinv)[kR], int t,
                                            int gbase, std::integer_sequence<int, J...>) {
    (chol_column<K, J>(L, dinv, t, gbase), ...);
}

// forward sweep step j of L y = v
template <int K, int J>
__device__ __forceinline__ void fwd_step(const float (&L)[Geo<K>::LEN], const float (&dinv)[kR],
                                         float (&v)[kR], int t, int gbase) {
    using Gm = Geo<K>;
    constexpr int G = Gm::G;
    constexpr int SJ = J / G;
    if (t == J % G) v[SJ] *= dinv[SJ];
    const float yj = __shfl_sync(kFull, v[SJ], gbase + J % G);
#pragma unroll
    for (int s = 0; s < kR; ++s)
        if (G * (s + 1) - 1 > J && G * s + t > J) v[s] = fmaf(-L[Gm::off(s) + J], yj, v[s]);
}

// transposed sweep step for column j = K-1-I of L^T x = y
template <int K, int I>
__device__ __forceinline__ void bwd_step(const float (&L)[Geo<K>::LEN], const float (&dinv)[kR],
                                         float (&v)[kR], int t) {
    using Gm = Geo<K>;
    constexpr int G = Gm::G;
    constexpr int J = K - 1 - I;
    constexpr int SJ = J / G;
    float q = 0.0f;
#pragma unroll
    for (int s = 0; s < kR; ++s)
        if (G * (s + 1) - 1 > J && G * s + t > J) q = fmaf(L[Gm::off(s) + J], v[s], q);
#pragma unroll
    for (int o = 1; o < G; o <<= 1) q += __shfl_xor_sync(kFull, q, o);
    if (t == J % G) v[SJ] = (v[SJ] - q) * dinv[SJ];
}

// L L^T v = v in place for the system of this thread's group.
template <int K, int... J>
__device__ __forceinline__ void chol_solve_seq(const float (&L)[Geo<K>::LEN],
                                               const float (&dinv)[kR], float (&v)[kR], int t,
                                               int gbase, std::integer_sequence<int, J...>) {
    (fwd_step<K, J>(L, dinv, v, t, gbase), ...);
    (bwd_step<K, J>(L, dinv, v, t), ...);
}

template <int K>
__device__ __forceinline__ void chol_solve(const float (&L)[Geo<K>::LEN], const float (&dinv)[kR],
                                           float (&v)[kR], int t, int gbase) {
    chol_solve_seq<K>(L, dinv, v, t, gbase, std::make_integer_sequence<int, K>{});
}

template <int K>
__global__ void __launch_bounds__(kSolveWarps * 32) k_okrige_solve(
    HashView h, GridView g, int k, OkParams p, int64_t node0, int64_t nodes,
    const int32_t* __restrict__ ids, float* __restrict__ depth, float* __restrict__ var) {
    using Gm = Geo<K>;
    constexpr int G = Gm::G;
    __shared__ float smem[kSolveWarps * Gm::WARP_FLOATS];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G, t = lane % G, gbase = grp * G;
    float* A0 = smem + warp * Gm::WARP_FLOATS + grp * Gm::MAT;
    float* tabs = smem + warp * Gm::WARP_FLOATS + Gm::SYS * Gm::MAT;
    int* tx = reinterpret_cast<int*>(tabs) + grp * Gm::TAB;                 // x of neighbour n
    int* ty = reinterpret_cast<int*>(tabs) + (Gm::SYS + grp) * Gm::TAB;     // y of neighbour n
    float* tz = tabs + (2 * Gm::SYS + grp) * Gm::TAB;                       // depth of neighbour 0
    float* tg = tabs + (3 * Gm::SYS + grp) * Gm::TAB;                       // Gamma(row r, 0)
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << gbase);

    for (int round = 0; round < kRounds; ++round) {
        const int64_t sys = ((int64_t)blockIdx.x * kSolveWarps + warp) * (Gm::SYS * kRounds) +
                            (int64_t)round * Gm::SYS + grp;
        const bool live = sys < nodes;  // uniform within a group
        const int64_t node = node0 + (live ? sys : 0);
        const int32_t* my = ids + (live ? sys : 0) * k;

        // neighbour ids of my rows (reduced row r <-> neighbour r + 1) and k_eff;
        // ids are -1 exactly past k_eff
        int nid[kR];
        unsigned cnt = 0;
#pragma unroll
        for (int s = 0; s < kR; ++s) {
            const int n = 1 + G * s + t;
            nid[s] = (live && n < k) ? __ldg(my + n) : -1;
            cnt += __popc(__ballot_sync(kFull, nid[s] >= 0) & gmask);
        }
        const int id0 = live ? __ldg(my) : -1;
        const int ke = (id0 >= 0) ? 1 + (int)cnt : 0;  // 0: no output (empty or past the end)
        const int qx = g.x0 + (int)(node % g.nx) * g.cell + g.cell / 2;
        const int qy = g.y0 + (int)(node / g.nx) * g.cell + g.cell / 2;

        // gather the neighbours' records into the system's table
        float zr[kR];
        if (t == 0) {
            int4 r0 = make_int4(0, 0, 0, 0);
            if (id0 >= 0) r0 = __ldg(h.orig + id0);
            tx[0] = r0.x;
            ty[0] = r0.y;
            tz[0] = __int_as_float(r0.z);
        }
#pragma unroll
        for (int s = 0; s < kR; ++s) {
            int4 rr = make_int4(0, 0, 0, 0);
            if (nid[s] >= 0) rr = __ldg(h.orig + nid[s]);
            const int n = 1 + G * s + t;  // <= K = TAB - 1
            tx[n] = rr.x;
            ty[n] = rr.y;
            zr[s] = __int_as_float(rr.z);
        }
        __syncwarp();
        const int x0 = tx[0], y0 = ty[0];
        const float z0 = tz[0];
        const float g00 = gamma_cm(p, x0 - qx, y0 - qy, 0.0f);
        float gr0[kR], g0r[kR];  // Gamma(neighbour of row, neighbour 0), gamma(node, that neighbour)
#pragma unroll
        for (int s = 0; s < kR; ++s) {
            const int n = 1 + G * s + t;
            const bool real = n < ke;
            gr0[s] = real ? gamma_cm(p, tx[n] - x0, ty[n] - y0, p.c0) : 0.0f;
            g0r[s] = real ? gamma_cm(p, tx[n] - qx, ty[n] - qy, 0.0f) : 0.0f;
            tg[G * s + t] = gr0[s];
        }
        __syncwarp();

        // assemble: lower triangle into registers, the full symmetric matrix into smem
        float L[Gm::LEN];
        float b[kR];
#pragma unroll
        for (int s = 0; s < kR; ++s) {
            const int r = G * s + t;
            const bool row = r + 1 < ke;
            const int xr = tx[r + 1], yr = ty[r + 1];
            b[s] = row ? (gr0[s] + g00) - g0r[s] : 0.0f;
#pragma unroll
            for (int c = 0; c < G * (s + 1); ++c) {
                float v;
                if (c < r) {
                    v = (row && c + 1 < ke)
                            ? (gr0[s] + tg[c]) - gamma_cm(p, xr - tx[c + 1], yr - ty[c + 1], p.c0)
                            : 0.0f;
                } else if (c == r) {
                    v = row ? 2.0f * gr0[s] : 1.0f;
                } else {
                    v = 0.0f;  // unused upper part
                }
                L[Gm::off(s) + c] = v;
                if (c <= r) {
                    A0[r * Gm::ROW + c] = v;
                    A0[c * Gm::ROW + r] = v;
                }
            }
        }

        // Cholesky in registers
        float dinv[kR];
#pragma unroll
        for (int s = 0; s < kR; ++s) dinv[s] = 1.0f;
        chol_factor<K>(L, dinv, t, gbase, std::make_integer_sequence<int, K>{});
        __syncwarp();

        float x[kR];
#pragma unroll
        for (int s = 0; s < kR; ++s) x[s] = b[s];
        chol_solve<K>(L, dinv, x, t, gbase);

        // residual b - A x against the original A, as an FP32 double-word:
        // exact products (FMA error term) and error-free running sums
        float rh[kR], rl[kR];
#pragma unroll
        for (int s = 0; s < kR; ++s) {
            rh[s] = b[s];
            rl[s] = 0.0f;
        }
#pragma unroll
        for (int sc = 0; sc < kR; ++sc) {
#pragma unroll 2
            for (int tc = 0; tc < G; ++tc) {
                const int c = G * sc + tc;
                const float xc = __shfl_sync(kFull, x[sc], gbase + tc);
#pragma unroll
                for (int s = 0; s < kR; ++s) {
                    const float a = A0[(G * s + t) * Gm::ROW + c];
                    const float ph = -a * xc;
                    const float pl = fmaf(-a, xc, -ph);
                    float sh, se;
                    two_sum(rh[s], ph, sh, se);
                    rh[s] = sh;
                    rl[s] += se + pl;
                }
            }
        }
        float dx[kR];
#pragma unroll
        for (int s = 0; s < kR; ++s) dx[s] = rh[s] + rl[s];
        chol_solve<K>(L, dinv, dx, t, gbase);
#pragma unroll
        for (int s = 0; s < kR; ++s) x[s] += dx[s];

        // weights and outputs; the weight sum closes in FP64
        float ps = 0.0f, pz = 0.0f, pv = 0.0f;
#pragma unroll
        for (int s = 0; s < kR; ++s) {
            const bool row = G * s + t + 1 < ke;
            const float lam = row ? x[s] : 0.0f;
            ps += lam;
            pz = fmaf(lam, zr[s] - z0, pz);
            pv = fmaf(lam, g0r[s] - gr0[s], pv);
        }
        double wsum = (double)ps;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) {
            wsum += __shfl_xor_sync(kFull, wsum, o);
            pz += __shfl_xor_sync(kFull, pz, o);
            pv += __shfl_xor_sync(kFull, pv, o);
        }
        const float lam0 = (float)(1.0 - wsum);
        if (live && t == 0) {
            if (ke == 0) {
                depth[node] = __int_as_float(0x7fc00000);  // no valid sounding
                if (var) var[node] = __int_as_float(0x7fc00000);
            } else {
                depth[node] = z0 + pz;
                if (var) var[node] = fmaf(lam0, g00, g00 + pv);
            }
        }
        __syncwarp();
    }
}

template <int K>
bg_status launch_k(const HashView& h, const GridView& g, int k, const OkParams& p, float* depth,
                   float* var, int32_t* nbr, bg_ctx_s* ctx, cudaStream_t st) {
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
    const int64_t sys_per_block = (int64_t)kSolveWarps * Gm::SYS * kRounds;
    for (int64_t j0 = 0; j0 < g.ny; j0 += rows) {
        const int64_t j1 = std::min<int64_t>(g.ny, j0 + rows);
        const int64_t nb = (int64_t)gx * ((j1 - j0 + 7) / 8);
        int32_t* chunk_ids = nbr ? nbr + j0 * g.nx * k : (int32_t*)((char*)scratch + flag_bytes);
        cudaError_t e = cudaMemsetAsync(flag, 0, sizeof(int), st);
        if (e != cudaSuccess) {
            rc = cuda_fail(e, "memset");
            break;
        }
        k_knn_ids<K><<<(unsigned)nb, 128, 0, st>>>(h, g, k, (int)j0, (int)j1, chunk_ids, flag);
        k_knn_ids_wide<K><<<(unsigned)std::min<int64_t>(nb, 152 * 4), 128, 0, st>>>(
            h, g, k, (int)j0, (int)j1, chunk_ids, flag);
        const int64_t nodes = (j1 - j0) * g.nx;
        const int64_t sb = (nodes + sys_per_block - 1) / sys_per_block;
        k_okrige_solve<K><<<(unsigned)sb, kSolveWarps * 32, 0, st>>>(h, g, k, p, j0 * g.nx, nodes,
                                                                     chunk_ids, depth, var);
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

bg_status launch_okrige(const bg_soundings_s* s, const GridView& g, int k, const OkParams& p,
                        float* depth, float* var, int32_t* nbr, cudaStream_t st) {
    HashView h = s->h;
    const int K = k <= 4 ? 4 : k <= 8 ? 8 : k <= 16 ? 16 : 32;
    h.r0 = start_halfwidth(s, K);
    switch (K) {
        case 4: return launch_k<4>(h, g, k, p, depth, var, nbr, s->ctx, st);
        case 8: return launch_k<8>(h, g, k, p, depth, var, nbr, s->ctx, st);
        case 16: return launch_k<16>(h, g, k, p, depth, var, nbr, s->ctx, st);
        default: return launch_k<32>(h, g, k, p, depth, var, nbr, s->ctx, st);
    }
}

}  // namespace bg
