// Device code of local ordinary kriging (Sec. III-C) over the exact k nearest
// soundings, shared by the per-grid kernels (okrige.cu) and the batched
// persistent kernels (batch.cu).
//
// Per grid node: exact k-NN to neighbour ids (knn_ids_node, one thread per
// node); then the kriging system, solved by G = K/4 threads that each own
// R = 4 rows, so a warp solves 32/G systems at once (okrige_solve_block).
//
// The bordered variogram system [Gamma 1; 1^T 0][lambda; mu] = [gamma_0; 1]
// is reduced with sum(lambda) = 1 by eliminating lambda_0 (the nearest
// neighbour) and mu. For reduced rows r, c (neighbours r+1, c+1):
//     A[r][c] = Gamma_r0 + Gamma_c0 - Gamma_rc,   b_r = Gamma_r0 + gamma_00 - gamma_r0,
//     A lambda' = b,  lambda_0 = 1 - sum(lambda'),  mu = gamma_00 - sum_a Gamma_0a lambda_a.
// A is symmetric positive definite for a conditionally negative definite
// variogram (spherical and exponential are, in 2-D), so |A[r][c]| is bounded
// by its largest diagonal entry. It is assembled once per entry straight into
// a 30-bit fixed-point copy in shared memory (packed lower triangle), factored
// by Cholesky in FP32 with each thread's rows in registers (thread t, slot s
// holds row G*s + t, columns 0 .. G*(s+1)-1; pivots move between the G
// threads by warp shuffles, column entries through a small column buffer in
// shared memory). The back sweeps also run on the register rows, one column at
// a time with a group sum (no transposed copy of the factor), so shared
// memory per system stays near 2.8 KB (K = 32) and,
// with the registers held to 128, a GB300 SM keeps 16 warps resident. One
// step of iterative refinement follows: x is rounded to 24-bit fixed point x'
// (exact in FP32), the residual b - A' x' is accumulated exactly in 64-bit
// integers, and the correction reuses the factor. The weight sum closes in FP64:
// lambda_0 = 1 - sum(lambda'). Outputs:
//     zhat    = z_0 + sum_a lambda_a (z_a - z_0)          (= sum lambda_i z_i)
//     sigma^2 = lambda_0 gamma_00 + sum_a lambda_a gamma_a0 + mu.
// Rows beyond k_eff - 1 are identity rows with zero right-hand side, so every
// system has the fixed size K and all loops over rows and columns unroll.
// Much of the FP32 work runs as packed two-lane instructions (add/sub/mul/fma
// .rn.f32x2: one instruction, two IEEE single operations, each lane rounded
// as its scalar form): the variogram assembly two rows at a time, the per-row
// variograms of the prologue, and column pairs of the Cholesky update. The
// solve is issue- and latency-bound, so halving those instructions pays, and
// the results are bitwise those of the scalar code.
#pragma once

#include <algorithm>
#include <cmath>
#include <utility>

#include "bg_internal.h"
#include "idw_dev.cuh"
#include "knn.cuh"

namespace bg {


constexpr int kR = 4;            // rows per thread
constexpr int kRounds = 1;       // system batches per warp (one: more, shorter blocks balance best)
constexpr int kBwdLook = 2;      // back-sweep pipeline depth (see bwd_step)
// The grid and point-list solve kernels run 8-warp blocks, 2 per SM (the same
// 16 warps): with the unrolled solve's long instruction stream, two blocks in
// different phases fetch far fewer distinct instructions than four.
constexpr int kGridSolveWarps = 8;
constexpr int kGridSolveBlocksPerSM = 2;
// solve blocks ahead whose neighbour ids a block prefetches into L2: two
// waves of the 152 SMs (one to eight waves measured the same)
constexpr int kIdsPrefetchBlocks = 2 * 152 * kGridSolveBlocksPerSM;

template <int K>
struct Geo {
    static constexpr int G = K / kR;                      // threads per system
    static constexpr int SYS = 32 / G;                    // systems per warp
    static constexpr int LEN = G * kR * (kR + 1) / 2;     // register floats of L
    static constexpr int TRI = K * (K + 1) / 2;           // packed lower triangle of A
    static constexpr int TRIP = (TRI + 3) / 4 * 4;        // the triangle padded to 16 bytes
    // per system: the fixed-point A as a packed lower triangle (row r at
    // r (r + 1) / 2), the rows' records (three arrays of K floats: x, y,
    // Gamma_r0, in a region of 4 K), and two column buffers for the Cholesky
    // broadcasts (16-byte aligned); the stride is = G (mod 32) so that the
    // G-thread groups of a warp spread over the banks
    static constexpr int CB = TRIP + 4 * K;
    static constexpr int RAW = CB + 2 * K;
    static constexpr int SYS_FLOATS = RAW + ((G - RAW % 32) + 32) % 32;
    static constexpr int WARP_FLOATS = SYS * SYS_FLOATS;
    static __host__ __device__ constexpr int off(int s) { return G * s * (s + 1) / 2; }
};

__device__ __forceinline__ float variogram(const OkParams& p, float h_m) {
    if (p.model == BG_VARIOGRAM_SPHERICAL) {
        const float t = h_m * p.inv_a;
        if (t >= 1.0f) return p.sill;
        return fmaf(p.c * t, fmaf(-0.5f * t, t, 1.5f), p.c0);
    }
    // 1 - exp(-t) as -expm1(-t): no cancellation at short range, where the
    // model without a nugget makes the kriging variance small
    return fmaf(p.c, -expm1f(-h_m * p.inv_a), p.c0);
}

// gamma from a separation in cm; zero separation gives `at_zero`
__device__ __forceinline__ float gamma_cm(const OkParams& p, int dx, int dy, float at_zero) {
    if ((dx | dy) == 0) return at_zero;
    const float fx = (float)dx, fy = (float)dy;
    const float d2 = fmaf(fx, fx, fy * fy);
    return variogram(p, d2 * rsqrtf(d2) * 0.01f);
}

// gamma between two distinct soundings from float offsets in cm (exact
// integers below 2^24); zero separation gives the nugget c0 (the h -> 0+
// limit) without a branch: t = min(h/a, 1) makes the spherical model's
// polynomial equal the sill beyond the range
__device__ __forceinline__ float gamma_pair_f(const OkParams& p, float dx, float dy) {
    const float d2 = fmaf(dx, dx, dy * dy);
    const float h_cm = d2 * rsqrtf(d2 + 1e-30f);
    if (p.model == BG_VARIOGRAM_SPHERICAL) {
        const float t = fminf(h_cm * p.inv_a * 0.01f, 1.0f);
        return fmaf(p.c * t, fmaf(-0.5f * t, t, 1.5f), p.c0);
    }
    return fmaf(p.c, -expm1f(-h_cm * p.inv_a * 0.01f), p.c0);
}

// one hardware square-root approximation (sqrt.approx.f32: a few ulp, 0 at 0)
__device__ __forceinline__ float sqrt_approx(float x) {
    float y;
    asm("sqrt.approx.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// The variogram of the assembly in the fixed-point scale of the system: with
// the scale sa a power of two, sa gamma(h) is the model with c0 and c scaled
// by sa. t^2 = d2 (1/a)^2 from the exact squared separation in cm^2.
struct ScaledVgm {
    float kinv2;  // (0.01 / a)^2: cm^2 -> (h / a)^2
    float c0s;    // sa c0
    float cs;     // sa c
    float k2, k3; // spherical: -0.5 sa c, 1.5 sa c
};

__device__ __forceinline__ ScaledVgm scaled_vgm(const OkParams& p, float sa) {
    const float kinv = p.inv_a * 0.01f;
    const float cs = p.c * sa;
    return ScaledVgm{kinv * kinv, p.c0 * sa, cs, -0.5f * cs, 1.5f * cs};
}

template <bool kSpherical>
__device__ __forceinline__ float gamma_pair_scaled(const ScaledVgm& v, float dx, float dy) {
    const float t2 = fmaf(dx, dx, dy * dy) * v.kinv2;
    if constexpr (kSpherical) {
        const float t = fminf(sqrt_approx(t2), 1.0f);  // the polynomial is the sill at t = 1
        return fmaf(t, fmaf(v.k2, t * t, v.k3), v.c0s);
    } else {
        return fmaf(v.cs, -expm1f(-sqrt_approx(t2)), v.c0s);
    }
}

// Packed two-lane FP32 arithmetic (one instruction for two IEEE single
// operations, each lane rounded as its scalar counterpart): two floats in one
// 64-bit register pair.
__device__ __forceinline__ unsigned long long pk2(float a, float b) {
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
    return r;
}
__device__ __forceinline__ void upk2(unsigned long long p, float& a, float& b) {
    asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(p));
}
__device__ __forceinline__ unsigned long long add2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b,
                                                   unsigned long long c) {
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}

// Two assembly entries of one column (x0, y0, gcc) from rows a and b at once,
// in the fixed-point scale, spherical model: each lane takes exactly the
// operations of (z + gcc) - gamma_pair_scaled<true>(sv, x - x0, y - y0).
__device__ __forceinline__ void gamma_rows2_sph(const ScaledVgm& v, float xa, float xb, float ya,
                                                float yb, float za, float zb, float x0, float y0,
                                                float gcc, float& oa, float& ob) {
    const unsigned long long dx = sub2(pk2(xa, xb), pk2(x0, x0));
    const unsigned long long dy = sub2(pk2(ya, yb), pk2(y0, y0));
    const unsigned long long t2 = mul2(fma2(dx, dx, mul2(dy, dy)), pk2(v.kinv2, v.kinv2));
    float ta, tb;
    upk2(t2, ta, tb);
    ta = fminf(sqrt_approx(ta), 1.0f);  // the polynomial is the sill at t = 1
    tb = fminf(sqrt_approx(tb), 1.0f);
    const unsigned long long t = pk2(ta, tb);
    const unsigned long long gm = fma2(t, fma2(pk2(v.k2, v.k2), mul2(t, t), pk2(v.k3, v.k3)),
                                       pk2(v.c0s, v.c0s));
    upk2(sub2(add2(pk2(za, zb), pk2(gcc, gcc)), gm), oa, ob);
}

// gamma_pair_f, spherical model, for two rows at once (packed FP32, each lane
// the scalar operations in the same order)
__device__ __forceinline__ void gamma_pair_sph2(const OkParams& p, float dxa, float dya, float dxb,
                                                float dyb, float& ga, float& gb) {
    const unsigned long long dx = pk2(dxa, dxb), dy = pk2(dya, dyb);
    const unsigned long long d2 = fma2(dx, dx, mul2(dy, dy));
    float ea, eb;
    upk2(add2(d2, pk2(1e-30f, 1e-30f)), ea, eb);
    const unsigned long long h = mul2(d2, pk2(rsqrtf(ea), rsqrtf(eb)));
    float ta, tb;
    upk2(mul2(mul2(h, pk2(p.inv_a, p.inv_a)), pk2(0.01f, 0.01f)), ta, tb);
    const unsigned long long t = pk2(fminf(ta, 1.0f), fminf(tb, 1.0f));
    const unsigned long long in = fma2(mul2(pk2(-0.5f, -0.5f), t), t, pk2(1.5f, 1.5f));
    upk2(fma2(mul2(pk2(p.c, p.c), t), in, pk2(p.c0, p.c0)), ga, gb);
}

// gamma_cm (zero separation gives 0), spherical model, for two rows at once
__device__ __forceinline__ void gamma_cm_sph2(const OkParams& p, int dxa, int dya, int dxb, int dyb,
                                              float& ga, float& gb) {
    const unsigned long long fx = pk2((float)dxa, (float)dxb), fy = pk2((float)dya, (float)dyb);
    const unsigned long long d2 = fma2(fx, fx, mul2(fy, fy));
    float da, db;
    upk2(d2, da, db);
    float ta, tb;
    upk2(mul2(mul2(mul2(d2, pk2(rsqrtf(da), rsqrtf(db))), pk2(0.01f, 0.01f)), pk2(p.inv_a, p.inv_a)),
         ta, tb);
    const unsigned long long t = pk2(ta, tb);
    const unsigned long long in = fma2(mul2(pk2(-0.5f, -0.5f), t), t, pk2(1.5f, 1.5f));
    float va, vb;
    upk2(fma2(mul2(pk2(p.c, p.c), t), in, pk2(p.c0, p.c0)), va, vb);
    ga = ((dxa | dya) == 0) ? 0.0f : (ta >= 1.0f ? p.sill : va);
    gb = ((dxb | dyb) == 0) ? 0.0f : (tb >= 1.0f ? p.sill : vb);
}

// ------------------------------------------------------------ k-NN -> ids

template <int K, bool kWide>
__device__ __forceinline__ void knn_ids_node(const HashView& h, const GridView& g, int k,
                                             int64_t node0, int32_t* __restrict__ ids,
                                             int* __restrict__ flag, NodeIdx nd, int j1,
                                             uint64_t* hp) {
    if (nd.i >= g.nx || nd.j >= j1) return;
    const int64_t node = (int64_t)nd.j * g.nx + nd.i;
    const int qx = g.x0 + nd.i * g.cell + g.cell / 2;
    const int qy = g.y0 + nd.j * g.cell + g.cell / 2;
    int32_t* o = ids + (node - node0) * k;
    if (h.n_valid == 0) {
        if (!kWide)
            for (int i = 0; i < k; ++i) o[i] = -1;
        return;
    }
    const Bound b = knn_bound<K>(h, qx, qy);
    const bool fits = packed_fits(h, b.tau0);
    if constexpr (kWide) {
        if (fits) return;
        uint64_t d2[K];
        int id[K];
        const int keff = knn_scan<K, true>(h, qx, qy, b, d2, id);
#pragma unroll
        for (int i = 0; i < K; ++i)
            if (i < k) o[i] = i < keff ? id[i] : -1;
    } else {
        if (!fits) {
            *flag = 1;
            return;
        }
        const int keff = knn_scan_heap<K, 128>(h, qx, qy, b, hp);
        const uint64_t mask = (1ull << h.idx_bits) - 1;
        for (int i = 0; i < k; ++i) o[i] = i < keff ? (int)(hp[i * 128] & mask) : -1;
    }
}

// Wide-key neighbour ids of one query point whose table bound does not fit
// the packed key; other points return.
template <int K>
__device__ __forceinline__ void knn_ids_point_wide(const HashView& h, int qx, int qy, int k,
                                                   int32_t* __restrict__ o) {
    if (h.n_valid == 0 || !query_in_range(qx, qy)) return;
    const Bound b = knn_bound<K>(h, qx, qy);
    if (packed_fits(h, b.tau0)) return;
    uint64_t d2[K];
    int id[K];
    const int keff = knn_scan<K, true>(h, qx, qy, b, d2, id);
#pragma unroll
    for (int i = 0; i < K; ++i)
        if (i < k) o[i] = i < keff ? id[i] : -1;
}

// ---------------------------------------------------------------- solve

__host__ __device__ constexpr int tri(int r) { return r * (r + 1) / 2; }

// d0 += a * b0, d1 += a * b1 in one packed two-lane FMA (each lane a correctly
// rounded fused multiply-add, so the results equal two fmaf calls)
__device__ __forceinline__ void ffma2(float& d0, float& d1, float a, float b0, float b1) {
    asm("{\n\t.reg .b64 d, a, b;\n\t"
        "mov.b64 d, {%0, %1};\n\t"
        "mov.b64 a, {%2, %2};\n\t"
        "mov.b64 b, {%3, %4};\n\t"
        "fma.rn.f32x2 d, a, b, d;\n\t"
        "mov.b64 {%0, %1}, d;\n\t}"
        : "+f"(d0), "+f"(d1)
        : "f"(a), "f"(b0), "f"(b1));
}

// Cholesky column j of the register-held lower triangle: scale by the pivot
// (one shuffle), then update the trailing rows with column j. Each thread
// publishes its four entries of the column with one 16-byte store to a
// column buffer and reads the group's entries back four rows per 16-byte
// load (broadcast): fewer instructions than one shuffle per row. Two buffers
// alternate by column, so one __syncwarp per column orders writes and reads.
// A thread's columns c and c + G of one row take the same multiplier, and
// the loaded rows c and c + G sit side by side in the 16-byte load: those two
// updates go in one packed two-lane FMA (ffma2).
// Expanded over j with an integer_sequence so every register index is a
// compile-time constant (a nested #pragma unroll over the whole triangle is
// beyond the unroller and would leave L in local memory).
template <int K, int J>
__device__ __forceinline__ void chol_column(float (&L)[Geo<K>::LEN], float (&dinv)[kR], int t,
                                            int gbase, float* cb) {
    using Gm = Geo<K>;
    constexpr int G = Gm::G;
    constexpr int SJ = J / G;
    const float d = __shfl_sync(kFull, L[Gm::off(SJ) + J], gbase + J % G);
    const float inv = rsqrtf(d);
    float pub[kR];
#pragma unroll
    for (int s = 0; s < kR; ++s) {
        pub[s] = 0.0f;
        if (G * (s + 1) - 1 >= J) {
            const int r = G * s + t;
            if (r > J) L[Gm::off(s) + J] *= inv;
            if (r == J) {
                L[Gm::off(s) + J] = d * inv;
                dinv[s] = inv;
            }
            pub[s] = L[Gm::off(s) + J];
        }
    }
    if constexpr (G >= 4) {
        // 16-byte aligned only when the per-system stride (= G mod 32) is a
        // multiple of 4 floats
        static_assert(kR == 4 && Gm::SYS_FLOATS % 4 == 0 && Gm::CB % 4 == 0, "float4 buffer");
        float* col = cb + (J & 1) * K;
        *reinterpret_cast<float4*>(col + 4 * t) = make_float4(pub[0], pub[1], pub[2], pub[3]);
        __syncwarp();
#pragma unroll
        for (int tc = 0; tc < G; ++tc) {
            if (G * (kR - 1) + tc <= J) continue;  // no row of this thread beyond J
            const float4 q4 = *reinterpret_cast<const float4*>(col + 4 * tc);
            const float q[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
            for (int s = 0; s < kR; ++s) {
                if (G * (s + 1) - 1 <= J) continue;  // slot s holds no column beyond J
                const float a = -L[Gm::off(s) + J];
#pragma unroll
                for (int p = 0; p < kR / 2; ++p) {
                    const int c1 = G * (2 * p) + tc, c2 = c1 + G;
                    const bool in1 = 2 * p <= s && c1 > J, in2 = 2 * p + 1 <= s && c2 > J;
                    if (in1 && in2) {
                        ffma2(L[Gm::off(s) + c1], L[Gm::off(s) + c2], a, q[2 * p], q[2 * p + 1]);
                    } else {
                        if (in1) L[Gm::off(s) + c1] = fmaf(a, q[2 * p], L[Gm::off(s) + c1]);
                        if (in2) L[Gm::off(s) + c2] = fmaf(a, q[2 * p + 1], L[Gm::off(s) + c2]);
                    }
                }
            }
        }
    } else {
        // small systems (G < 4): one shuffle per trailing row
#pragma unroll
        for (int c = J + 1; c < K; ++c) {
            const float lcj = __shfl_sync(kFull, L[Gm::off(c / G) + J], gbase + c % G);
#pragma unroll
            for (int s = 0; s < kR; ++s)
                if (G * (s + 1) - 1 >= c)
                    L[Gm::off(s) + c] = fmaf(-L[Gm::off(s) + J], lcj, L[Gm::off(s) + c]);
        }
    }
}

// The factorization also runs the first solve's forward sweep: column J's
// step of L y = v right after column J is final, the same operations in the
// same order as the separate sweep, in the latency gaps of the factorization.
template <int K, int J>
__device__ __forceinline__ void fwd_step(const float (&L)[Geo<K>::LEN], const float (&dinv)[kR],
                                         float (&v)[kR], int t, int gbase);

template <int K, int... J>
__device__ __forceinline__ void chol_factor(float (&L)[Geo<K>::LEN], float (&dinv)[kR], int t,
                                            int gbase, float* cb, float (&v)[kR],
                                            std::integer_sequence<int, J...>) {
    ((chol_column<K, J>(L, dinv, t, gbase, cb), fwd_step<K, J>(L, dinv, v, t, gbase)), ...);
}

// forward sweep step j of L y = v (L rows in registers)
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

// back sweep for column J = K-1-I of L^T x = y in dot-product form, software
// pipelined: each thread sums its register rows of L (no transposed copy of
// the factor) and the group adds the partial sums by xor shuffles, but the
// sum over the rows far below J is reduced kLook steps ahead, so that its
// shuffles overlap the finishing of the columns in between; the terms of the
// kLook rows just below J come from their owners by one shuffle each.
//   kLook = 1: x_J = (y_J - P_J - L[J+1][J] x_{J+1}) / L[J][J], P_J over rows > J+1
//   kLook = 2: x_J = (y_J - Q_J - E_J - L[J+1][J] x_{J+1}) / L[J][J], Q_J over
//              rows > J+2, E_J = L[J+2][J] x_{J+2} (sent one step early)
// p0 carries the far sum for column J into the step; p1 and e0 (kLook = 2)
// carry Q_{J-1} and E_{J-1}. Every kernel takes the same depth (kBwdLook), so
// the fused IDW + kriging pass stays bitwise equal to the kriging call.
template <int K, int kLook, int I>
__device__ __forceinline__ void bwd_step(const float (&L)[Geo<K>::LEN], const float (&dinv)[kR],
                                         float (&v)[kR], int t, int gbase, float& p0, float& p1,
                                         float& e0) {
    static_assert(kLook == 1 || kLook == 2, "pipeline depth");
    using Gm = Geo<K>;
    constexpr int G = Gm::G;
    constexpr int J = K - 1 - I;
    constexpr int SJ = J / G;
    float dj = 0.0f, en = 0.0f;
    if constexpr (J + 1 < K) {
        constexpr int S1 = (J + 1) / G;
        dj = __shfl_sync(kFull, L[Gm::off(S1) + J] * v[S1], gbase + (J + 1) % G);
        if constexpr (kLook == 2 && J > 0)
            en = __shfl_sync(kFull, L[Gm::off(S1) + J - 1] * v[S1], gbase + (J + 1) % G);
    }
    // far sum for column J - kLook over the rows > J (all solved)
    float pn = 0.0f;
    if constexpr (J >= kLook) {
#pragma unroll
        for (int s = 0; s < kR; ++s)
            if (G * (s + 1) - 1 > J)
                pn = (G * s + t > J) ? fmaf(L[Gm::off(s) + J - kLook], v[s], pn) : pn;
#pragma unroll
        for (int o = 1; o < G; o <<= 1) pn += __shfl_xor_sync(kFull, pn, o);
    }
    if (t == J % G) v[SJ] = (((v[SJ] - p0) - e0) - dj) * dinv[SJ];
    if constexpr (kLook == 1) {
        p0 = pn;
    } else {
        p0 = p1;
        p1 = pn;
        e0 = en;
    }
}

template <int K, int kLook, int... J>
__device__ __forceinline__ void chol_solve_seq(const float (&L)[Geo<K>::LEN],
                                               const float (&dinv)[kR], float (&v)[kR], int t,
                                               int gbase, bool fwd, std::integer_sequence<int, J...>) {
    if (fwd) (fwd_step<K, J>(L, dinv, v, t, gbase), ...);  // else done in the factorization
    float p0 = 0.0f, p1 = 0.0f, e0 = 0.0f;
    (bwd_step<K, kLook, J>(L, dinv, v, t, gbase, p0, p1, e0), ...);
}

// L2 prefetch of the neighbour ids of solve block pb (sys systems of k ids
// each, from ids[pb * sys * k]): warp 0, one 128-byte line per lane, within
// the `nodes` systems of the launch. A hint that nothing waits on.
__device__ __forceinline__ void prefetch_ids_l2(const int32_t* ids, int64_t nodes, int k,
                                                int64_t pb, int sys) {
    if (threadIdx.x >= 32) return;
    const int64_t s0 = pb * sys;
    if (s0 >= nodes) return;
    const int64_t bytes = min((int64_t)sys, nodes - s0) * k * (int64_t)sizeof(int32_t);
    const char* base = reinterpret_cast<const char*>(ids + s0 * k);
    for (int64_t off = (int64_t)threadIdx.x * 128; off < bytes; off += 32 * 128)
        asm volatile("prefetch.global.L2 [%0];" ::"l"(base + off));
}

// 2^e as a float (|e| <= 126)
__device__ __forceinline__ float pow2f(int e) { return __int_as_float((127 + e) << 23); }

// exponent e with 2^(e-1) <= v < 2^e for finite v > 0
__device__ __forceinline__ int exp_above(float v) { return ((__float_as_int(v) >> 23) & 0xff) - 126; }

// The kriging systems of solve block `blk` (kWarps warps x SYS systems x
// kRounds rounds) of a range of `nodes` grid nodes starting at node0, with the
// neighbour ids of node node0 + i at ids[i * k]. smem: kWarps * WARP_FLOATS.
// With kPts the "nodes" are query points whose coordinates are px[], py[]
// (g unused).
// With kIdw the block also writes the IDW depth over the first fz.k of the
// node's sorted neighbours (fz.k <= k): the same value bg_interp_idw gives, as
// its operations are those of idw_from in the same order.
template <int K, bool kPts, bool kIdw, int kWarps>
__device__ __forceinline__ void okrige_solve_block(const HashView& h, const GridView& g, int k,
                                                   const OkParams& p, int64_t node0, int64_t nodes,
                                                   const int32_t* __restrict__ ids,
                                                   float* __restrict__ depth,
                                                   float* __restrict__ var, int64_t blk,
                                                   float* smem,
                                                   const int32_t* __restrict__ px = nullptr,
                                                   const int32_t* __restrict__ py = nullptr,
                                                   IdwFuse fz = IdwFuse{}) {
    using Gm = Geo<K>;
    constexpr int G = Gm::G;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int grp = lane / G, t = lane % G, gbase = grp * G;
    float* sysmem = smem + warp * Gm::WARP_FLOATS + grp * Gm::SYS_FLOATS;
    int* Aq = reinterpret_cast<int*>(sysmem);      // packed lower triangle: fixed-point A
    // per row r (neighbour r + 1), three arrays of K: x and y minus those of
    // neighbour 0 (cm) at T[r] and T[K + r], Gamma(neighbour r + 1,
    // neighbour 0) in the fixed-point scale at T[2K + r]; four consecutive
    // rows load as one 16-byte vector. After assembly T[r] and T[K + r] hold
    // the row's output terms.
    float* T = sysmem + Gm::TRIP;
    auto rec = [&](int r) { return make_float4(T[r], T[K + r], T[2 * K + r], 0.0f); };
    const unsigned gmask = (G == 32) ? 0xffffffffu : (((1u << G) - 1u) << gbase);

    for (int round = 0; round < kRounds; ++round) {
        const int64_t sys = (blk * kWarps + warp) * (Gm::SYS * kRounds) +
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
        const int ke = (id0 >= 0) ? 1 + (int)cnt : 0;  // 0: no output (no data, or past the end)
        int qx, qy;
        if constexpr (kPts) {
            qx = __ldg(px + node);
            qy = __ldg(py + node);
        } else {
            qx = g.x0 + (int)(node % g.nx) * g.cell + g.cell / 2;
            qy = g.y0 + (int)(node / g.nx) * g.cell + g.cell / 2;
        }

        // gather the neighbours' records; offsets from neighbour 0 as exact floats
        int4 r0 = make_int4(0, 0, 0, 0);
        if (id0 >= 0) r0 = __ldg(h.orig + id0);
        const float z0 = __int_as_float(r0.z);
        const float g00 = gamma_cm(p, r0.x - qx, r0.y - qy, 0.0f);
        float zr[kR], gr0[kR], g0r[kR];  // depth; Gamma(row's neighbour, nbr 0); gamma(node, row's nbr)
        float pox[kR], poy[kR];  // row's offsets from neighbour 0 (cm)
        int pdx[kR], pdy[kR];    // and from the node
        bool preal[kR];
        float gmax = 0.0f;
        // fused IDW: squared distance to the nearest, and each row's weight and anomaly
        uint64_t idw_d0 = 0;
        float idw_d1 = 0.0f, idw_l1 = 0.0f, idw_w[kR], idw_a[kR];
        if constexpr (kIdw) {
            const long long dx = (long long)r0.x - qx, dy = (long long)r0.y - qy;
            idw_d0 = (uint64_t)(dx * dx + dy * dy);
            idw_d1 = idw_d2f(idw_d0);
            if (fz.power != 2.0f) idw_l1 = log2f(idw_d1);
        }
#pragma unroll
        for (int s = 0; s < kR; ++s) {
            int4 rr = make_int4(0, 0, 0, 0);
            const bool real = nid[s] >= 0;
            if (real) rr = __ldg(h.orig + nid[s]);
            const int r = G * s + t;
            if constexpr (kIdw) {
                idw_w[s] = idw_a[s] = 0.0f;
                if (G * s + 1 < fz.k) {  // uniform: this slot holds IDW neighbours
                    const long long dx = (long long)rr.x - qx, dy = (long long)rr.y - qy;
                    idw_w[s] = idw_weight(idw_d1, idw_l1, 0.5f * fz.power, fz.power,
                                          idw_d2f((uint64_t)(dx * dx + dy * dy)));
                    idw_a[s] = __int_as_float(rr.z) - z0;
                }
            }
            const float ox = (float)(rr.x - r0.x), oy = (float)(rr.y - r0.y);
            T[r] = ox;
            T[K + r] = oy;
            zr[s] = __int_as_float(rr.z);
            pox[s] = ox;
            poy[s] = oy;
            pdx[s] = rr.x - qx;
            pdy[s] = rr.y - qy;
            preal[s] = real;
        }
        if (p.model == BG_VARIOGRAM_SPHERICAL && kR % 2 == 0) {
            // two rows per packed instruction: the same operations as
            // gamma_pair_f and gamma_cm, lane by lane
#pragma unroll
            for (int s = 0; s < kR; s += 2) {
                float ga, gb, ha, hb;
                gamma_pair_sph2(p, pox[s], poy[s], pox[s + 1], poy[s + 1], ga, gb);
                gamma_cm_sph2(p, pdx[s], pdy[s], pdx[s + 1], pdy[s + 1], ha, hb);
                gr0[s] = preal[s] ? ga : 0.0f;
                gr0[s + 1] = preal[s + 1] ? gb : 0.0f;
                g0r[s] = preal[s] ? ha : 0.0f;
                g0r[s + 1] = preal[s + 1] ? hb : 0.0f;
            }
        } else {
#pragma unroll
            for (int s = 0; s < kR; ++s) {
                gr0[s] = preal[s] ? gamma_pair_f(p, pox[s], poy[s]) : 0.0f;
                g0r[s] = preal[s] ? gamma_cm(p, pdx[s], pdy[s], 0.0f) : 0.0f;
            }
        }
#pragma unroll
        for (int s = 0; s < kR; ++s) gmax = fmaxf(gmax, gr0[s]);
#pragma unroll
        for (int o = 1; o < G; o <<= 1) gmax = fmaxf(gmax, __shfl_xor_sync(kFull, gmax, o));
        if constexpr (kIdw) {
            // thread t's partial holds neighbours 1 + t + G s in ascending s,
            // and the xor shuffles combine the partials as idw_tree8 does
            static_assert(G == kIdwLanes, "the fused IDW runs with 8 threads per system");
            const int ki = min(fz.k, ke);
            float num = 0.0f, den = 0.0f;
#pragma unroll
            for (int s = 0; s < kR; ++s)
                if (1 + G * s + t < ki) {
                    num = fmaf(idw_w[s], idw_a[s], num);
                    den += idw_w[s];
                }
#pragma unroll
            for (int o = 1; o < G; o <<= 1) {
                num += __shfl_xor_sync(kFull, num, o);
                den += __shfl_xor_sync(kFull, den, o);
            }
            if (live && t == 0)
                fz.out[node] = ke == 0 ? __int_as_float(0x7fc00000)
                                       : (idw_d0 == 0 ? z0 : z0 + num / (1.0f + den));
        }
        // A is SPD, so |A[r][c]| <= its largest diagonal entry max(1, 2 max Gamma_r0);
        // fixed point with 30 bits below that bound
        const int ea = 30 - exp_above(fmaxf(1.0f, 2.0f * gmax));
        const float sa = pow2f(ea);
#pragma unroll
        for (int s = 0; s < kR; ++s) T[2 * K + G * s + t] = gr0[s] * sa;  // Gamma_r0, fixed-point scale
        const ScaledVgm sv = scaled_vgm(p, sa);
        __syncwarp();

        // assemble the lower triangle once per entry, straight into fixed
        // point. Every term is in the fixed-point scale already (the records'
        // Gamma_r0 and the scaled variogram), so an entry is one rounding to
        // integer. The triangle splits into G x G blocks: below the diagonal
        // blocks, thread t owns the columns c = t + G q and the group walks
        // the rows in step (a row's entries land in consecutive banks), four
        // rows per batch, two per packed instruction. With G >= 4 a diagonal
        // block is taken by a circulant assignment in each thread's own
        // column (below); smaller groups deal its G (G + 1) / 2 entries out to
        // the group's threads in turn.
        auto entry_value = [&](auto spherical, int r, int c) {
            constexpr bool kSph = decltype(spherical)::value;
            const float4 a = rec(r), b = rec(c);
            // a real row r (r + 1 < ke) implies a real column c < r
            return (r == c) ? ((c + 1 < ke) ? 2.0f * b.z : sa)
                   : (r + 1 < ke) ? (a.z + b.z) - gamma_pair_scaled<kSph>(sv, a.x - b.x, a.y - b.y)
                                  : 0.0f;
        };
        constexpr int kDiag = G * (G + 1) / 2, kDiagSlots = (kDiag + G - 1) / G;
        int dij[kDiagSlots];  // (row, column) in a diagonal block of this thread's slots
#pragma unroll
        for (int m = 0; m < kDiagSlots; ++m) {
            const int e = t + G * m;
            int i = 0;
            while (tri(i + 1) <= e) ++i;
            dij[m] = (i << 8) | (e - tri(i));
        }
        // loads and arithmetic of a batch ahead of its stores: the stores to
        // the triangle then never sit between one entry's loads and the next
        auto assemble = [&](auto spherical) {
            constexpr bool kSph = decltype(spherical)::value;
#pragma unroll
            for (int q = 0; q < kR; ++q) {
                const int c = t + G * q;
                const float4 cc = rec(c);
                const float xc = cc.x, yc = cc.y, gcc = cc.z;
                if constexpr (G >= 4) {
                    // the diagonal block: entry (t + d mod G, t) of this thread's
                    // column for d = 1 .. G/2 (d = G/2 only for t < G/2, so each
                    // pair of the block is taken once), evaluated with the
                    // other row's record and stored at its lower-triangle place;
                    // the value is symmetric, bit for bit, in the two records
                    constexpr int kH = G / 2;
                    float dv[kH];
                    int ri[kH];
#pragma unroll
                    for (int d = 1; d <= kH; ++d) ri[d - 1] = G * q + (t + d) % G;
                    if constexpr (kSph) {
#pragma unroll
                        for (int d = 0; d < kH; d += 2)
                            gamma_rows2_sph(sv, T[ri[d]], T[ri[d + 1]], T[K + ri[d]], T[K + ri[d + 1]],
                                            T[2 * K + ri[d]], T[2 * K + ri[d + 1]], xc, yc, gcc,
                                            dv[d], dv[d + 1]);
                    } else {
#pragma unroll
                        for (int d = 0; d < kH; ++d)
                            dv[d] = (T[2 * K + ri[d]] + gcc) -
                                    gamma_pair_scaled<false>(sv, T[ri[d]] - xc, T[K + ri[d]] - yc);
                    }
                    Aq[tri(c) + c] = __float2int_rn((c + 1 < ke) ? 2.0f * gcc : sa);
#pragma unroll
                    for (int d = 0; d < kH; ++d) {
                        if (d + 1 == kH && t >= kH) break;  // the other half takes these
                        const int hi = max(ri[d], c), lo = min(ri[d], c);
                        Aq[tri(hi) + lo] = __float2int_rn((hi + 1 < ke) ? dv[d] : 0.0f);
                    }
                } else {
                float dv[kDiagSlots];
#pragma unroll
                for (int m = 0; m < kDiagSlots; ++m)
                    dv[m] = (kDiag % G == 0 || m + 1 < kDiagSlots || t + G * m < kDiag)
                                ? entry_value(spherical, G * q + (dij[m] >> 8), G * q + (dij[m] & 0xff))
                                : 0.0f;
#pragma unroll
                for (int m = 0; m < kDiagSlots; ++m)
                    if (kDiag % G == 0 || m + 1 < kDiagSlots || t + G * m < kDiag)
                        Aq[tri(G * q + (dij[m] >> 8)) + G * q + (dij[m] & 0xff)] = __float2int_rn(dv[m]);
                }
                constexpr int kB = 4;
#pragma unroll
                for (int r0 = G * (q + 1); r0 < K; r0 += kB) {
                    // (K - G (q + 1) need not be a multiple of kB: rows from K on
                    // are skipped at compile time)
                    float vb[kB];
                    if constexpr (G >= 4 && kSph) {
                        // r0 is a multiple of 4: rows r0 .. r0 + 3 in one vector per
                        // array, two rows per packed operation
                        const float4 X = *reinterpret_cast<const float4*>(T + r0);
                        const float4 Y = *reinterpret_cast<const float4*>(T + K + r0);
                        const float4 Z = *reinterpret_cast<const float4*>(T + 2 * K + r0);
                        gamma_rows2_sph(sv, X.x, X.y, Y.x, Y.y, Z.x, Z.y, xc, yc, gcc, vb[0], vb[1]);
                        gamma_rows2_sph(sv, X.z, X.w, Y.z, Y.w, Z.z, Z.w, xc, yc, gcc, vb[2], vb[3]);
#pragma unroll
                        for (int u = 0; u < kB; ++u)
                            if (!(r0 + u + 1 < ke)) vb[u] = 0.0f;
                    } else {
#pragma unroll
                    for (int u = 0; u < kB; ++u) {
                        const int r = r0 + u;
                        vb[u] = 0.0f;
                        if (r < K) {
                            const float4 a = rec(r);
                            if (r + 1 < ke)
                                vb[u] = (a.z + gcc) - gamma_pair_scaled<kSph>(sv, a.x - xc, a.y - yc);
                        }
                    }
                    }
#pragma unroll
                    for (int u = 0; u < kB; ++u)
                        if (r0 + u < K) Aq[tri(r0 + u) + c] = __float2int_rn(vb[u]);
                }
            }
        };
        if (p.model == BG_VARIOGRAM_SPHERICAL)
            assemble(std::true_type{});
        else
            assemble(std::false_type{});
        __syncwarp();

        // my rows into registers (zero above the diagonal), in the fixed-point
        // scale: the factor is that of sa A, and the solves scale their
        // right-hand sides by sa to match, so x comes out in A's units
        float L[Gm::LEN];
        float b[kR];
#pragma unroll
        for (int s = 0; s < kR; ++s) {
            const int r = G * s + t;
            b[s] = (r + 1 < ke) ? (gr0[s] + g00) - g0r[s] : 0.0f;
            // the tables are free after assembly: keep the row's output terms
            // there rather than in registers through the solve
            T[r] = zr[s] - z0;
            T[K + r] = g0r[s] - gr0[s];
#pragma unroll
            for (int c = 0; c < G * (s + 1); ++c) {
                const int q = Aq[c <= r ? tri(r) + c : 0];
                L[Gm::off(s) + c] = c <= r ? (float)q : 0.0f;
            }
        }

        // factor in registers
        float dinv[kR];
#pragma unroll
        for (int s = 0; s < kR; ++s) dinv[s] = 1.0f;
        float v[kR], x[kR];
#pragma unroll
        for (int s = 0; s < kR; ++s) v[s] = b[s] * sa;
        chol_factor<K>(L, dinv, t, gbase, sysmem + Gm::CB, v, std::make_integer_sequence<int, K>{});

        // solve, one refinement step, solve again. The residual b - A' x' is
        // exact: x' is x rounded to 24-bit fixed point (representable in FP32),
        // A' the 30-bit copy, and the sum of the 2^54-bounded products is
        // accumulated in 64-bit integers without rounding.
#pragma unroll 1
        for (int pass = 0; pass < 2; ++pass) {
            chol_solve_seq<K, kBwdLook>(L, dinv, v, t, gbase, pass != 0,
                                        std::make_integer_sequence<int, K>{});
            if (pass == 1) {
#pragma unroll
                for (int s = 0; s < kR; ++s) x[s] += v[s];
                break;
            }
            float xmax = 0.0f;
#pragma unroll
            for (int s = 0; s < kR; ++s) xmax = fmaxf(xmax, fabsf(v[s]));
#pragma unroll
            for (int o = 1; o < G; o <<= 1) xmax = fmaxf(xmax, __shfl_xor_sync(kFull, xmax, o));
            const int ex = xmax > 0.0f ? 24 - exp_above(xmax) : 0;
            const float sx = pow2f(ex), isx = pow2f(-ex);
            int xq[kR];
            long long acc[kR];
#pragma unroll
            for (int s = 0; s < kR; ++s) {
                xq[s] = __float2int_rn(v[s] * sx);
                x[s] = (float)xq[s] * isx;
                acc[s] = __float2ll_rn((b[s] * sa) * sx);
            }
            if constexpr (G >= 4) {
                // x' of the group through the column buffer: one 16-byte store
                // per thread, four columns per 16-byte load
                int* xb = reinterpret_cast<int*>(sysmem + Gm::CB);
                *reinterpret_cast<int4*>(xb + 4 * t) = make_int4(xq[0], xq[1], xq[2], xq[3]);
                __syncwarp();
#pragma unroll 2
                for (int tc = 0; tc < G; ++tc) {
                    const int4 q4 = *reinterpret_cast<const int4*>(xb + 4 * tc);
                    const int q[4] = {q4.x, q4.y, q4.z, q4.w};
#pragma unroll
                    for (int sc = 0; sc < kR; ++sc) {
                        const int c = G * sc + tc;
#pragma unroll
                        for (int s = 0; s < kR; ++s) {
                            // slots below / above mine hold columns below / above my row
                            const int r = G * s + t;
                            const int a = sc < s   ? Aq[tri(r) + c]
                                          : sc > s ? Aq[tri(c) + r]
                                                   : Aq[tri(max(r, c)) + min(r, c)];
                            acc[s] -= (long long)a * (long long)q[sc];
                        }
                    }
                }
                __syncwarp();  // the buffer serves the next system's factor
            } else {
#pragma unroll
                for (int sc = 0; sc < kR; ++sc) {
#pragma unroll 4
                    for (int tc = 0; tc < G; ++tc) {
                        const int c = G * sc + tc;
                        const int xc = __shfl_sync(kFull, xq[sc], gbase + tc);
#pragma unroll
                        for (int s = 0; s < kR; ++s) {
                            const int r = G * s + t;
                            const int a = Aq[tri(max(r, c)) + min(r, c)];
                            acc[s] -= (long long)a * (long long)xc;
                        }
                    }
                }
            }
#pragma unroll
            for (int s = 0; s < kR; ++s) v[s] = (float)acc[s] * isx;  // sa (b - A' x')
        }

        // weights and outputs; the weight sum closes in FP64
        float ps = 0.0f, pz = 0.0f, pv = 0.0f;
#pragma unroll
        for (int s = 0; s < kR; ++s) {
            const bool row = G * s + t + 1 < ke;
            const float lam = row ? x[s] : 0.0f;
            ps += lam;
            pz = fmaf(lam, T[G * s + t], pz);      // z_a - z_0
            pv = fmaf(lam, T[K + G * s + t], pv);  // gamma_0a - Gamma_a0
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

}  // namespace bg
