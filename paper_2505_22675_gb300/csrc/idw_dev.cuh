// Device code of fused k-NN + IDW, shared by the per-grid kernels (idw.cu)
// and the batched persistent kernels (batch.cu).
//
// Fused exact k-NN + inverse-distance weighting, one thread per grid node.
//
// zhat = sum w_i z_i / sum w_i with w_i = d_i^-p over the k nearest valid
// soundings. It is evaluated as z_1 + sum w_i (z_i - z_1) / sum w_i with
// z_1 the nearest sounding's depth and w_i = (d_1^2 / d_i^2)^(p/2): the same
// quantity, but every term is an anomaly of a few metres (so only the final
// add rounds at ~3500 m) and every weight is in (0, 1]. The sums run in one
// fixed order over the ascending (d2, index) list (idw_tree8), so a node's
// result does not depend on the cell size, the launch shape, the kernel or
// what else runs.


#pragma once

#include <cmath>

#include "bg_internal.h"
#include "knn.cuh"

namespace bg {


// d2 as float: a 32-bit conversion when it fits (64-bit ones use the FP64 pipe)
__device__ __forceinline__ float idw_d2f(uint64_t v) {
    return v < (1ull << 31) ? __int2float_rn((int)v) : __ull2float_rn(v);
}

// weight of a neighbour at squared distance di relative to the nearest (d1):
// (d1 / di)^(p/2), with l1 = log2(d1) and hp = p / 2
__device__ __forceinline__ float idw_weight(float d1, float l1, float hp, float power, float di) {
    if (power == 2.0f) return d1 / di;
    return exp2f(hp * (l1 - log2f(di)));
}

// The sums of an IDW run in one fixed order, so that every kernel that forms
// them gets bitwise the same depth: neighbour n >= 1 goes to partial n_t =
// (n - 1) mod 8, each partial adds its neighbours in ascending n, and the 8
// partials combine pairwise as ((p0 + p1) + (p2 + p3)) + ((p4 + p5) + (p6 +
// p7)). The kriging solve (8 threads per system, thread t holding neighbours
// 1 + t + 8 s) forms the same partials in registers and combines them with
// xor shuffles in that pattern.
constexpr int kIdwLanes = 8;

__device__ __forceinline__ float idw_tree8(const float (&p)[kIdwLanes]) {
    return ((p[0] + p[1]) + (p[2] + p[3])) + ((p[4] + p[5]) + (p[6] + p[7]));
}

// IDW from the neighbours in ascending (d2, index) order; get(i) returns
// (d2, upload index) of the i-th.
template <class Get>
__device__ __forceinline__ float idw_from(const HashView& h, int keff, float power, Get get) {
    if (keff == 0) return __int_as_float(0x7fc00000);  // NaN: no valid sounding
    const int* zb = reinterpret_cast<const int*>(h.orig) + 2;  // z bits of record i at zb[4*i]
    uint64_t d0;
    int i0;
    get(0, d0, i0);
    const float z1 = __int_as_float(__ldg(zb + 4 * (int64_t)i0));
    if (d0 == 0) return z1;  // node on top of a sounding
    const float d1 = idw_d2f(d0);
    float l1 = 0.0f;  // log2(d1), for powers other than 2
    if (power != 2.0f) l1 = log2f(d1);
    const float hp = 0.5f * power;
    float num[kIdwLanes], den[kIdwLanes];
#pragma unroll
    for (int q = 0; q < kIdwLanes; ++q) num[q] = den[q] = 0.0f;
#pragma unroll
    for (int n = 1; n < 32; ++n) {
        if (n >= keff) break;
        uint64_t di2;
        int ii;
        get(n, di2, ii);
        const float zi = __int_as_float(__ldg(zb + 4 * (int64_t)ii));
        const float w = idw_weight(d1, l1, hp, power, idw_d2f(di2));
        num[(n - 1) % kIdwLanes] = fmaf(w, zi - z1, num[(n - 1) % kIdwLanes]);
        den[(n - 1) % kIdwLanes] += w;
    }
    // neighbour 0 contributes weight 1 and anomaly 0
    return z1 + idw_tree8(num) / (1.0f + idw_tree8(den));
}

template <int K, bool kWide>
__device__ __forceinline__ void idw_node(const HashView& h, const GridView& g, int k, float power,
                                         float* __restrict__ depth, int32_t* __restrict__ nbr,
                                         int* __restrict__ flag, NodeIdx nd, uint64_t* hp) {
    if (nd.i >= g.nx || nd.j >= g.ny) return;
    const int64_t node = (int64_t)nd.j * g.nx + nd.i;
    const int qx = g.x0 + nd.i * g.cell + g.cell / 2;
    const int qy = g.y0 + nd.j * g.cell + g.cell / 2;
    int32_t* o = nbr ? nbr + node * k : nullptr;
    if (h.n_valid == 0) {
        if (kWide) return;
        depth[node] = __int_as_float(0x7fc00000);
        if (o)
            for (int i = 0; i < k; ++i) o[i] = -1;
        return;
    }
    const Bound b = knn_bound<K>(h, qx, qy);
    const bool fits = packed_fits(h, b.tau0);
    if constexpr (kWide) {
        if (fits) return;  // done by the packed pass
        uint64_t d2[K];
        int id[K];
        const int keff = min(knn_scan<K, true>(h, qx, qy, b, d2, id), k);
        depth[node] = idw_from(h, keff, power, [&](int i, uint64_t& dd, int& ii) {
            // the register arrays are read with a runtime index only here, in the rare wide pass
            dd = d2[i];
            ii = id[i];
        });
        if (o)
            for (int i = 0; i < k; ++i) o[i] = i < keff ? id[i] : -1;
    } else {
        if (!fits) {
            *flag = 1;  // the wide pass picks this node up
            return;
        }
        const int keff = min(knn_scan_heap<K, 128>(h, qx, qy, b, hp), k);
        const int bits = h.idx_bits;
        const uint64_t mask = (1ull << bits) - 1;
        depth[node] = idw_from(h, keff, power, [&](int i, uint64_t& dd, int& ii) {
            const uint64_t key = hp[i * 128];
            dd = key >> bits;
            ii = (int)(key & mask);
        });
        if (o)
            for (int i = 0; i < k; ++i) o[i] = i < keff ? (int)(hp[i * 128] & mask) : -1;
    }
}

// Wide-key IDW of one query point whose table bound does not fit the packed
// key (the rare pass after knn_chain flagged a point); other points return.
template <int K>
__device__ __forceinline__ void idw_point_wide(const HashView& h, int qx, int qy, int k,
                                               float power, float* __restrict__ dout,
                                               int32_t* __restrict__ o) {
    if (h.n_valid == 0 || !query_in_range(qx, qy)) return;
    const Bound b = knn_bound<K>(h, qx, qy);
    if (packed_fits(h, b.tau0)) return;
    uint64_t d2[K];
    int id[K];
    const int keff = min(knn_scan<K, true>(h, qx, qy, b, d2, id), k);
    *dout = idw_from(h, keff, power, [&](int i, uint64_t& dd, int& ii) {
        dd = d2[i];
        ii = id[i];
    });
    if (o)
        for (int i = 0; i < k; ++i) o[i] = i < keff ? id[i] : -1;
}

}  // namespace bg
