// Gridded input: bilinear (Sec. III-A) and Catmull-Rom (Sec. III-B)
// resampling of a regular grid at query points or at the nodes of another
// grid.
//
// Each query finds the lattice cell that holds it (exact integer
// arithmetic: index i and remainder r in [0, cell] along each axis) and
// reads the 2 x 2 (bilinear) or 4 x 4 (Catmull-Rom, edge nodes repeated)
// nodes around it. A node is needed when its weight is not zero: a query on
// a node line (r = 0 or r = cell) needs only that line. A needed NaN node
// gives NaN for bilinear, which has no fallback, and sends Catmull-Rom to
// bilinear. Sums are taken as anomalies from one needed node, so at depths of
// thousands of metres only the final add rounds at that magnitude.
//
// Point lists and general output grids: a thread takes 4 queries 256 apart
// and reads the needed stencil nodes of all four with predicated loads, so
// they overlap; a warp takes 32 neighbouring queries, so the source rows it
// reads are contiguous and shared through L1. Output grids at the source's
// spacing on its node columns (the row-filling shape) take k_resample_rows:
// four columns per thread in 16-byte vectors. The work is a gather bounded
// by HBM: 4 B per output (+ 8 B of coordinates for point lists), plus one
// read of the source grid.
#include <algorithm>
#include <cmath>

#include "bg_internal.h"

namespace bg {
namespace {

struct Src {
    const float* v;
    int32_t cx0, cy0;  // first node centre (cm)
    int32_t cell, nx, ny;
    float inv_cell;    // 1 / cell
};

// r / cell for r in [0, cell], exactly 0 and 1 at the ends (a multiply by the
// reciprocal elsewhere: one rounding more than a division, far below the
// tolerance of a depth)
__device__ __forceinline__ float frac_of(int r, const Src& s) {
    return r == s.cell ? 1.0f : (float)r * s.inv_cell;
}

// Position of a query along one axis of the node lattice: cell index i in
// [0, n - 2], remainder r = u - i * cell in [0, cell] (u: offset from the
// first node centre), and whether u lies inside the hull [0, (n-1) cell].
// Outside, i = r = 0 so that every load the caller makes stays in bounds.
struct Axis {
    int i, r;
    bool in;
};

__device__ __forceinline__ Axis axis_of(int64_t u, int cell, int n) {
    Axis a;
    a.in = u >= 0 && u <= (int64_t)(n - 1) * cell;
    const unsigned uu = a.in ? (unsigned)u : 0u;  // < 2^31: node centres lie in (-2^30, 2^30)
    unsigned q = uu / (unsigned)cell;
    if (q > (unsigned)(n - 2)) q = (unsigned)(n - 2);
    a.i = (int)q;
    a.r = (int)(uu - q * (unsigned)cell);
    return a;
}

// Which of the stencil points P0..P3 (nodes i-1 .. i+2) carry weight: all four
// inside the cell, only P1 on the near node line, only P2 on the far one.
__device__ __forceinline__ bool needed(const Axis& a, int cell, int k) {
    return a.r == 0 ? k == 1 : (a.r == cell ? k == 2 : true);
}

// Bilinear (Sec. III-A) from the corner values; corners whose weight is zero
// must come in as 0 (a NaN there does not enter), and a needed NaN corner
// propagates through its term. Anomalies from a needed corner.
__device__ __forceinline__ float bilinear_from(const Src& s, const Axis& ax, const Axis& ay,
                                               float q00, float q10, float q01, float q11) {
    const float t = frac_of(ax.r, s), u = frac_of(ay.r, s);
    const bool x0 = ax.r != s.cell, y0 = ay.r != s.cell;
    const float ref = x0 ? (y0 ? q00 : q01) : (y0 ? q10 : q11);
    const float a = fmaf(1.0f - t, (1.0f - u) * (q00 - ref),
                         fmaf(t, (1.0f - u) * (q10 - ref),
                              fmaf(1.0f - t, u * (q01 - ref), t * u * (q11 - ref))));
    return ref + a;
}

// Catmull-Rom weights of P0..P3 at t (Sec. III-B, C(t) expanded per point)
__device__ __forceinline__ void cr_weights(float t, float (&w)[4]) {
    const float t2 = t * t, t3 = t2 * t;
    w[0] = 0.5f * (-t + 2.0f * t2 - t3);
    w[1] = 0.5f * (2.0f - 5.0f * t2 + 3.0f * t3);
    w[2] = 0.5f * (t + 4.0f * t2 - 3.0f * t3);
    w[3] = 0.5f * (t3 - t2);
}

// One query from its two axes. fetch(b, c) returns the source node at column
// c (clamped into the grid by the caller) of stencil row b, i.e. source row
// j - 1 + b clamped into the grid (bilinear uses rows 1 and 2). Only the
// needed stencil nodes are read (predicated loads, no branches), so the loads
// of a thread's queries overlap. how: 0 by the method, 1 by the bilinear
// fallback, 2 no value.
// kColX: every query of the launch lies on a node column (the row-filling
// shape), so only the column case is compiled.
template <int kMethod, bool kColX, class Fetch>
__device__ __forceinline__ float resample_at(const Src& s, const Axis& ax, const Axis& ay,
                                             const Fetch& fetch, int8_t& how) {
    float f;
    const int i = ax.i;
    if constexpr (kMethod == BG_RESAMPLE_CATMULL_ROM) {
        if (kColX || ax.r == 0 || ax.r == s.cell) {
            // on a node column (the row-filling shape): one column of the stencil,
            // the same arithmetic as the general case with x weights (0, 1, 0, 0)
            const int a = ax.r == 0 ? 1 : 2;
            const int c = i - 1 + a;
            bool ny_[4];
            float P[4];
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                ny_[b] = needed(ay, s.cell, b);
                P[b] = ny_[b] ? fetch(b, c) : 0.0f;
            }
            const float ref = P[ay.r == s.cell ? 2 : 1];
            float wy[4];
            cr_weights(frac_of(ay.r, s), wy);
            float acc = 0.0f;
            bool nan = false;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                nan |= ny_[b] && isnan(P[b]);
                acc = ny_[b] ? fmaf(wy[b], P[b] - ref, acc) : acc;
            }
            if (!nan) {
                f = ref + acc;
                how = 0;
            } else {
                f = bilinear_from(s, ax, ay, a == 1 ? P[1] : 0.0f, a == 2 ? P[1] : 0.0f,
                                  a == 1 ? P[2] : 0.0f, a == 2 ? P[2] : 0.0f);
                how = isnan(f) ? 2 : 1;
            }
        } else {
            int col[4];
            bool nx_[4], ny_[4];
#pragma unroll
            for (int a = 0; a < 4; ++a) {
                col[a] = min(max(i - 1 + a, 0), s.nx - 1);
                nx_[a] = needed(ax, s.cell, a);
                ny_[a] = needed(ay, s.cell, a);
            }
            float P[4][4];
#pragma unroll
            for (int b = 0; b < 4; ++b)
#pragma unroll
                for (int a = 0; a < 4; ++a)
                    P[b][a] = (nx_[a] && ny_[b]) ? fetch(b, col[a]) : 0.0f;
            const float ref = P[ay.r == s.cell ? 2 : 1][ax.r == s.cell ? 2 : 1];
            float wx[4], wy[4];
            cr_weights(frac_of(ax.r, s), wx);
            cr_weights(frac_of(ay.r, s), wy);
            float acc = 0.0f;
            bool nan = false;
#pragma unroll
            for (int b = 0; b < 4; ++b) {
                float r = 0.0f;
#pragma unroll
                for (int a = 0; a < 4; ++a) {
                    const bool need = nx_[a] && ny_[b];
                    nan |= need && isnan(P[b][a]);
                    r = need ? fmaf(wx[a], P[b][a] - ref, r) : r;
                }
                acc = ny_[b] ? fmaf(wy[b], r, acc) : acc;
            }
            if (!nan) {
                f = ref + acc;
                how = 0;
            } else {
                // the bilinear corners are stencil nodes (1,1), (2,1), (1,2), (2,2)
                // and were read exactly when needed by bilinear too
                f = bilinear_from(s, ax, ay, P[1][1], P[1][2], P[2][1], P[2][2]);
                how = isnan(f) ? 2 : 1;
            }
        }
    } else {
        const bool x0 = ax.r != s.cell, x1 = ax.r != 0, y0 = ay.r != s.cell, y1 = ay.r != 0;
        const float q00 = (x0 && y0) ? fetch(1, i) : 0.0f;
        const float q10 = (x1 && y0) ? fetch(1, i + 1) : 0.0f;
        const float q01 = (x0 && y1) ? fetch(2, i) : 0.0f;
        const float q11 = (x1 && y1) ? fetch(2, i + 1) : 0.0f;
        f = bilinear_from(s, ax, ay, q00, q10, q01, q11);
        how = isnan(f) ? 2 : 0;
    }
    if (!(ax.in && ay.in)) {
        how = 2;
        f = __int_as_float(0x7fc00000);
    }
    return f;
}

__device__ __forceinline__ void row_ptrs(const Src& s, int j, const float* (&rows)[4]) {
#pragma unroll
    for (int b = 0; b < 4; ++b) rows[b] = s.v + (int64_t)min(max(j - 1 + b, 0), s.ny - 1) * s.nx;
}

constexpr int kThreads = 256;
constexpr int kPer = 4;  // outputs per thread, kThreads apart: every access stays coalesced

// Queries past the end are computed on a clamped index and not stored, so
// that no load depends on a branch and the queries' loads overlap.
template <int kMethod>
__global__ void __launch_bounds__(kThreads) k_resample_pts(Src s, const int32_t* __restrict__ qx,
                                                           const int32_t* __restrict__ qy,
                                                           int64_t m, float* __restrict__ out,
                                                           int8_t* __restrict__ how_out) {
    for (int64_t base = (int64_t)blockIdx.x * kThreads * kPer; base < m;
         base += (int64_t)gridDim.x * kThreads * kPer) {
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int64_t p = base + k * kThreads + threadIdx.x;
            const int64_t pc = p < m ? p : m - 1;
            const Axis ax = axis_of((int64_t)__ldg(qx + pc) - s.cx0, s.cell, s.nx);
            const Axis ay = axis_of((int64_t)__ldg(qy + pc) - s.cy0, s.cell, s.ny);
            const float* rows[4];
            row_ptrs(s, ay.i, rows);
            const auto fetch = [&](int b, int c) { return __ldg(rows[b] + c); };
            int8_t how;
            const float f = resample_at<kMethod, false>(s, ax, ay, fetch, how);
            if (p < m) {
                out[p] = f;
                if (how_out) how_out[p] = how;
            }
        }
    }
}

// output grid: block b takes kThreads * kPer columns (chunk b % chunks) of
// kRowsPerBlock consecutive rows; a thread's four column positions in the
// source lattice (one integer division each) serve all its rows
constexpr int kRowsPerBlock = 8;

template <int kMethod, bool kColX>
__global__ void __launch_bounds__(kThreads, 4)
    k_resample_grid(Src s, GridView o, int chunks, float* __restrict__ out,
                    int8_t* __restrict__ how_out) {
    const int band = blockIdx.x / chunks;
    const int c0 = (blockIdx.x - band * chunks) * kThreads * kPer + threadIdx.x;
    const int64_t ux0 = (int64_t)o.x0 + o.cell / 2 - s.cx0;
    Axis ax[kPer];
#pragma unroll
    for (int k = 0; k < kPer; ++k) {
        const int c = c0 + k * kThreads;
        ax[k] = axis_of(ux0 + (int64_t)(c < o.nx ? c : o.nx - 1) * o.cell, s.cell, s.nx);
    }
    const int row1 = min(o.ny, (band + 1) * kRowsPerBlock);
    for (int row = band * kRowsPerBlock; row < row1; ++row) {
        const Axis ay =
            axis_of((int64_t)o.y0 + (int64_t)row * o.cell + o.cell / 2 - s.cy0, s.cell, s.ny);
        const float* rows[4];
        row_ptrs(s, ay.i, rows);
        const auto fetch = [&](int b, int c) { return __ldg(rows[b] + c); };
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
            const int c = c0 + k * kThreads;
            int8_t how;
            const float f = resample_at<kMethod, kColX>(s, ax[k], ay, fetch, how);
            if (c < o.nx) {
                const int64_t p = (int64_t)row * o.nx + c;
                out[p] = f;
                if (how_out) how_out[p] = how;
            }
        }
    }
}

// Output grid at the source's own spacing whose columns lie on source columns
// (output column c on source column c + d; d, both row lengths a multiple of
// 4 and the arrays 16-byte aligned; the row-filling shape): a thread takes 4
// consecutive columns in each of kVecGroups places of its band's rows and
// moves them with 16-byte loads and stores (a 4-byte store of the how-codes);
// its stencil rows come from those vectors, held in registers. They are
// loaded exactly when the row's stencil needs them, and a vector lies either
// wholly inside the source's columns or wholly outside (no value). A row on a
// source row line takes resample_at's node-column case itself; a row between
// two takes the same roundings without the selects of zero weights (results
// equal to k_resample_grid's up to the sign of a zero). This kernel moves
// 9 B per output (a read of the source row, the value and the how-code) at
// 1:1 and has few instructions per byte: with 8 (bilinear) or 6 (Catmull-
// Rom) blocks per SM it runs close to the copy bandwidth.
constexpr int kVec = 4;
constexpr int kVecGroups = 1;

__device__ __forceinline__ float lane_of(const float4& v, int k) {
    return k == 0 ? v.x : (k == 1 ? v.y : (k == 2 ? v.z : v.w));
}

template <int kMethod>
__global__ void __launch_bounds__(kThreads, kMethod == BG_RESAMPLE_CATMULL_ROM ? 6 : 8)
    k_resample_rows(Src s, GridView o, int64_t d, int chunks, float* __restrict__ out,
                    int8_t* __restrict__ how_out) {
    const int band = blockIdx.x / chunks;
    const int cb = (blockIdx.x - band * chunks) * (kThreads * kVec * kVecGroups) + threadIdx.x * kVec;
    const int64_t uy0 = (int64_t)o.y0 + o.cell / 2 - s.cy0;
    const int row0 = band * kRowsPerBlock;
    const int row1 = min(o.ny, row0 + kRowsPerBlock);
    Axis ay = axis_of(uy0 + (int64_t)row0 * o.cell, s.cell, s.ny);
    float u = frac_of(ay.r, s);
    float wy[4];
    cr_weights(u, wy);
    for (int row = row0; row < row1; ++row) {
        if (row > row0) {
            // one source row further: the same remainder while the next cell
            // index stays below the clamp, else the axis afresh
            if (ay.in && ay.r < s.cell && ay.i + 1 <= s.ny - 2) {
                ++ay.i;
            } else {
                ay = axis_of(uy0 + (int64_t)row * o.cell, s.cell, s.ny);
                u = frac_of(ay.r, s);
                cr_weights(u, wy);
            }
        }
        const float* rows[4];
        row_ptrs(s, ay.i, rows);
        bool use[4];
#pragma unroll
        for (int b = 0; b < 4; ++b)
            use[b] = (kMethod == BG_RESAMPLE_CATMULL_ROM || b == 1 || b == 2) && needed(ay, s.cell, b);
        const bool interior = ay.in && ay.r != 0 && ay.r != s.cell;
#pragma unroll
        for (int g = 0; g < kVecGroups; ++g) {
            const int c = cb + g * kThreads * kVec;
            if (c >= o.nx) break;
            const int64_t i0 = c + d;
            const bool vin = i0 >= 0 && i0 < s.nx;
            float4 R[4];
#pragma unroll
            for (int b = 0; b < 4; ++b)
                R[b] = (vin && use[b]) ? __ldg(reinterpret_cast<const float4*>(rows[b] + i0))
                                       : make_float4(0.0f, 0.0f, 0.0f, 0.0f);
            float f[kVec];
            int8_t h[kVec];
            if (interior) {
                // every stencil row carries weight: resample_at's node-column
                // arithmetic without its weight-zero selects. Bilinear's terms of
                // the other column vanish (t is 0 or 1), leaving ref + u (q1 - ref)
                // with ref = q0, rounded as there; Catmull-Rom's FMA chain is the
                // same, and a NaN among the four rows is a NaN in the sum of their
                // magnitudes.
#pragma unroll
                for (int k = 0; k < kVec; ++k) {
                    if constexpr (kMethod == BG_RESAMPLE_CATMULL_ROM) {
                        const float p0 = lane_of(R[0], k), p1 = lane_of(R[1], k),
                                    p2 = lane_of(R[2], k), p3 = lane_of(R[3], k);
                        float acc = fmaf(wy[0], p0 - p1, 0.0f);
                        acc = fmaf(wy[1], p1 - p1, acc);
                        acc = fmaf(wy[2], p2 - p1, acc);
                        acc = fmaf(wy[3], p3 - p1, acc);
                        if (!isnan(fabsf(p0) + fabsf(p1) + fabsf(p2) + fabsf(p3))) {
                            f[k] = p1 + acc;
                            h[k] = 0;
                        } else {
                            f[k] = __fadd_rn(p1, __fmul_rn(u, __fsub_rn(p2, p1)));
                            h[k] = isnan(f[k]) ? 2 : 1;
                        }
                    } else {
                        const float q0 = lane_of(R[1], k), q1 = lane_of(R[2], k);
                        f[k] = __fadd_rn(q0, __fmul_rn(u, __fsub_rn(q1, q0)));
                        h[k] = isnan(f[k]) ? 2 : 0;
                    }
                    if (!vin) {
                        f[k] = __int_as_float(0x7fc00000);
                        h[k] = 2;
                    }
                }
            } else {
#pragma unroll
                for (int k = 0; k < kVec; ++k) {
                    // the node column i0 + k as axis_of gives it: cell index clamped
                    // to nx - 2, remainder 0, or cell on the last column
                    Axis ax;
                    ax.in = vin;
                    ax.i = vin ? (int)min(i0 + k, (int64_t)s.nx - 2) : 0;
                    ax.r = (vin && i0 + k == s.nx - 1) ? s.cell : 0;
                    const auto fetch = [&](int b, int) { return lane_of(R[b], k); };
                    f[k] = resample_at<kMethod, true>(s, ax, ay, fetch, h[k]);
                }
            }
            const int64_t p = (int64_t)row * o.nx + c;
            *reinterpret_cast<float4*>(out + p) = make_float4(f[0], f[1], f[2], f[3]);
            if (how_out)
                *reinterpret_cast<uint32_t*>(how_out + p) =
                    (uint32_t)(uint8_t)h[0] | (uint32_t)(uint8_t)h[1] << 8 |
                    (uint32_t)(uint8_t)h[2] << 16 | (uint32_t)(uint8_t)h[3] << 24;
        }
    }
}

}  // namespace

bg_status launch_resample_points(const float* src, const GridView& g, int method,
                                 const int32_t* qx, const int32_t* qy, int64_t m, float* out,
                                 int8_t* how, cudaStream_t st) {
    if (m == 0) return BG_OK;
    const Src s{src, g.x0 + g.cell / 2, g.y0 + g.cell / 2, g.cell, g.nx, g.ny, 1.0f / (float)g.cell};
    const int64_t blocks =
        std::min<int64_t>((m + kThreads * kPer - 1) / (kThreads * kPer), (int64_t)152 * 64);
    if (method == BG_RESAMPLE_CATMULL_ROM)
        k_resample_pts<BG_RESAMPLE_CATMULL_ROM><<<(unsigned)blocks, kThreads, 0, st>>>(s, qx, qy, m,
                                                                                     out, how);
    else
        k_resample_pts<BG_RESAMPLE_BILINEAR><<<(unsigned)blocks, kThreads, 0, st>>>(s, qx, qy, m,
                                                                                  out, how);
    note_launches(1);
    BG_CUDA(cudaGetLastError());
    return BG_OK;
}

bg_status launch_resample_grid(const float* src, const GridView& g, int method, const GridView& o,
                               float* out, int8_t* how, cudaStream_t st) {
    const Src s{src, g.x0 + g.cell / 2, g.y0 + g.cell / 2, g.cell, g.nx, g.ny, 1.0f / (float)g.cell};
    // output columns on node columns of the source: the column case only
    const int64_t off = (int64_t)o.x0 + o.cell / 2 - s.cx0;
    const bool colx = o.cell % s.cell == 0 && ((off % s.cell) + s.cell) % s.cell == 0;
    const int64_t d = off / s.cell;  // source column of output column 0, when colx
    if (colx && o.cell == s.cell && ((d % kVec) + kVec) % kVec == 0 && g.nx % kVec == 0 &&
        o.nx % kVec == 0 && (uintptr_t)src % 16 == 0 && (uintptr_t)out % 16 == 0 &&
        (uintptr_t)how % 4 == 0) {
        const int per = kThreads * kVec * kVecGroups;
        const int chunks = (o.nx + per - 1) / per;
        const int64_t blocks = (int64_t)chunks * ((o.ny + kRowsPerBlock - 1) / kRowsPerBlock);
        if (blocks >= ((int64_t)1 << 31)) {
            set_error("output grid too large for one launch");
            return BG_ERR_INVALID_ARG;
        }
        if (method == BG_RESAMPLE_CATMULL_ROM)
            k_resample_rows<BG_RESAMPLE_CATMULL_ROM><<<(unsigned)blocks, kThreads, 0, st>>>(
                s, o, d, chunks, out, how);
        else
            k_resample_rows<BG_RESAMPLE_BILINEAR><<<(unsigned)blocks, kThreads, 0, st>>>(
                s, o, d, chunks, out, how);
        note_launches(1);
        BG_CUDA(cudaGetLastError());
        return BG_OK;
    }
    const int chunks = (o.nx + kThreads * kPer - 1) / (kThreads * kPer);
    const int64_t blocks = (int64_t)chunks * ((o.ny + kRowsPerBlock - 1) / kRowsPerBlock);
    if (blocks >= ((int64_t)1 << 31)) {
        set_error("output grid too large for one launch");
        return BG_ERR_INVALID_ARG;
    }
    const unsigned nb = (unsigned)blocks;
    if (method == BG_RESAMPLE_CATMULL_ROM) {
        if (colx)
            k_resample_grid<BG_RESAMPLE_CATMULL_ROM, true><<<nb, kThreads, 0, st>>>(s, o, chunks, out, how);
        else
            k_resample_grid<BG_RESAMPLE_CATMULL_ROM, false><<<nb, kThreads, 0, st>>>(s, o, chunks, out, how);
    } else {
        k_resample_grid<BG_RESAMPLE_BILINEAR, false><<<nb, kThreads, 0, st>>>(s, o, chunks, out, how);
    }
    note_launches(1);
    BG_CUDA(cudaGetLastError());
    return BG_OK;
}

}  // namespace bg
