// Exact k-nearest-neighbour search of one grid node over the device hash.
//
// The neighbours of a node are the K smallest keys (d2, upload index), with
// d2 = dx^2 + dy^2 an exact int64 in cm^2 and ties broken by the lower upload
// index (Sec. III-D's "nearest n valid candidate neighbors", made exact).
//
// Two phases, both per thread:
//   1. Bound. With the summed-area table, find the smallest square of cells
//      around the node's cell (half-width R) that holds at least K soundings
//      (or the whole hash). Every sounding in that square is within tau0 =
//      the squared distance to the square's farthest corner, so d_K^2 <= tau0.
//   2. Scan. Visit rows of cells in order of their distance from the node,
//      and in each row only the run of cells that can hold a point with
//      d2 <= tau (one contiguous range of the cell-sorted records). tau starts
//      at tau0 and drops to the current K-th key after every row; a row whose
//      nearest edge is farther than tau ends that side. Every sounding with
//      d2 <= d_K^2 is visited, so the result is exact.
// Keys are packed as (d2 << idx_bits) | index in a uint64 when tau0 leaves
// room for it (the usual case: tau0 < 2^(64 - idx_bits)); otherwise the wide
// form keeps d2 and the index apart. Both give the same ordering.
#pragma once

#include <climits>
#include <cstdint>

#include "bg_internal.h"

namespace bg {

constexpr unsigned kFull = 0xffffffffu;

// floor(off / cs) for 0 <= off < ncx*cs (< 2^31; exact: float estimate, integer
// fix-up). 32-bit conversions only: 64-bit int <-> float conversions run on
// the FP64 pipe, a small fraction of the FP32 rate on this GPU.
__device__ __forceinline__ int cell_of(const HashView& h, int64_t off) {
    const unsigned o = (unsigned)off, cs = (unsigned)h.cs;  // c * cs < 2^32 below
    int c = max(0, __float2int_rz(__uint2float_rz(o) * h.inv_cs));
    while ((unsigned)c * cs > o) --c;
    while ((unsigned)(c + 1) * cs <= o) ++c;
    return c;
}

// Node coordinate -> hash cell, clamped into the hash.
__device__ __forceinline__ int clamp_cell(const HashView& h, int64_t off, int n) {
    if (off < 0) return 0;
    if (off >= (int64_t)n * h.cs) return n - 1;
    return cell_of(h, off);
}

// An upper bound on floor(sqrt(v)) for 0 <= v < 2^62; 32-bit conversions
// whenever v < 2^31 (the usual case: neighbour radii below ~460 m).
__device__ __forceinline__ int64_t isqrt_ub(int64_t v) {
    if (v < ((int64_t)1 << 31)) {
        const float f = sqrtf(__int2float_ru((int)v));
        return (int64_t)__float2int_ru(f * 1.0000020f) + 1;
    }
    const float f = sqrtf((float)v);
    return (int64_t)(f * 1.0000020f) + 1;
}

__device__ __forceinline__ int sat_count(const HashView& h, int xa, int ya, int xb, int yb) {
    const int W = h.ncx + 1;
    const int32_t* s = h.sat;
    return __ldg(s + (yb + 1) * W + xb + 1) - __ldg(s + ya * W + xb + 1) -
           __ldg(s + (yb + 1) * W + xa) + __ldg(s + ya * W + xa);
}

// Number of rows beyond `row` in direction dir (+1 up, -1 down) that hold no
// sounding within cell columns [ca, cb], up to `limit` rows: doubling then
// bisection over summed-area-table counts of the band next to the row.
__device__ __forceinline__ int empty_rows_beyond(const HashView& h, int row, int dir, int ca,
                                                 int cb, int limit) {
    auto band_empty = [&](int m) {  // rows row+dir .. row+dir*m
        const int ra = dir > 0 ? row + 1 : row - m, rb = dir > 0 ? row + m : row - 1;
        return sat_count(h, ca, ra, cb, rb) == 0;
    };
    int lo = 0, hi = 1;  // band of lo rows empty; band of hi rows not (or past limit)
    while (hi <= limit && band_empty(hi)) {
        lo = hi;
        hi = 2 * hi;
    }
    hi = min(hi, limit + 1);
    while (hi - lo > 1) {
        const int mid = (lo + hi) >> 1;
        if (band_empty(mid))
            lo = mid;
        else
            hi = mid;
    }
    return lo;
}

struct Bound {
    int64_t tau0;   // d_K^2 <= tau0
    int cy;         // the node's (clamped) cell row
    int count;      // soundings in the table's square (0: unknown)
    int64_t area;   // its area in cm^2
};

// Phase 1: the smallest square around the node's cell holding >= kc soundings.
__device__ __forceinline__ Bound knn_bound_rt(const HashView& h, int qx, int qy, int kc) {
    const int cx = clamp_cell(h, (int64_t)qx - h.hx0, h.ncx);
    const int cy = clamp_cell(h, (int64_t)qy - h.hy0, h.ncy);
    const int rmax = max(max(cx, h.ncx - 1 - cx), max(cy, h.ncy - 1 - cy));
    auto cnt = [&](int r) {
        return sat_count(h, max(cx - r, 0), max(cy - r, 0), min(cx + r, h.ncx - 1),
                         min(cy + r, h.ncy - 1));
    };
    int r = min(h.r0, rmax);
    int lo, hi;
    if (cnt(r) >= kc) {
        lo = -1;
        hi = r;
    } else {
        lo = r;
        hi = r;
        while (hi < rmax) {
            hi = min(2 * hi + 1, rmax);
            if (cnt(hi) >= kc) break;
            lo = hi;
        }
    }
    while (hi - lo > 1) {  // invariant: cnt(lo) < kc (or lo = -1), cnt(hi) >= kc
        const int mid = (lo + hi) >> 1;
        if (cnt(mid) >= kc)
            hi = mid;
        else
            lo = mid;
    }
    const int xa = max(cx - hi, 0), xb = min(cx + hi, h.ncx - 1);
    const int ya = max(cy - hi, 0), yb = min(cy + hi, h.ncy - 1);
    const int64_t xlo = (int64_t)h.hx0 + (int64_t)xa * h.cs;
    const int64_t xhi = (int64_t)h.hx0 + (int64_t)(xb + 1) * h.cs - 1;
    const int64_t ylo = (int64_t)h.hy0 + (int64_t)ya * h.cs;
    const int64_t yhi = (int64_t)h.hy0 + (int64_t)(yb + 1) * h.cs - 1;
    const int64_t mdx = max((int64_t)qx - xlo, xhi - (int64_t)qx);
    const int64_t mdy = max((int64_t)qy - ylo, yhi - (int64_t)qy);
    return Bound{mdx * mdx + mdy * mdy, cy, cnt(hi), (xhi - xlo + 1) * (yhi - ylo + 1)};
}

template <int K>
__device__ __forceinline__ Bound knn_bound(const HashView& h, int qx, int qy) {
    return knn_bound_rt(h, qx, qy, K);
}

// Does (tau0 + 1) << idx_bits fit in 64 bits?
__device__ __forceinline__ bool packed_fits(const HashView& h, int64_t tau0) {
    return ((uint64_t)(tau0 + 1) >> (64 - h.idx_bits)) == 0;
}

template <int K>
__device__ __forceinline__ void insert_packed(uint64_t (&key)[K], uint64_t c) {
    // precondition: c < key[K-1]; keeps key[] ascending
#pragma unroll
    for (int j = K - 1; j > 0; --j) key[j] = (c < key[j - 1]) ? key[j - 1] : ((c < key[j]) ? c : key[j]);
    key[0] = (c < key[0]) ? c : key[0];
}

__device__ __forceinline__ bool wide_less(uint64_t ad, int ai, uint64_t bd, int bi) {
    return ad < bd || (ad == bd && ai < bi);
}

template <int K>
__device__ __forceinline__ void insert_wide(uint64_t (&kd)[K], int (&ki)[K], uint64_t cd, int ci) {
#pragma unroll
    for (int j = K - 1; j > 0; --j) {
        if (wide_less(cd, ci, kd[j - 1], ki[j - 1])) {
            kd[j] = kd[j - 1];
            ki[j] = ki[j - 1];
        } else if (wide_less(cd, ci, kd[j], ki[j])) {
            kd[j] = cd;
            ki[j] = ci;
        }
    }
    if (wide_less(cd, ci, kd[0], ki[0])) {
        kd[0] = cd;
        ki[0] = ci;
    }
}

// Phase 2. On return d2o[0..keff) / ido[0..keff) hold the neighbours in
// ascending (d2, index) order; returns keff (<= K).
template <int K, bool kWide>
__device__ __forceinline__ int knn_scan(const HashView& h, int qx, int qy, const Bound& b,
                                        uint64_t (&d2o)[K], int (&ido)[K]) {
    const int bits = h.idx_bits;
    const int64_t tau0 = b.tau0;
    uint64_t key[K];   // packed form (or the d2 half of the wide form)
    int kid[kWide ? K : 1];
    const uint64_t sentinel = kWide ? (uint64_t)(tau0 + 1) : ((uint64_t)(tau0 + 1) << bits);
#pragma unroll
    for (int i = 0; i < K; ++i) key[i] = sentinel;
#pragma unroll
    for (int i = 0; i < (kWide ? K : 1); ++i) kid[i] = INT_MAX;
    int64_t tau = tau0;
    int up = b.cy, dn = b.cy - 1;
    const int64_t xmin = h.hx0;
    const int64_t xmax = (int64_t)h.hx0 + (int64_t)h.ncx * h.cs - 1;
    for (;;) {
        int64_t dyu = LLONG_MAX, dyd = LLONG_MAX;
        if (up < h.ncy) {
            const int64_t ylo = (int64_t)h.hy0 + (int64_t)up * h.cs, yhi = ylo + h.cs - 1;
            dyu = qy < ylo ? ylo - qy : (qy > yhi ? qy - yhi : 0);
        }
        if (dn >= 0) {
            const int64_t ylo = (int64_t)h.hy0 + (int64_t)dn * h.cs, yhi = ylo + h.cs - 1;
            dyd = qy < ylo ? ylo - qy : (qy > yhi ? qy - yhi : 0);
        }
        const bool take_up = dyu <= dyd;
        const int64_t dy = take_up ? dyu : dyd;
        if (dy == LLONG_MAX || dy * dy > tau) break;
        const int row = take_up ? up++ : dn--;
        const int64_t dxm = isqrt_ub(tau - dy * dy);
        const int64_t xa = max((int64_t)qx - dxm, xmin), xb = min((int64_t)qx + dxm, xmax);
        if (xa > xb) continue;
        const int ca = cell_of(h, xa - h.hx0), cb = cell_of(h, xb - h.hx0);
        const int rowbase = row * h.ncx;
        const int s = __ldg(h.cell_start + rowbase + ca);
        const int e = __ldg(h.cell_start + rowbase + cb + 1);
        const uint64_t utau = (uint64_t)tau;
        for (int p = s; p < e; ++p) {
            const int4 v = __ldg(h.rec + p);
            const int ddx = v.x - qx, ddy = v.y - qy;
            const uint64_t d2 = (uint64_t)((long long)ddx * ddx + (long long)ddy * ddy);
            if (d2 > utau) continue;
            if constexpr (kWide) {
                if (wide_less(d2, v.w, key[K - 1], kid[K - 1])) insert_wide<K>(key, kid, d2, v.w);
            } else {
                const uint64_t c = (d2 << bits) | (uint32_t)v.w;
                if (c < key[K - 1]) insert_packed<K>(key, c);
            }
        }
        int64_t kth;
        if constexpr (kWide)
            kth = (int64_t)key[K - 1];
        else
            kth = (int64_t)(key[K - 1] >> bits);
        tau = min(tau, kth);
    }
    int keff = 0;
    const uint64_t mask = (bits >= 64) ? ~0ull : ((1ull << bits) - 1);
#pragma unroll
    for (int i = 0; i < K; ++i) {
        const bool ok = key[i] < sentinel;  // every real key has d2 <= tau0
        if constexpr (kWide) {
            d2o[i] = key[i];
            ido[i] = ok ? kid[i] : -1;
        } else {
            d2o[i] = key[i] >> bits;
            ido[i] = ok ? (int)(key[i] & mask) : -1;
        }
        keff += ok ? 1 : 0;
    }
    return keff;
}

// ---------------------------------------------------------------------------
// Packed-key search with the K best kept in a per-thread max-heap in shared
// memory (element i of a thread's heap at hp[i * S], S = threads per block,
// so the warp's accesses never share a bank whatever the heap positions).
// Inserting into a full heap replaces the root and sifts it down: O(log K)
// instead of the O(K) compare-select chain of a sorted register array, which
// SIMT pays for whenever any lane of the warp inserts. The heap fills by
// pushes (sift-up from the new leaf, about two levels on average): one heap
// build when the K-th key arrives would run at a different candidate in
// every lane, and the warp would execute all 32 builds one after another.

template <int S>
__device__ __forceinline__ void heap_sift_down(uint64_t* hp, int i, int n, uint64_t v) {
    for (;;) {
        const int l = 2 * i + 1;
        if (l >= n) break;
        int m = l;
        uint64_t km = hp[l * S];
        if (l + 1 < n) {
            const uint64_t kr = hp[(l + 1) * S];
            if (kr > km) {
                m = l + 1;
                km = kr;
            }
        }
        if (km < v) break;
        hp[i * S] = km;
        i = m;
    }
    hp[i * S] = v;
}

// Push v onto a max-heap of n keys (stride S): sift up from the new leaf.
template <int S>
__device__ __forceinline__ void heap_push(uint64_t* hp, int n, uint64_t v) {
    int i = n;
    while (i > 0) {
        const int p = (i - 1) >> 1;
        const uint64_t pv = hp[p * S];
        if (pv >= v) break;
        hp[i * S] = pv;
        i = p;
    }
    hp[i * S] = v;
}

// Phase 2 with the heap. On return hp[0 .. keff) holds the neighbours' packed
// keys in ascending order; returns keff (<= kc). Requires packed_fits(tau0).
template <int S, bool kSort = true>
__device__ __forceinline__ int knn_scan_heap_rt(const HashView& h, int qx, int qy, const Bound& b,
                                                uint64_t* hp, int kc) {
    const int bits = h.idx_bits;
    const int64_t tau0 = b.tau0;
    const uint64_t sentinel = (uint64_t)(tau0 + 1) << bits;
    uint64_t root = sentinel;  // the K-th best key once the heap is full
    int cnt = 0;
    int64_t tau = tau0;
    int up = b.cy, dn = b.cy - 1;
    const int64_t xmin = h.hx0;
    const int64_t xmax = (int64_t)h.hx0 + (int64_t)h.ncx * h.cs - 1;
    for (;;) {
        int64_t dyu = LLONG_MAX, dyd = LLONG_MAX;
        if (up < h.ncy) {
            const int64_t ylo = (int64_t)h.hy0 + (int64_t)up * h.cs, yhi = ylo + h.cs - 1;
            dyu = qy < ylo ? ylo - qy : (qy > yhi ? qy - yhi : 0);
        }
        if (dn >= 0) {
            const int64_t ylo = (int64_t)h.hy0 + (int64_t)dn * h.cs, yhi = ylo + h.cs - 1;
            dyd = qy < ylo ? ylo - qy : (qy > yhi ? qy - yhi : 0);
        }
        const bool take_up = dyu <= dyd;
        const int64_t dy = take_up ? dyu : dyd;
        if (dy == LLONG_MAX || dy * dy > tau) break;
        const int row = take_up ? up++ : dn--;
        const int64_t dxm = isqrt_ub(tau - dy * dy);
        const int64_t xa = max((int64_t)qx - dxm, xmin), xb = min((int64_t)qx + dxm, xmax);
        if (xa > xb) continue;
        const int ca = cell_of(h, xa - h.hx0), cb = cell_of(h, xb - h.hx0);
        const int rowbase = row * h.ncx;
        const int s = __ldg(h.cell_start + rowbase + ca);
        const int e = __ldg(h.cell_start + rowbase + cb + 1);
        if (s == e) {
            // an empty run (a node in a gap of the coverage): the rows beyond it
            // in this direction have runs within [ca, cb] (tau only shrinks and
            // dy grows), so skip the ones the table shows empty over [ca, cb]
            const int avail = take_up ? h.ncy - 1 - row : row;
            const int within = (int)min((int64_t)avail, isqrt_ub(tau) / h.cs + 1);
            const int skip = empty_rows_beyond(h, row, take_up ? 1 : -1, ca, cb, within);
            if (take_up)
                up += skip;
            else
                dn -= skip;
            continue;
        }
        const uint64_t utau = (uint64_t)tau;
        auto take = [&](const int4 v) {
            const int ddx = v.x - qx, ddy = v.y - qy;
            const uint64_t d2 = (uint64_t)((long long)ddx * ddx + (long long)ddy * ddy);
            if (d2 > utau) return;
            const uint64_t c = (d2 << bits) | (uint32_t)v.w;
            if (c < root) {
                if (cnt < kc) {
                    heap_push<S>(hp, cnt, c);
                    if (++cnt == kc) root = hp[0];
                } else {
                    heap_sift_down<S>(hp, 0, kc, c);
                    root = hp[0];
                }
            }
        };
        // two records in flight at a time (the run's loads do not depend on the heap)
        int p = s;
        for (; p + 1 < e; p += 2) {
            const int4 v0 = __ldg(h.rec + p), v1 = __ldg(h.rec + p + 1);
            take(v0);
            take(v1);
        }
        if (p < e) take(__ldg(h.rec + p));
        tau = min(tau, (int64_t)(root >> bits));
    }
    if constexpr (kSort) {  // heapsort into ascending order (else the caller drains the max-heap)
        for (int e = cnt - 1; e > 0; --e) {
            const uint64_t v = hp[e * S];
            hp[e * S] = hp[0];
            heap_sift_down<S>(hp, 0, e, v);
        }
    }
    return cnt;
}

template <int K, int S>
__device__ __forceinline__ int knn_scan_heap(const HashView& h, int qx, int qy, const Bound& b,
                                             uint64_t* hp) {
    return knn_scan_heap_rt<S>(h, qx, qy, b, hp, K);
}

// The first k ids of a thread's sorted heap (stride S) to out, -1 from cnt
// on: four ids per 16-byte store when k is a multiple of 4 and out is
// 16-byte aligned (a node's ids then never straddle a boundary), else one by
// one.
template <int S>
__device__ __forceinline__ void emit_ids(int32_t* __restrict__ out, const uint64_t* hp, int k,
                                         int cnt, uint64_t mask) {
    auto id = [&](int q) { return q < cnt ? (int)(hp[q * S] & mask) : -1; };
    if ((k & 3) == 0 && (reinterpret_cast<uintptr_t>(out) & 15) == 0) {
        for (int q = 0; q < k; q += 4)
            *reinterpret_cast<int4*>(out + q) = make_int4(id(q), id(q + 1), id(q + 2), id(q + 3));
    } else {
        for (int q = 0; q < k; ++q) out[q] = id(q);
    }
}

// Drain a full max-heap of K keys (stride S) into the ids of ascending
// order: each extraction's maximum is the id of the next slot from the end,
// written four at a time with one 16-byte store (out 16-byte aligned), so
// the heap is never written back in sorted order and read again.
template <int K, int S>
__device__ __forceinline__ void drain_ids(int32_t* __restrict__ out, uint64_t* hp, uint64_t mask) {
    static_assert(K % 4 == 0, "whole 16-byte groups");
    for (int m = K / 4 - 1; m >= 0; --m) {
        int v[4];
#pragma unroll
        for (int u = 3; u >= 0; --u) {
            const int e = 4 * m + u;  // heap size before this extraction is e + 1
            v[u] = (int)(hp[0] & mask);
            if (e > 0) heap_sift_down<S>(hp, 0, e, hp[e * S]);
        }
        *reinterpret_cast<int4*>(out + 4 * m) = make_int4(v[0], v[1], v[2], v[3]);
    }
}

// Grid node (i, j) owned by this thread inside the 16 x 8 node patch (px, py).
// Each warp covers 8 x 4 nodes, so a warp's nodes are spatially compact.
struct NodeIdx {
    int i, j;
};
__device__ __forceinline__ NodeIdx patch_node(int px, int py, int warp, int lane) {
    return NodeIdx{px * 16 + (warp & 1) * 8 + (lane & 7), py * 8 + (warp >> 1) * 4 + (lane >> 3)};
}

// ---------------------------------------------------------------------------
// Strips: a thread grids kStrip consecutive nodes along x, one after another.
// The first node's bound comes from the summed-area table. The next node is
// one grid cell further along x, so its K-th distance is at most the
// previous node's plus the cell (triangle inequality): a bound far tighter
// than the table's square, which cuts the rows and candidates visited and the
// heap inserts that are later evicted.
constexpr int kStrip = 4;

// Strip length of a launch over `nodes` grid nodes: strips of 4 save search
// work (each node bounded by the previous one's k-th distance) but leave a
// quarter of the threads, which a small grid needs more (a 256 x 256 tile:
// 0.119 ms of IDW k = 8 with strips of 4, 0.056 ms with strips of 1).
inline int strip_len_for(int64_t nodes) {
    return nodes >= ((int64_t)1 << 21) ? 4 : (nodes >= ((int64_t)1 << 19) ? 2 : 1);
}

// Strip origin of this thread in the (16 * kLen) x 8 node patch (px, py).
template <int kLen = kStrip>
__device__ __forceinline__ NodeIdx strip_origin(int px, int py, int warp, int lane) {
    return NodeIdx{px * 16 * kLen + (warp & 1) * 8 * kLen + (lane & 7) * kLen,
                   py * 8 + (warp >> 1) * 4 + (lane >> 3)};
}

// Packed-key k-NN of nodes (i0 .. i0 + kLen - 1, j) with the kc best in the
// shared-memory heap hp (stride S). emit(i, cnt) runs after each node with its
// keys sorted ascending in hp[0 .. cnt) (with kSort; else hp holds the max-heap);
// a node whose table bound does not fit the packed key is left to the wide
// pass (*flag = 1).
template <int S, class Emit, bool kSort = true, int kLen = kStrip>
__device__ __forceinline__ void knn_strip(const HashView& h, const GridView& g, int kc, int i0,
                                          int j, uint64_t* hp, int* flag, Emit emit) {
    const int qy = g.y0 + j * g.cell + g.cell / 2;
    int64_t prev = -1;  // K-th squared distance of the previous node, -1 if none
    int cy = 0;
    for (int s = 0; s < kLen; ++s) {
        const int i = i0 + s;
        if (i >= g.nx) break;
        const int qx = g.x0 + i * g.cell + g.cell / 2;
        Bound b{0, cy, 0, 0};
        bool ok = false;
        if (prev >= 0) {
            const int64_t r = isqrt_ub(prev) + g.cell;  // >= ceil(d_K(prev)) + |step|
            b.tau0 = r * r;
            ok = packed_fits(h, b.tau0);
        }
        bool guessed = false;
        Bound bt = b;
        if (!ok) {
            b = knn_bound_rt(h, qx, qy, kc);
            cy = b.cy;
            if (!packed_fits(h, b.tau0)) {
                *flag = 1;
                prev = -1;
                continue;
            }
            // the table's square is loose (its far corner): start instead from
            // 1.5 times the area that holds K soundings at the square's density.
            // The search is exact whenever K soundings lie within that bound
            // (everything within it is visited); otherwise it runs again from
            // the square's bound.
            bt = b;
            if (b.count > 0) {
                const float tg = 1.5f * (float)kc * (float)b.area / (3.14159265f * (float)b.count);
                if (tg < (float)b.tau0) {
                    bt.tau0 = (int64_t)tg;
                    guessed = true;
                }
            }
        }
        int cnt = knn_scan_heap_rt<S, kSort>(h, qx, qy, bt, hp, kc);
        if (guessed && cnt < kc) cnt = knn_scan_heap_rt<S, kSort>(h, qx, qy, b, hp, kc);
        // the K-th key: the last one when sorted, the root of the heap when not
        prev = cnt == kc ? (int64_t)(hp[(kSort ? kc - 1 : 0) * S] >> h.idx_bits) : -1;
        emit(i, cnt);
    }
}

// ---------------------------------------------------------------------------
// Query points instead of grid nodes. A thread takes kLen consecutive points
// of the caller's list (strip_len_for the list's length). The next point's K-th distance is at most the previous
// point's plus the distance between the two (triangle inequality); that bound
// is used when the step is no longer than the previous K-th distance (lists
// in scan order, such as the holes of a grid), else the summed-area table's.

constexpr int32_t kQueryLimit = 1 << 30;  // query coordinates lie in (-2^30, 2^30) cm

__device__ __forceinline__ bool query_in_range(int qx, int qy) {
    return qx > -kQueryLimit && qx < kQueryLimit && qy > -kQueryLimit && qy < kQueryLimit;
}

// Packed-key k-NN of points p0 .. p0 + kLen - 1 (those below m). emit(p, cnt)
// runs after each point with its keys sorted ascending in hp[0 .. cnt), or
// with cnt = -1 for a point outside the coordinate range; a point whose table
// bound does not fit the packed key is left to the wide pass (*flag = 1).
template <int S, class Emit, int kLen = kStrip>
__device__ __forceinline__ void knn_chain(const HashView& h, const int32_t* __restrict__ px,
                                          const int32_t* __restrict__ py, int64_t p0, int64_t m,
                                          int kc, uint64_t* hp, int* flag, Emit emit) {
    int64_t prev = -1;  // K-th squared distance of the previous point, -1 if none
    int qxp = 0, qyp = 0;
    for (int s = 0; s < kLen; ++s) {
        const int64_t p = p0 + s;
        if (p >= m) break;
        const int qx = __ldg(px + p), qy = __ldg(py + p);
        if (!query_in_range(qx, qy)) {
            emit(p, -1);
            prev = -1;
            continue;
        }
        Bound b{0, 0, 0, 0};
        bool ok = false;
        if (prev >= 0 && prev < ((int64_t)1 << 60)) {  // r below 2^31 + 4: r * r cannot wrap
            const int64_t dx = (int64_t)qx - qxp, dy = (int64_t)qy - qyp;
            const int64_t step2 = dx * dx + dy * dy;
            if (step2 <= prev) {
                const int64_t r = isqrt_ub(prev) + isqrt_ub(step2);  // >= d_K(prev) + |step|
                b.tau0 = r * r;
                b.cy = clamp_cell(h, (int64_t)qy - h.hy0, h.ncy);
                ok = packed_fits(h, b.tau0);
            }
        }
        if (!ok) {
            b = knn_bound_rt(h, qx, qy, kc);
            if (!packed_fits(h, b.tau0)) {
                *flag = 1;
                prev = -1;
                continue;
            }
        }
        const int cnt = knn_scan_heap_rt<S>(h, qx, qy, b, hp, kc);
        prev = cnt == kc ? (int64_t)(hp[(kc - 1) * S] >> h.idx_bits) : -1;
        qxp = qx;
        qyp = qy;
        emit(p, cnt);
    }
}

}  // namespace bg
