/*
 * Plain FP64 CPU oracle for scattered-sounding gridding.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the product path may link, load or
 * call this file; only the test suite, the smoke check and the CPU-baseline
 * leg of the benchmark use it. It shares no code, header or constant with
 * the CUDA library.
 *
 * What it computes, in the order the method defines it:
 *   - exact k nearest neighbours of a grid node by brute force: every valid
 *     sounding (depth not NaN, the "valid candidate neighbours" of Sec. III-B
 *     and III-D) ranked by (squared distance in int64 cm^2, upload index);
 *     for large inputs the same k smallest (d2, index) pairs come from a 2-d
 *     tree (median splits, bounding boxes, lexicographic insertion), which
 *     the tests hold equal to the brute force;
 *   - inverse-distance weighting over those neighbours in FP64;
 *   - local ordinary kriging (Sec. III-C): the variogram gamma(h) of the
 *     neighbours, the bordered system [Gamma 1; 1^T 0][lambda; mu] =
 *     [gamma_0; 1] solved by Gaussian elimination with partial pivoting
 *     (the solver Sec. III-C names), the estimate sum(lambda_i z_i)
 *     (Sec. III-C, estimate equation) and the kriging variance
 *     sum(lambda_i gamma_i0) + mu.
 *
 * Readings where the paper is silent (all listed in the design notes):
 *   - the paper prints only the exponential model C0 (1 - exp(-h/a))
 *     (Sec. III-C, variogram equation); the spherical model with a nugget is
 *     added, and "sill" is the total sill c0 + c;
 *   - distinct soundings at one position have gamma = c0 (the h -> 0+ limit),
 *     gamma_ii = 0, and a node on top of a sounding has gamma_0i = 0;
 *   - the kriging system is the textbook one with the Lagrange row, which
 *     the printed matrix equation of Sec. III-C omits;
 *   - fewer valid soundings than k: k_eff = min(k, N_valid); none gives NaN.
 *
 *
 * Gridded input (the paper's own stencil methods, Sec. III-A and III-B):
 *   - bilinear interpolation of a regular grid at a query point from the
 *     four nodes of the cell that holds it (Sec. III-A, the formula with
 *     (x2 - x)(y2 - y) Q11 + ... over (x2 - x1)(y2 - y1));
 *   - Catmull-Rom: the 4 x 4 nodes around that cell, the cubic C(t) of
 *     Sec. III-B applied along x on each of the 4 rows, then along y.
 *   Readings: a node is needed when its weight is not zero (a query on a
 *   node line needs only that line); a needed NaN node makes bilinear NaN
 *   (it has no fallback, Sec. III-D) and sends Catmull-Rom to bilinear
 *   (Sec. III-B, read as "if not enough valid neighbours"); stencil indices
 *   past the grid edge repeat the edge node; a query outside the hull of
 *   the node centres gets NaN.
 *
 * Build: gcc -O2 -std=c11 -shared -fPIC -pthread oracle.c -o liboracle.so -lm
 * (no -ffast-math: the NaN tests and the rounding of every step must be IEEE).
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#define ORACLE_SPHERICAL 0
#define ORACLE_EXPONENTIAL 1

/* ---------------------------------------------------------------- helpers */

static int default_threads(int requested) {
    if (requested > 0) return requested;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

typedef void (*range_fn)(void* arg, int64_t lo, int64_t hi);

typedef struct {
    range_fn fn;
    void* arg;
    int64_t lo, hi;
} range_job;

static void* range_thread(void* p) {
    range_job* j = (range_job*)p;
    j->fn(j->arg, j->lo, j->hi);
    return NULL;
}

/* Run fn over [0, m) split into contiguous chunks, one per thread. */
static void parallel_for(int64_t m, int nthreads, range_fn fn, void* arg) {
    nthreads = default_threads(nthreads);
    if (nthreads > m) nthreads = (int)(m > 0 ? m : 1);
    if (nthreads <= 1) {
        fn(arg, 0, m);
        return;
    }
    pthread_t* th = (pthread_t*)malloc(sizeof(pthread_t) * nthreads);
    range_job* jobs = (range_job*)malloc(sizeof(range_job) * nthreads);
    char* live = (char*)calloc(nthreads, 1);
    int64_t chunk = (m + nthreads - 1) / nthreads;
    for (int t = 0; t < nthreads; ++t) {
        int64_t lo = t * chunk, hi = lo + chunk < m ? lo + chunk : m;
        jobs[t].fn = fn;
        jobs[t].arg = arg;
        jobs[t].lo = lo;
        jobs[t].hi = hi;
        if (lo >= hi) continue;
        if (pthread_create(&th[t], NULL, range_thread, &jobs[t]) == 0)
            live[t] = 1;
        else
            fn(arg, lo, hi); /* could not start a thread: run this chunk inline */
    }
    for (int t = 0; t < nthreads; ++t)
        if (live[t]) pthread_join(th[t], NULL);
    free(live);
    free(th);
    free(jobs);
}

/* ------------------------------------------------------------ grid nodes */

/* Node (i, j) of a regular grid sits at the centre of pixel (i, j):
 * x = x0 + i*cell + cell/2, y = y0 + j*cell + cell/2 (cm); row-major j*nx+i. */
void oracle_grid_nodes(int32_t x0, int32_t y0, int32_t cell, int32_t nx, int32_t ny,
                       int32_t* qx, int32_t* qy) {
    for (int64_t j = 0; j < ny; ++j)
        for (int64_t i = 0; i < nx; ++i) {
            qx[j * nx + i] = (int32_t)(x0 + i * cell + cell / 2);
            qy[j * nx + i] = (int32_t)(y0 + j * cell + cell / 2);
        }
}

/* -------------------------------------------------------------------- kNN */

/* The k smallest (d2, index) pairs over all valid soundings, ascending.
 * Soundings are visited in index order, so among equal d2 the earlier index
 * is kept and stays in front. Returns k_eff. */
static int knn_one(const int32_t* x, const int32_t* y, const float* z, int64_t n,
                   int32_t qx, int32_t qy, int k, int32_t* bi, int64_t* bd) {
    int cnt = 0;
    for (int64_t p = 0; p < n; ++p) {
        if (isnan(z[p])) continue;
        int64_t dx = (int64_t)x[p] - (int64_t)qx;
        int64_t dy = (int64_t)y[p] - (int64_t)qy;
        int64_t d2 = dx * dx + dy * dy;
        if (cnt == k && d2 >= bd[k - 1]) continue;
        int i = cnt < k ? cnt : k - 1;
        while (i > 0 && bd[i - 1] > d2) {
            bd[i] = bd[i - 1];
            bi[i] = bi[i - 1];
            --i;
        }
        bd[i] = d2;
        bi[i] = (int32_t)p;
        if (cnt < k) ++cnt;
    }
    for (int i = cnt; i < k; ++i) {
        bd[i] = -1;
        bi[i] = -1;
    }
    return cnt;
}

/* ---------------------------------------------------------- 2-d tree */

/* A 2-d tree over the valid soundings: the same k smallest (d2, index) pairs
 * as knn_one, found without visiting every sounding. Build: the points of a
 * node (a contiguous range of the tree-ordered array) are split at their
 * median along the longer side of the node's bounding box; node i's children
 * are 2i + 1 (lower half) and 2i + 2. Ranges of at most TREE_LEAF points are
 * leaves. Query: visit the nearer child first and skip a node whose box lies
 * farther than the current k-th distance (a box exactly at that distance is
 * still visited: an equally distant point with a lower index would win). */
#define TREE_LEAF 8

typedef struct {
    int32_t x, y, id;
} tree_pt;

typedef struct {
    int64_t n;        /* valid soundings in the tree */
    tree_pt* pt;      /* tree order */
    int32_t* box;     /* 4 per node: x0, y0, x1, y1 (inclusive) */
    int64_t nodes;    /* node slots (heap numbering) */
} oracle_tree;

static int32_t pt_key(const tree_pt* p, int axis) { return axis ? p->y : p->x; }

/* Reorder a[lo, hi) so that a[mid] holds the element of rank mid - lo along
 * the axis, with no larger key before it and no smaller after it. Each round
 * splits the range three ways around a pivot key taken from it (below, equal,
 * above); the equal part is never empty, so every round shrinks the range. */
static void select_median(tree_pt* a, int64_t lo, int64_t hi, int64_t mid, int axis) {
    while (hi - lo > 1) {
        const int32_t k0 = pt_key(&a[lo], axis), k1 = pt_key(&a[lo + (hi - lo) / 2], axis);
        const int32_t k2 = pt_key(&a[hi - 1], axis);
        const int32_t piv = k0 < k1 ? (k1 < k2 ? k1 : (k0 < k2 ? k2 : k0))
                                    : (k0 < k2 ? k0 : (k1 < k2 ? k2 : k1));
        int64_t lt = lo, i = lo, gt = hi;  /* [lo, lt) < piv, [lt, i) = piv, [gt, hi) > piv */
        while (i < gt) {
            const int32_t key = pt_key(&a[i], axis);
            if (key < piv) {
                tree_pt t = a[lt];
                a[lt++] = a[i];
                a[i++] = t;
            } else if (key > piv) {
                tree_pt t = a[--gt];
                a[gt] = a[i];
                a[i] = t;
            } else {
                ++i;
            }
        }
        if (mid < lt) hi = lt;
        else if (mid >= gt) lo = gt;
        else return;
    }
}

typedef struct {
    oracle_tree* t;
    int64_t node, lo, hi;
    int depth, spawn_depth;
} build_job;

static void* build_node(void* p);

static void build_range(oracle_tree* t, int64_t node, int64_t lo, int64_t hi, int depth,
                        int spawn_depth) {
    int32_t x0 = INT32_MAX, y0 = INT32_MAX, x1 = INT32_MIN, y1 = INT32_MIN;
    for (int64_t j = lo; j < hi; ++j) {
        const tree_pt* q = &t->pt[j];
        if (q->x < x0) x0 = q->x;
        if (q->x > x1) x1 = q->x;
        if (q->y < y0) y0 = q->y;
        if (q->y > y1) y1 = q->y;
    }
    int32_t* b = t->box + 4 * node;
    b[0] = x0;
    b[1] = y0;
    b[2] = x1;
    b[3] = y1;
    if (hi - lo <= TREE_LEAF) return;
    const int axis = ((int64_t)y1 - y0) > ((int64_t)x1 - x0) ? 1 : 0;
    const int64_t mid = lo + (hi - lo) / 2;
    select_median(t->pt, lo, hi, mid, axis);
    /* the two halves are disjoint: near the root, build the lower one on a new thread */
    if (depth < spawn_depth) {
        build_job job = {t, 2 * node + 1, lo, mid, depth + 1, spawn_depth};
        pthread_t th;
        if (pthread_create(&th, NULL, build_node, &job) == 0) {
            build_range(t, 2 * node + 2, mid, hi, depth + 1, spawn_depth);
            pthread_join(th, NULL);
            return;
        }
    }
    build_range(t, 2 * node + 1, lo, mid, depth + 1, spawn_depth);
    build_range(t, 2 * node + 2, mid, hi, depth + 1, spawn_depth);
}

static void* build_node(void* p) {
    build_job* j = (build_job*)p;
    build_range(j->t, j->node, j->lo, j->hi, j->depth, j->spawn_depth);
    return NULL;
}

void oracle_tree_free(void* p) {
    oracle_tree* t = (oracle_tree*)p;
    if (!t) return;
    free(t->pt);
    free(t->box);
    free(t);
}

/* Build the tree over the valid soundings of (x, y, z) on up to nthreads
 * threads (0: every online core). Returns NULL when memory runs out. The tree
 * keeps copies of the coordinates and upload indices; queries still read
 * depths from the caller's arrays. */
void* oracle_tree_build(const int32_t* x, const int32_t* y, const float* z, int64_t n,
                        int nthreads) {
    oracle_tree* t = (oracle_tree*)calloc(1, sizeof(oracle_tree));
    if (!t || n < 0) {
        free(t);
        return NULL;
    }
    int64_t nv = 0;
    for (int64_t p = 0; p < n; ++p)
        if (!isnan(z[p])) ++nv;
    t->n = nv;
    t->pt = (tree_pt*)malloc(sizeof(tree_pt) * (size_t)(nv > 0 ? nv : 1));
    /* the largest range at depth d holds ceil(nv / 2^d) points */
    int depth = 0;
    for (int64_t s = nv; s > TREE_LEAF; s = (s + 1) / 2) ++depth;
    t->nodes = nv > 0 ? ((int64_t)1 << (depth + 1)) - 1 : 0;
    t->box = (int32_t*)malloc(sizeof(int32_t) * 4 * (size_t)(t->nodes > 0 ? t->nodes : 1));
    if (!t->pt || !t->box) {
        oracle_tree_free(t);
        return NULL;
    }
    int64_t j = 0;
    for (int64_t p = 0; p < n; ++p)
        if (!isnan(z[p])) {
            t->pt[j].x = x[p];
            t->pt[j].y = y[p];
            t->pt[j].id = (int32_t)p;
            ++j;
        }
    int spawn_depth = 0;
    for (int th = default_threads(nthreads); th > 1; th >>= 1) ++spawn_depth;
    if (nv > 0) build_range(t, 0, 0, nv, 0, spawn_depth);
    return t;
}

/* Keep the k smallest (d2, index) pairs in ascending order in bd/bi. */
static void insert_lex(int k, int* cnt, int32_t* bi, int64_t* bd, int64_t d2, int32_t id) {
    if (*cnt == k && (d2 > bd[k - 1] || (d2 == bd[k - 1] && id > bi[k - 1]))) return;
    int i = *cnt < k ? *cnt : k - 1;
    while (i > 0 && (bd[i - 1] > d2 || (bd[i - 1] == d2 && bi[i - 1] > id))) {
        bd[i] = bd[i - 1];
        bi[i] = bi[i - 1];
        --i;
    }
    bd[i] = d2;
    bi[i] = id;
    if (*cnt < k) ++*cnt;
}

/* Squared distance from (qx, qy) to the nearest point of a node's box. */
static int64_t box_d2(const int32_t* b, int32_t qx, int32_t qy) {
    int64_t dx = 0, dy = 0;
    if (qx < b[0]) dx = (int64_t)b[0] - qx;
    else if (qx > b[2]) dx = (int64_t)qx - b[2];
    if (qy < b[1]) dy = (int64_t)b[1] - qy;
    else if (qy > b[3]) dy = (int64_t)qy - b[3];
    return dx * dx + dy * dy;
}

static void tree_visit(const oracle_tree* t, int64_t node, int64_t lo, int64_t hi, int32_t qx,
                       int32_t qy, int k, int* cnt, int32_t* bi, int64_t* bd) {
    if (*cnt == k && box_d2(t->box + 4 * node, qx, qy) > bd[k - 1]) return;
    if (hi - lo <= TREE_LEAF) {
        for (int64_t j = lo; j < hi; ++j) {
            const tree_pt* q = &t->pt[j];
            const int64_t dx = (int64_t)q->x - qx, dy = (int64_t)q->y - qy;
            insert_lex(k, cnt, bi, bd, dx * dx + dy * dy, q->id);
        }
        return;
    }
    const int64_t mid = lo + (hi - lo) / 2, l = 2 * node + 1, r = 2 * node + 2;
    if (box_d2(t->box + 4 * l, qx, qy) <= box_d2(t->box + 4 * r, qx, qy)) {
        tree_visit(t, l, lo, mid, qx, qy, k, cnt, bi, bd);
        tree_visit(t, r, mid, hi, qx, qy, k, cnt, bi, bd);
    } else {
        tree_visit(t, r, mid, hi, qx, qy, k, cnt, bi, bd);
        tree_visit(t, l, lo, mid, qx, qy, k, cnt, bi, bd);
    }
}

static int tree_knn_one(const oracle_tree* t, int32_t qx, int32_t qy, int k, int32_t* bi,
                        int64_t* bd) {
    int cnt = 0;
    if (t->n > 0) tree_visit(t, 0, 0, t->n, qx, qy, k, &cnt, bi, bd);
    for (int i = cnt; i < k; ++i) {
        bd[i] = -1;
        bi[i] = -1;
    }
    return cnt;
}

/* k nearest of (qx, qy): from the tree when one is given, else brute force. */
static int nearest(const oracle_tree* t, const int32_t* x, const int32_t* y, const float* z,
                   int64_t n, int32_t qx, int32_t qy, int k, int32_t* bi, int64_t* bd) {
    return t ? tree_knn_one(t, qx, qy, k, bi, bd) : knn_one(x, y, z, n, qx, qy, k, bi, bd);
}

typedef struct {
    const int32_t *x, *y;
    const float* z;
    int64_t n;
    const int32_t *qx, *qy;
    int k;
    int32_t* idx;
    int64_t* d2;
    int32_t* keff;
    const oracle_tree* tree;
} knn_args;

static void knn_range(void* p, int64_t lo, int64_t hi) {
    knn_args* a = (knn_args*)p;
    for (int64_t q = lo; q < hi; ++q) {
        int c = nearest(a->tree, a->x, a->y, a->z, a->n, a->qx[q], a->qy[q], a->k,
                        a->idx + q * a->k, a->d2 + q * a->k);
        if (a->keff) a->keff[q] = c;
    }
}

/* tree: NULL for brute force, else a tree built from the same x, y, z. */
int oracle_knn(const int32_t* x, const int32_t* y, const float* z, int64_t n,
               const int32_t* qx, const int32_t* qy, int64_t m, int k,
               int32_t* idx_out, int64_t* d2_out, int32_t* keff_out, int nthreads,
               const void* tree) {
    if (k <= 0 || n < 0 || m < 0) return -1;
    knn_args a = {x, y, z, n, qx, qy, k, idx_out, d2_out, keff_out, (const oracle_tree*)tree};
    parallel_for(m, nthreads, knn_range, &a);
    return 0;
}

/* -------------------------------------------------------------------- IDW */

/* IDW over the k nearest: w_i = (d_i)^-p with d in metres (scale-free, the
 * units cancel in the ratio); zhat = sum w_i z_i / sum w_i. A node on top of
 * a sounding returns that sounding's depth (the nearest one, lowest index). */
static double idw_one(const float* z, const int32_t* bi, const int64_t* bd, int keff,
                      double power) {
    if (keff == 0) return NAN;
    if (bd[0] == 0) return (double)z[bi[0]];
    double num = 0.0, den = 0.0;
    for (int i = 0; i < keff; ++i) {
        double d2_m2 = (double)bd[i] / 1.0e4;
        double w = (power == 2.0) ? 1.0 / d2_m2 : pow(d2_m2, -0.5 * power);
        num += w * (double)z[bi[i]];
        den += w;
    }
    return num / den;
}

typedef struct {
    const int32_t *x, *y;
    const float* z;
    int64_t n;
    const int32_t *qx, *qy;
    int k;
    double power;
    double* depth;
    int32_t* idx;
    const oracle_tree* tree;
} idw_args;

static void idw_range(void* p, int64_t lo, int64_t hi) {
    idw_args* a = (idw_args*)p;
    int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * a->k);
    int64_t* bd = (int64_t*)malloc(sizeof(int64_t) * a->k);
    for (int64_t q = lo; q < hi; ++q) {
        int c = nearest(a->tree, a->x, a->y, a->z, a->n, a->qx[q], a->qy[q], a->k, bi, bd);
        a->depth[q] = idw_one(a->z, bi, bd, c, a->power);
        if (a->idx) memcpy(a->idx + q * a->k, bi, sizeof(int32_t) * a->k);
    }
    free(bi);
    free(bd);
}

int oracle_idw(const int32_t* x, const int32_t* y, const float* z, int64_t n,
               const int32_t* qx, const int32_t* qy, int64_t m, int k, double power,
               double* depth_out, int32_t* idx_out, int nthreads, const void* tree) {
    if (k <= 0 || n < 0 || m < 0 || !(power > 0.0)) return -1;
    idw_args a = {x, y, z, n, qx, qy, k, power, depth_out, idx_out, (const oracle_tree*)tree};
    parallel_for(m, nthreads, idw_range, &a);
    return 0;
}

/* ---------------------------------------------------------------- kriging */

/* Variogram at separation h metres (h > 0). Spherical: c0 + c (1.5 h/a -
 * 0.5 (h/a)^3) up to the range, c0 + c beyond. Exponential (Sec. III-C):
 * c0 + c (1 - exp(-h/a)). c = sill - nugget (sill is the total sill). */
double oracle_variogram(int model, double nugget, double sill, double range_m, double h) {
    double c = sill - nugget;
    if (model == ORACLE_SPHERICAL) {
        if (h >= range_m) return sill;
        double t = h / range_m;
        return nugget + c * (1.5 * t - 0.5 * t * t * t);
    }
    if (model == ORACLE_EXPONENTIAL) return nugget + c * (1.0 - exp(-h / range_m));
    return NAN;
}

/* Gaussian elimination with partial pivoting (first row of largest |a| in
 * the column), then back substitution. A is n x n row-major and is
 * overwritten, as is b. Returns -1 on an exactly zero pivot. */
int oracle_solve(int n, double* A, double* b, double* x) {
    for (int c = 0; c < n; ++c) {
        int piv = c;
        double best = fabs(A[(int64_t)c * n + c]);
        for (int r = c + 1; r < n; ++r) {
            double v = fabs(A[(int64_t)r * n + c]);
            if (v > best) {
                best = v;
                piv = r;
            }
        }
        if (best == 0.0) return -1;
        if (piv != c) {
            for (int j = 0; j < n; ++j) {
                double t = A[(int64_t)c * n + j];
                A[(int64_t)c * n + j] = A[(int64_t)piv * n + j];
                A[(int64_t)piv * n + j] = t;
            }
            double t = b[c];
            b[c] = b[piv];
            b[piv] = t;
        }
        for (int r = c + 1; r < n; ++r) {
            double f = A[(int64_t)r * n + c] / A[(int64_t)c * n + c];
            for (int j = c; j < n; ++j) A[(int64_t)r * n + j] -= f * A[(int64_t)c * n + j];
            b[r] -= f * b[c];
        }
    }
    for (int r = n - 1; r >= 0; --r) {
        double s = b[r];
        for (int j = r + 1; j < n; ++j) s -= A[(int64_t)r * n + j] * x[j];
        x[r] = s / A[(int64_t)r * n + r];
    }
    return 0;
}

/* Ordinary kriging at node (qx, qy) from its keff nearest soundings.
 * Writes depth, variance and (optionally) lambda[keff], mu. */
static void okrige_one(const int32_t* x, const int32_t* y, const float* z,
                       const int32_t* bi, const int64_t* bd,
                       int keff, int model, double nugget, double sill, double range_m,
                       double* A, double* b, double* sol,
                       double* depth, double* var, double* lam, double* mu) {
    if (keff == 0) {
        *depth = NAN;
        *var = NAN;
        if (mu) *mu = NAN;
        return;
    }
    int n = keff + 1;
    for (int i = 0; i < keff; ++i) {
        for (int j = 0; j < keff; ++j) {
            double g;
            if (i == j) {
                g = 0.0;
            } else {
                int64_t dx = (int64_t)x[bi[i]] - x[bi[j]];
                int64_t dy = (int64_t)y[bi[i]] - y[bi[j]];
                int64_t d2 = dx * dx + dy * dy;
                g = d2 == 0 ? nugget
                            : oracle_variogram(model, nugget, sill, range_m, sqrt((double)d2) / 100.0);
            }
            A[(int64_t)i * n + j] = g;
        }
        A[(int64_t)i * n + keff] = 1.0;
        A[(int64_t)keff * n + i] = 1.0;
        b[i] = bd[i] == 0 ? 0.0
                          : oracle_variogram(model, nugget, sill, range_m, sqrt((double)bd[i]) / 100.0);
    }
    A[(int64_t)keff * n + keff] = 0.0;
    b[keff] = 1.0;
    double g0[256 + 1];
    double* gam0 = keff <= 256 ? g0 : (double*)malloc(sizeof(double) * keff);
    for (int i = 0; i < keff; ++i) gam0[i] = b[i];
    if (oracle_solve(n, A, b, sol) != 0) {
        *depth = NAN;
        *var = NAN;
        if (mu) *mu = NAN;
        if (gam0 != g0) free(gam0);
        return;
    }
    double zh = 0.0, v = 0.0;
    for (int i = 0; i < keff; ++i) {
        zh += sol[i] * (double)z[bi[i]];
        v += sol[i] * gam0[i];
        if (lam) lam[i] = sol[i];
    }
    v += sol[keff];
    *depth = zh;
    *var = v;
    if (mu) *mu = sol[keff];
    if (gam0 != g0) free(gam0);
}

typedef struct {
    const int32_t *x, *y;
    const float* z;
    int64_t n;
    const int32_t *qx, *qy;
    int k, model;
    double nugget, sill, range_m;
    double *depth, *var, *lam, *mu;
    int32_t* idx;
    const oracle_tree* tree;
} ok_args;

static void ok_range(void* p, int64_t lo, int64_t hi) {
    ok_args* a = (ok_args*)p;
    int k = a->k;
    int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * k);
    int64_t* bd = (int64_t*)malloc(sizeof(int64_t) * k);
    double* A = (double*)malloc(sizeof(double) * (k + 1) * (k + 1));
    double* b = (double*)malloc(sizeof(double) * (k + 1));
    double* s = (double*)malloc(sizeof(double) * (k + 1));
    for (int64_t q = lo; q < hi; ++q) {
        int c = nearest(a->tree, a->x, a->y, a->z, a->n, a->qx[q], a->qy[q], k, bi, bd);
        double* lam = a->lam ? a->lam + q * k : NULL;
        if (lam)
            for (int i = 0; i < k; ++i) lam[i] = 0.0;
        okrige_one(a->x, a->y, a->z, bi, bd, c, a->model, a->nugget,
                   a->sill, a->range_m, A, b, s, a->depth + q, a->var + q, lam,
                   a->mu ? a->mu + q : NULL);
        if (a->idx) memcpy(a->idx + q * k, bi, sizeof(int32_t) * k);
    }
    free(bi);
    free(bd);
    free(A);
    free(b);
    free(s);
}

int oracle_okrige(const int32_t* x, const int32_t* y, const float* z, int64_t n,
                  const int32_t* qx, const int32_t* qy, int64_t m, int k, int model,
                  double nugget, double sill, double range_m, double* depth_out,
                  double* var_out, double* lambda_out, double* mu_out, int32_t* idx_out,
                  int nthreads, const void* tree) {
    if (k <= 0 || n < 0 || m < 0) return -1;
    if (model != ORACLE_SPHERICAL && model != ORACLE_EXPONENTIAL) return -1;
    if (!(range_m > 0.0) || nugget < 0.0 || !(sill > nugget)) return -1;
    ok_args a = {x, y, z, n, qx, qy, k, model, nugget, sill, range_m,
                 depth_out, var_out, lambda_out, mu_out, idx_out, (const oracle_tree*)tree};
    parallel_for(m, nthreads, ok_range, &a);
    return 0;
}

/* ------------------------------------------------------ gridded input */

/* The cell of the node lattice that holds query offset u (cm from the first
 * node centre) along an axis of n nodes at spacing cell: index i in
 * [0, n - 2] and remainder r in [0, cell] with u = i * cell + r; -1 outside. */
static int lattice_cell(int64_t u, int64_t cell, int n, int64_t* r) {
    if (u < 0 || u > (int64_t)(n - 1) * cell) return -1;
    int64_t i = u / cell;
    if (i > n - 2) i = n - 2;
    *r = u - i * cell;
    return (int)i;
}

/* Bilinear (Sec. III-A) at (qx, qy): Q11, Q21, Q12, Q22 are the nodes at
 * (x1, y1), (x2, y1), (x1, y2), (x2, y2). Returns NaN when a node whose
 * weight is not zero is NaN, or outside the hull. */
static double bilinear_one(const float* v, int64_t x0, int64_t y0, int64_t cell, int nx, int ny,
                           int64_t qx, int64_t qy) {
    int64_t rx, ry;
    const int i = lattice_cell(qx - (x0 + cell / 2), cell, nx, &rx);
    const int j = lattice_cell(qy - (y0 + cell / 2), cell, ny, &ry);
    if (i < 0 || j < 0) return NAN;
    const double x1 = (double)(x0 + cell / 2 + (int64_t)i * cell), x2 = x1 + (double)cell;
    const double y1 = (double)(y0 + cell / 2 + (int64_t)j * cell), y2 = y1 + (double)cell;
    const double x = (double)qx, y = (double)qy;
    const double q11 = v[(int64_t)j * nx + i], q21 = v[(int64_t)j * nx + i + 1];
    const double q12 = v[(int64_t)(j + 1) * nx + i], q22 = v[(int64_t)(j + 1) * nx + i + 1];
    const double w11 = (x2 - x) * (y2 - y), w21 = (x - x1) * (y2 - y);
    const double w12 = (x2 - x) * (y - y1), w22 = (x - x1) * (y - y1);
    const double q[4] = {q11, q21, q12, q22}, w[4] = {w11, w21, w12, w22};
    double acc = 0.0;
    for (int c = 0; c < 4; ++c) {
        if (w[c] == 0.0) continue;  /* not needed */
        if (isnan(q[c])) return NAN;
        acc += w[c] * q[c];
    }
    return acc / ((x2 - x1) * (y2 - y1));
}

/* The Catmull-Rom cubic of Sec. III-B through P1 (t = 0) and P2 (t = 1). */
static double catmull_rom_1d(double p0, double p1, double p2, double p3, double t) {
    return 0.5 * (2.0 * p1 + (-p0 + p2) * t + (2.0 * p0 - 5.0 * p1 + 4.0 * p2 - p3) * t * t +
                  (-p0 + 3.0 * p1 - 3.0 * p2 + p3) * t * t * t);
}

/* Which of P0..P3 carry weight at t: all four inside the cell, only P1 at
 * t = 0, only P2 at t = 1 (the cubic's weights vanish nowhere else in [0, 1]). */
static void cr_needed(int64_t r, int64_t cell, int need[4]) {
    for (int a = 0; a < 4; ++a) need[a] = (r == 0) ? (a == 1) : (r == cell) ? (a == 2) : 1;
}

static int clampi(int v, int lo, int hi) { return v < lo ? lo : (v > hi ? hi : v); }

/* Catmull-Rom at (qx, qy); *how = 0 cubic, 1 bilinear fallback, 2 no value. */
static double catmull_rom_one(const float* v, int64_t x0, int64_t y0, int64_t cell, int nx,
                              int ny, int64_t qx, int64_t qy, int8_t* how) {
    int64_t rx, ry;
    const int i = lattice_cell(qx - (x0 + cell / 2), cell, nx, &rx);
    const int j = lattice_cell(qy - (y0 + cell / 2), cell, ny, &ry);
    if (i < 0 || j < 0) {
        *how = 2;
        return NAN;
    }
    int nxd[4], nyd[4];
    cr_needed(rx, cell, nxd);
    cr_needed(ry, cell, nyd);
    double P[4][4];  /* P[b][a]: row j - 1 + b, column i - 1 + a (edges repeated) */
    int ok = 1;
    for (int b = 0; b < 4; ++b)
        for (int a = 0; a < 4; ++a) {
            const int ii = clampi(i - 1 + a, 0, nx - 1), jj = clampi(j - 1 + b, 0, ny - 1);
            const double val = v[(int64_t)jj * nx + ii];
            if (nxd[a] && nyd[b]) {
                if (isnan(val)) ok = 0;
                P[b][a] = val;
            } else {
                P[b][a] = 0.0;  /* weight zero: the value does not enter */
            }
        }
    if (!ok) {
        const double f = bilinear_one(v, x0, y0, cell, nx, ny, qx, qy);
        *how = isnan(f) ? 2 : 1;
        return f;
    }
    const double t = (double)rx / (double)cell, s = (double)ry / (double)cell;
    double row[4];
    for (int b = 0; b < 4; ++b) row[b] = catmull_rom_1d(P[b][0], P[b][1], P[b][2], P[b][3], t);
    *how = 0;
    return catmull_rom_1d(row[0], row[1], row[2], row[3], s);
}

/* method 0 = bilinear, 1 = Catmull-Rom; how may be NULL. */
int oracle_resample(const float* v, int32_t x0, int32_t y0, int32_t cell, int32_t nx, int32_t ny,
                    int method, const int32_t* qx, const int32_t* qy, int64_t m, double* out,
                    int8_t* how) {
    if (!v || cell <= 0 || nx < 2 || ny < 2 || m < 0 || (m > 0 && (!qx || !qy || !out)) ||
        (method != 0 && method != 1))
        return -1;
    for (int64_t p = 0; p < m; ++p) {
        int8_t h = 0;
        double f;
        if (method == 0) {
            f = bilinear_one(v, x0, y0, cell, nx, ny, qx[p], qy[p]);
            h = isnan(f) ? 2 : 0;
        } else {
            f = catmull_rom_one(v, x0, y0, cell, nx, ny, qx[p], qy[p], &h);
        }
        out[p] = f;
        if (how) how[p] = h;
    }
    return 0;
}

int oracle_threads(int requested) { return default_threads(requested); }
