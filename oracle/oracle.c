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

typedef struct {
    const int32_t *x, *y;
    const float* z;
    int64_t n;
    const int32_t *qx, *qy;
    int k;
    int32_t* idx;
    int64_t* d2;
    int32_t* keff;
} knn_args;

static void knn_range(void* p, int64_t lo, int64_t hi) {
    knn_args* a = (knn_args*)p;
    for (int64_t q = lo; q < hi; ++q) {
        int c = knn_one(a->x, a->y, a->z, a->n, a->qx[q], a->qy[q], a->k,
                        a->idx + q * a->k, a->d2 + q * a->k);
        if (a->keff) a->keff[q] = c;
    }
}

int oracle_knn(const int32_t* x, const int32_t* y, const float* z, int64_t n,
               const int32_t* qx, const int32_t* qy, int64_t m, int k,
               int32_t* idx_out, int64_t* d2_out, int32_t* keff_out, int nthreads) {
    if (k <= 0 || n < 0 || m < 0) return -1;
    knn_args a = {x, y, z, n, qx, qy, k, idx_out, d2_out, keff_out};
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
} idw_args;

static void idw_range(void* p, int64_t lo, int64_t hi) {
    idw_args* a = (idw_args*)p;
    int32_t* bi = (int32_t*)malloc(sizeof(int32_t) * a->k);
    int64_t* bd = (int64_t*)malloc(sizeof(int64_t) * a->k);
    for (int64_t q = lo; q < hi; ++q) {
        int c = knn_one(a->x, a->y, a->z, a->n, a->qx[q], a->qy[q], a->k, bi, bd);
        a->depth[q] = idw_one(a->z, bi, bd, c, a->power);
        if (a->idx) memcpy(a->idx + q * a->k, bi, sizeof(int32_t) * a->k);
    }
    free(bi);
    free(bd);
}

int oracle_idw(const int32_t* x, const int32_t* y, const float* z, int64_t n,
               const int32_t* qx, const int32_t* qy, int64_t m, int k, double power,
               double* depth_out, int32_t* idx_out, int nthreads) {
    if (k <= 0 || n < 0 || m < 0 || !(power > 0.0)) return -1;
    idw_args a = {x, y, z, n, qx, qy, k, power, depth_out, idx_out};
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
        int c = knn_one(a->x, a->y, a->z, a->n, a->qx[q], a->qy[q], k, bi, bd);
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
                  int nthreads) {
    if (k <= 0 || n < 0 || m < 0) return -1;
    if (model != ORACLE_SPHERICAL && model != ORACLE_EXPONENTIAL) return -1;
    if (!(range_m > 0.0) || nugget < 0.0 || !(sill > nugget)) return -1;
    ok_args a = {x, y, z, n, qx, qy, k, model, nugget, sill, range_m,
                 depth_out, var_out, lambda_out, mu_out, idx_out};
    parallel_for(m, nthreads, ok_range, &a);
    return 0;
}

int oracle_threads(int requested) { return default_threads(requested); }
