/*
 * dfd_oracle.c -- plain, slow CPU oracle for the discrete Frechet distance.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product (the CUDA
 * library and its Python binding) never calls it, links it or shares code
 * with it: the two sides have no common kernels, headers, helpers or tables.
 *
 * What is computed (paper, Sec. 2-3): for curves p (n points) and q (m
 * points) in R^dim and the ground distance d_ij = || p_i - q_j ||, the
 * discrete Frechet distance is M_{n,m} of the recurrence of Eq. 1,
 *     M_ij = max( min(M_{i-1,j}, M_{i-1,j-1}, M_{i,j-1}), d_ij ),
 * with the first row and first column given by running maxima (Alg. 1/3).
 * Because the recurrence only selects among d values with min and max, the
 * DP over squared distances d_ij^2 returns delta^2 exactly (any nondecreasing
 * map commutes with the DP), so every function here returns the SQUARED
 * distance delta^2; callers take one square root.
 *
 * Precision: float32 input coordinates are widened exactly to float64 and
 * every step runs in float64; int32 input coordinates are widened to int64
 * and every step is exact integer arithmetic.  Build with -O2
 * -ffp-contract=off and without -ffast-math, so that the rounding of the
 * float64 sums is the plain left-to-right one on every host.
 *
 * Functions (each follows one passage of the paper):
 *   dfo_memo_*      Alg. 1 (top-down memoised recursion; explicit stack)
 *   dfo_full_*      Alg. 3 (bottom-up full matrix with the four branches)
 *   dfo_linear_*    Alg. 5 (one row of length m, branch-free)
 *   dfo_decide_*    independent check: smallest threshold eps among the
 *                   d^2 values for which a monotone coupling path of cells
 *                   with d^2 <= eps exists (Sec. 2, the frog/leash view),
 *                   found by binary search + breadth-first search
 *   dfo_hausdorff_* symmetric discrete Hausdorff distance (Sec. 2, the
 *                   lower bound the Frechet distance always meets)
 *   dfo_linear_f32mirror  Alg. 5 carried out in float32 with the squared
 *                   distance evaluated in the kernel's stated order (see
 *                   below); a selection check, not a precision reference
 *   dfo_batch_*     Alg. 5 over a list of (a, b) curve pairs, threaded
 *   dfo_dtw_*       the DTW variant of the appendix (max replaced by +)
 *   dfo_dtw_f32mirror  DTW in float32, one rounding per cell (GPU selection mirror)
 *   dfo_perturb_f32    x + sigma * z with one rounding (Monte Carlo samples)
 *   dfo_levenshtein Wagner-Fischer edit distance (the appendix's third
 *                   variant, read as the textbook definition: unit insert,
 *                   delete and substitute costs, D[i][0] = i, D[0][j] = j)
 *
 * Parity pins: every function above except the mirror is checked against
 * brute-force enumeration of monotone couplings, closed forms and the
 * metric invariants by the CPU test suite; none is "parity unpinned".
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#include <pthread.h>

#ifndef DFO_MUTANT
#define DFO_MUTANT 0   /* test hook: a nonzero value plants one known mistake */
#endif

/* ---------------------------------------------------------------- distances */

static double d2_f64(const float* a, const float* b, int dim) {
    double s = 0.0;
    for (int k = 0; k < dim; ++k) {
        double t = (double)a[k] - (double)b[k];
#if DFO_MUTANT == 5
        if (k == dim - 1 && dim > 1) continue;     /* mutant: drops a coordinate */
#endif
        s += t * t;
    }
    return s;
}

static int64_t d2_i64(const int32_t* a, const int32_t* b, int dim) {
    int64_t s = 0;
    for (int k = 0; k < dim; ++k) {
        int64_t t = (int64_t)a[k] - (int64_t)b[k];
        s += t * t;
    }
    return s;
}

static double dmin(double a, double b) { return a < b ? a : b; }
static double dmax(double a, double b) { return a > b ? a : b; }
static int64_t imin(int64_t a, int64_t b) { return a < b ? a : b; }
static int64_t imax(int64_t a, int64_t b) { return a > b ? a : b; }

/* ------------------------------------------------- Alg. 5 (linear memory) */
/*
 * v holds one row of M.  Row 1 is the running maximum of d(p_1, q_j).  For
 * every further row i: the vertical step replaces v_j by min(v_{j-1}, v_j)
 * for j >= 2 (simultaneously, so in place it runs right to left), then
 * v_1 <- max(v_1, d_i1) and, left to right, v_j <- max(min(v_{j-1}, v_j), d_ij).
 */
#define DFO_LINEAR_BODY(T, D2, MIN, MAX)                                        \
    T* v = (T*)malloc((size_t)m * sizeof(T));                                   \
    if (!v) return (T)-1;                                                       \
    v[0] = D2(p, q, dim);                                                       \
    for (int64_t j = 1; j < m; ++j) v[j] = MAX(v[j - 1], D2(p, q + j * dim, dim)); \
    for (int64_t i = 1; i < n; ++i) {                                           \
        const ELEM* pi = p + i * dim;                                           \
        for (int64_t j = m - 1; j >= 1; --j) v[j] = MIN(v[j - 1], v[j]);        \
        v[0] = MAX(v[0], D2(pi, q, dim));                                       \
        for (int64_t j = 1; j < m; ++j)                                         \
            v[j] = MAX(LINEAR_INNER_MIN(MIN, v[j - 1], v[j]), D2(pi, q + j * dim, dim)); \
    }                                                                           \
    T r = v[m - 1];                                                             \
    free(v);                                                                    \
    return r;

#if DFO_MUTANT == 1
/* mutant: the horizontal predecessor v_{j-1} is dropped */
#define LINEAR_INNER_MIN(MIN, a, b) (b)
#elif DFO_MUTANT == 2
/* mutant: min replaced by max in the horizontal step */
#define LINEAR_INNER_MIN(MIN, a, b) ((a) > (b) ? (a) : (b))
#else
#define LINEAR_INNER_MIN(MIN, a, b) MIN(a, b)
#endif

#define ELEM float
double dfo_linear_f64(const float* p, int64_t n, const float* q, int64_t m, int dim) {
    DFO_LINEAR_BODY(double, d2_f64, dmin, dmax)
}
#undef ELEM
#define ELEM int32_t
int64_t dfo_linear_i64(const int32_t* p, int64_t n, const int32_t* q, int64_t m, int dim) {
    DFO_LINEAR_BODY(int64_t, d2_i64, imin, imax)
}
#undef ELEM

/* ---------------------------------------- Alg. 3 (full matrix, branches) */

#define DFO_FULL_BODY(T, D2, MIN, MAX)                                          \
    T* M = (T*)malloc((size_t)n * (size_t)m * sizeof(T));                       \
    if (!M) return (T)-1;                                                       \
    for (int64_t i = 0; i < n; ++i) {                                           \
        for (int64_t j = 0; j < m; ++j) {                                       \
            T d = D2(p + i * dim, q + j * dim, dim);                            \
            T r;                                                                \
            if (i == 0 && j == 0) r = d;                                        \
            else if (i > 0 && j == 0) r = MAX(M[(i - 1) * m], d);               \
            else if (i == 0 && j > 0) r = MAX(M[j - 1], d);                     \
            else r = MAX(MIN(MIN(M[(i - 1) * m + j], FULL_DIAG(M, i, j, m)),    \
                             M[i * m + j - 1]), d);                             \
            M[i * m + j] = r;                                                   \
        }                                                                       \
    }                                                                           \
    T res = M[n * m - 1];                                                       \
    free(M);                                                                    \
    return res;

#if DFO_MUTANT == 3
/* mutant: the diagonal predecessor M_{i-1,j-1} is dropped */
#define FULL_DIAG(M, i, j, m) M[((i) - 1) * (m) + (j)]
#else
#define FULL_DIAG(M, i, j, m) M[((i) - 1) * (m) + (j) - 1]
#endif

double dfo_full_f64(const float* p, int64_t n, const float* q, int64_t m, int dim) {
    DFO_FULL_BODY(double, d2_f64, dmin, dmax)
}
int64_t dfo_full_i64(const int32_t* p, int64_t n, const int32_t* q, int64_t m, int dim) {
    DFO_FULL_BODY(int64_t, d2_i64, imin, imax)
}

/* ------------------------------------ Alg. 1 (memoised, explicit stack) */
/*
 * The memo starts at the sentinel -1 ("not computed"; all d >= 0).  eval(i,j)
 * needs eval of its predecessors first; instead of recursing, a work stack
 * holds the cells whose predecessors are still pending.
 */
#define DFO_MEMO_BODY(T, D2, MIN, MAX)                                          \
    size_t cells = (size_t)n * (size_t)m;                                       \
    T* M = (T*)malloc(cells * sizeof(T));                                       \
    int64_t* st = (int64_t*)malloc((cells + 4) * 3 * sizeof(int64_t));         \
    if (!M || !st) { free(M); free(st); return (T)-1; }                         \
    for (size_t c = 0; c < cells; ++c) M[c] = (T)-1;                            \
    int64_t top = 0;                                                            \
    st[0] = (n - 1) * m + (m - 1);                                              \
    top = 1;                                                                    \
    while (top > 0) {                                                           \
        int64_t c = st[top - 1];                                                \
        int64_t i = c / m, j = c % m;                                           \
        if (M[c] > (T)-1) { --top; continue; }                                  \
        int pending = 0;                                                        \
        if (i > 0 && !(M[c - m] > (T)-1)) { st[top++] = c - m; pending = 1; }   \
        if (j > 0 && !(M[c - 1] > (T)-1)) { st[top++] = c - 1; pending = 1; }   \
        if (i > 0 && j > 0 && !(M[c - m - 1] > (T)-1)) { st[top++] = c - m - 1; pending = 1; } \
        if (pending) continue;                                                  \
        T d = D2(p + i * dim, q + j * dim, dim);                                \
        T r;                                                                    \
        if (i == 0 && j == 0) r = d;                                            \
        else if (i > 0 && j == 0) r = MAX(M[c - m], d);                         \
        else if (i == 0 && j > 0) r = MEMO_ROW1(MAX, M[c - 1], d);              \
        else r = MAX(MIN(MIN(M[c - m], M[c - m - 1]), M[c - 1]), d);            \
        M[c] = r;                                                               \
        --top;                                                                  \
    }                                                                           \
    T res = M[cells - 1];                                                       \
    free(M); free(st);                                                          \
    return res;

#if DFO_MUTANT == 4
/* mutant: the first row forgets its running maximum */
#define MEMO_ROW1(MAX, a, d) (d)
#else
#define MEMO_ROW1(MAX, a, d) MAX(a, d)
#endif

double dfo_memo_f64(const float* p, int64_t n, const float* q, int64_t m, int dim) {
    DFO_MEMO_BODY(double, d2_f64, dmin, dmax)
}
int64_t dfo_memo_i64(const int32_t* p, int64_t n, const int32_t* q, int64_t m, int dim) {
    DFO_MEMO_BODY(int64_t, d2_i64, imin, imax)
}

/* ------------------------------------- decision search (independent) */
/*
 * delta^2 is the smallest value eps among the d_ij^2 such that the cells with
 * d^2 <= eps contain a path from (1,1) to (n,m) moving by (1,0), (0,1) or
 * (1,1) (a monotone coupling of the two point sequences).  Feasibility is a
 * breadth-first search over that cell set; eps is found by binary search
 * over the sorted distinct values.  Quadratic memory; small inputs only.
 */
static int cmp_f64(const void* a, const void* b) {
    double x = *(const double*)a, y = *(const double*)b;
    return (x > y) - (x < y);
}
static int cmp_i64(const void* a, const void* b) {
    int64_t x = *(const int64_t*)a, y = *(const int64_t*)b;
    return (x > y) - (x < y);
}

#define DFO_DECIDE_BODY(T, D2, CMP)                                             \
    size_t cells = (size_t)n * (size_t)m;                                       \
    T* d = (T*)malloc(cells * sizeof(T));                                       \
    T* s = (T*)malloc(cells * sizeof(T));                                       \
    unsigned char* seen = (unsigned char*)malloc(cells);                        \
    int64_t* queue = (int64_t*)malloc(cells * sizeof(int64_t));                 \
    if (!d || !s || !seen || !queue) { free(d); free(s); free(seen); free(queue); return (T)-1; } \
    for (int64_t i = 0; i < n; ++i)                                             \
        for (int64_t j = 0; j < m; ++j) d[i * m + j] = D2(p + i * dim, q + j * dim, dim); \
    memcpy(s, d, cells * sizeof(T));                                            \
    qsort(s, cells, sizeof(T), CMP);                                            \
    size_t nd = 0;                                                              \
    for (size_t c = 0; c < cells; ++c) if (nd == 0 || s[c] != s[nd - 1]) s[nd++] = s[c]; \
    size_t lo = 0, hi = nd - 1; /* s[hi] (the maximum) is always feasible */    \
    while (lo < hi) {                                                           \
        size_t mid = lo + (hi - lo) / 2;                                        \
        T eps = s[mid];                                                         \
        memset(seen, 0, cells);                                                 \
        int ok = 0;                                                             \
        size_t qh = 0, qt = 0;                                                  \
        if (d[0] <= eps) { seen[0] = 1; queue[qt++] = 0; }                      \
        while (qh < qt) {                                                       \
            int64_t c = queue[qh++];                                            \
            int64_t i = c / m, j = c % m;                                       \
            if (i == n - 1 && j == m - 1) { ok = 1; break; }                    \
            int64_t nb[3] = { (i + 1 < n) ? c + m : -1, (j + 1 < m) ? c + 1 : -1, \
                              (i + 1 < n && j + 1 < m) ? c + m + 1 : -1 };      \
            for (int t = 0; t < 3; ++t) {                                       \
                int64_t e = nb[t];                                              \
                if (e >= 0 && !seen[e] && d[e] <= eps) { seen[e] = 1; queue[qt++] = e; } \
            }                                                                   \
        }                                                                       \
        if (ok) hi = mid; else lo = mid + 1;                                    \
    }                                                                           \
    T res = s[lo];                                                              \
    free(d); free(s); free(seen); free(queue);                                  \
    return res;

double dfo_decide_f64(const float* p, int64_t n, const float* q, int64_t m, int dim) {
    DFO_DECIDE_BODY(double, d2_f64, cmp_f64)
}
int64_t dfo_decide_i64(const int32_t* p, int64_t n, const int32_t* q, int64_t m, int dim) {
    DFO_DECIDE_BODY(int64_t, d2_i64, cmp_i64)
}

/* ----------------------------------------------- discrete Hausdorff (Sec. 2) */

double dfo_hausdorff_f64(const float* p, int64_t n, const float* q, int64_t m, int dim) {
    double h = 0.0;
    for (int64_t i = 0; i < n; ++i) {
        double best = INFINITY;
        for (int64_t j = 0; j < m; ++j) best = dmin(best, d2_f64(p + i * dim, q + j * dim, dim));
        h = dmax(h, best);
    }
#if DFO_MUTANT == 6
    m = 0;   /* planted mistake: one-sided (p -> q only) */
#endif
    for (int64_t j = 0; j < m; ++j) {
        double best = INFINITY;
        for (int64_t i = 0; i < n; ++i) best = dmin(best, d2_f64(p + i * dim, q + j * dim, dim));
        h = dmax(h, best);
    }
    return h;
}

int64_t dfo_hausdorff_i64(const int32_t* p, int64_t n, const int32_t* q, int64_t m, int dim) {
    int64_t h = 0;
    for (int64_t i = 0; i < n; ++i) {
        int64_t best = INT64_MAX;
        for (int64_t j = 0; j < m; ++j) best = imin(best, d2_i64(p + i * dim, q + j * dim, dim));
        h = imax(h, best);
    }
#if DFO_MUTANT == 6
    m = 0;   /* planted mistake: one-sided (p -> q only) */
#endif
    for (int64_t j = 0; j < m; ++j) {
        int64_t best = INT64_MAX;
        for (int64_t i = 0; i < n; ++i) best = imin(best, d2_i64(p + i * dim, q + j * dim, dim));
        h = imax(h, best);
    }
    return h;
}

/* ------------------------------------ float32 selection mirror of Alg. 5 */
/*
 * Same recurrence as dfo_linear_f64 but every value is a float32: the
 * coordinate difference t_k = p_k - q_k rounded to float32, then the squared
 * distance as acc = t_0 * t_0 (rounded) followed by acc = fma(t_k, t_k, acc)
 * for k = 1 .. dim-1 (one rounding each, fused).  The DP then selects among
 * those float32 values with fminf/fmaxf, which never round.
 */
static float d2_f32(const float* a, const float* b, int dim) {
    float t = a[0] - b[0];
    float acc = t * t;
    for (int k = 1; k < dim; ++k) {
        float u = a[k] - b[k];
        acc = fmaf(u, u, acc);
    }
    return acc;
}

float dfo_linear_f32mirror(const float* p, int64_t n, const float* q, int64_t m, int dim) {
    float* v = (float*)malloc((size_t)m * sizeof(float));
    if (!v) return -1.0f;
    v[0] = d2_f32(p, q, dim);
    for (int64_t j = 1; j < m; ++j) v[j] = fmaxf(v[j - 1], d2_f32(p, q + j * dim, dim));
    for (int64_t i = 1; i < n; ++i) {
        const float* pi = p + i * dim;
        for (int64_t j = m - 1; j >= 1; --j) v[j] = fminf(v[j - 1], v[j]);
        v[0] = fmaxf(v[0], d2_f32(pi, q, dim));
        for (int64_t j = 1; j < m; ++j) v[j] = fmaxf(fminf(v[j - 1], v[j]), d2_f32(pi, q + j * dim, dim));
    }
    float r = v[m - 1];
    free(v);
    return r;
}

/* ----------------------------- Alg. 5 over many pairs (CPU threads) */

typedef struct {
    const void* points;
    const int64_t* offsets;
    const int32_t* pairs;
    int64_t n_pairs;
    int dim;
    int kind;          /* 0: f64 oracle, 1: i64 oracle, 2: f32 mirror */
    void* out;
    int64_t next;      /* shared work counter */
    pthread_mutex_t mu;
} batch_job;

static void* batch_worker(void* arg) {
    batch_job* J = (batch_job*)arg;
    for (;;) {
        pthread_mutex_lock(&J->mu);
        int64_t k = J->next;
        J->next += 16;
        pthread_mutex_unlock(&J->mu);
        if (k >= J->n_pairs) break;
        int64_t e = k + 16 < J->n_pairs ? k + 16 : J->n_pairs;
        for (; k < e; ++k) {
            int64_t a = J->pairs[2 * k], b = J->pairs[2 * k + 1];
            int64_t na = J->offsets[a + 1] - J->offsets[a], nb = J->offsets[b + 1] - J->offsets[b];
            if (J->kind == 1) {
                const int32_t* P = (const int32_t*)J->points;
                ((int64_t*)J->out)[k] = dfo_linear_i64(P + J->offsets[a] * J->dim, na,
                                                       P + J->offsets[b] * J->dim, nb, J->dim);
            } else if (J->kind == 0) {
                const float* P = (const float*)J->points;
                ((double*)J->out)[k] = dfo_linear_f64(P + J->offsets[a] * J->dim, na,
                                                      P + J->offsets[b] * J->dim, nb, J->dim);
            } else {
                const float* P = (const float*)J->points;
                ((float*)J->out)[k] = dfo_linear_f32mirror(P + J->offsets[a] * J->dim, na,
                                                           P + J->offsets[b] * J->dim, nb, J->dim);
            }
        }
    }
    return NULL;
}

static int run_batch(batch_job* J, int nthreads) {
    if (nthreads < 1) nthreads = 1;
    if (nthreads > 256) nthreads = 256;
    pthread_t th[256];
    J->next = 0;
    pthread_mutex_init(&J->mu, NULL);
    int started = 0;
    for (int t = 0; t < nthreads; ++t) {
        if (pthread_create(&th[t], NULL, batch_worker, J) != 0) break;
        ++started;
    }
    if (started == 0) batch_worker(J);
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    pthread_mutex_destroy(&J->mu);
    return started;
}

/* Returns the number of threads used.  out: double[n_pairs] (delta^2). */
int dfo_batch_f64(const float* points, const int64_t* offsets, const int32_t* pairs, int64_t n_pairs,
                  int dim, double* out, int nthreads) {
    batch_job J = { points, offsets, pairs, n_pairs, dim, 0, out, 0 };
    return run_batch(&J, nthreads);
}

int dfo_batch_i64(const int32_t* points, const int64_t* offsets, const int32_t* pairs, int64_t n_pairs,
                  int dim, int64_t* out, int nthreads) {
    batch_job J = { points, offsets, pairs, n_pairs, dim, 1, out, 0 };
    return run_batch(&J, nthreads);
}

int dfo_batch_f32mirror(const float* points, const int64_t* offsets, const int32_t* pairs, int64_t n_pairs,
                        int dim, float* out, int nthreads) {
    batch_job J = { points, offsets, pairs, n_pairs, dim, 2, out, 0 };
    return run_batch(&J, nthreads);
}

/* ------------------------------------------------ appendix variants */
/*
 * DTW (appendix, DTW algorithm): the Frechet recurrence with the outer max
 * replaced by addition, D_ij = min(D_{i-1,j}, D_{i-1,j-1}, D_{i,j-1}) + c_ij,
 * first row/column by running sums.  The ground cost c_ij is the squared
 * Euclidean distance here (the same d^2 the Frechet path carries).
 */
double dfo_dtw_f64(const float* p, int64_t n, const float* q, int64_t m, int dim) {
    double* v = (double*)malloc((size_t)m * sizeof(double));
    if (!v) return -1.0;
    v[0] = d2_f64(p, q, dim);
    for (int64_t j = 1; j < m; ++j) v[j] = v[j - 1] + d2_f64(p, q + j * dim, dim);
    for (int64_t i = 1; i < n; ++i) {
        const float* pi = p + i * dim;
        double diag = v[0];
        v[0] = v[0] + d2_f64(pi, q, dim);
        for (int64_t j = 1; j < m; ++j) {
            double up = v[j];
            v[j] = dmin(dmin(up, diag), v[j - 1]) + d2_f64(pi, q + j * dim, dim);
            diag = up;
        }
    }
    double r = v[m - 1];
    free(v);
    return r;
}

/*
 * DTW in float32 with a fixed evaluation order, the selection mirror of the
 * GPU kernel: the ground cost is d2_f32 (the squared-distance order above)
 * and each cell is one float32 addition after an exact minimum,
 * D_ij = fl(min(min(D_{i-1,j}, D_{i-1,j-1}), D_{i,j-1}) + c_ij).  Any
 * evaluation order with one rounding per cell gives this value bit for bit.
 */
float dfo_dtw_f32mirror(const float* p, int64_t n, const float* q, int64_t m, int dim) {
    float* v = (float*)malloc((size_t)m * sizeof(float));
    if (!v) return -1.0f;
    v[0] = d2_f32(p, q, dim);
    for (int64_t j = 1; j < m; ++j) v[j] = v[j - 1] + d2_f32(p, q + j * dim, dim);
    for (int64_t i = 1; i < n; ++i) {
        const float* pi = p + i * dim;
        float diag = v[0];
        v[0] = v[0] + d2_f32(pi, q, dim);
        for (int64_t j = 1; j < m; ++j) {
            float up = v[j];
            v[j] = fminf(fminf(up, diag), v[j - 1]) + d2_f32(pi, q + j * dim, dim);
            diag = up;
        }
    }
    float r = v[m - 1];
    free(v);
    return r;
}

/*
 * Perturbed coordinates of an uncertain curve (Monte Carlo sampling, the
 * application named in Sec. 5): out_i = x_i + sigma * z_i with one rounding
 * (C99 fmaf), z the caller's noise.
 */
void dfo_perturb_f32(const float* x, const float* z, float sigma, int64_t count, float* out) {
    for (int64_t i = 0; i < count; ++i) out[i] = fmaf(sigma, z[i], x[i]);
}

/*
 * Levenshtein distance of two symbol sequences by the textbook
 * Wagner-Fischer table: E_{i,0} = i, E_{0,j} = j,
 * E_ij = min(E_{i-1,j} + 1, E_{i,j-1} + 1, E_{i-1,j-1} + [a_i != b_j]).
 */
int64_t dfo_levenshtein(const int32_t* a, int64_t n, const int32_t* b, int64_t m) {
    int64_t* v = (int64_t*)malloc((size_t)(m + 1) * sizeof(int64_t));
    if (!v) return -1;
    for (int64_t j = 0; j <= m; ++j) v[j] = j;
    for (int64_t i = 1; i <= n; ++i) {
        int64_t diag = v[0];
        v[0] = i;
        for (int64_t j = 1; j <= m; ++j) {
            int64_t up = v[j];
            int64_t sub = diag + (a[i - 1] != b[j - 1] ? 1 : 0);
            v[j] = imin(imin(up + 1, v[j - 1] + 1), sub);
            diag = up;
        }
    }
    int64_t r = v[m];
    free(v);
    return r;
}
