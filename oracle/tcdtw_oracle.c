/*
 * tcdtw_oracle.c -- plain, slow FP64 CPU oracle for TC-DTW (Shen & Chi,
 * "TC-DTW: Accelerating Multivariate Dynamic Time Warping Through Triangle
 * Inequality and Point Clustering").
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the benchmark's
 * CPU-baseline leg may load this library.  It shares no code, header, table or
 * helper with the CUDA path and must never be called from the product path.
 *
 * Inputs are the float32 series the user supplies, layout [L][D] (D innermost).
 * All arithmetic is FP64 except the LB_PC cell ids, which are taken in FP32 on
 * purpose (see orc_pc_boxes) so that the discrete clustering is the same one the
 * GPU takes.  Build with -ffp-contract=off: no fused multiply-adds, so a result
 * depends only on the operation order written here.
 *
 * Readings of the paper that are not spelled out there:
 *   - the point cost is the SQUARED Euclidean distance, summed along the path and
 *     returned without a square root (LB_MV is then taken without its outer sqrt;
 *     LB_TI works on unsquared distances and squares its per-point minima);
 *   - windows are clipped to [0, L-1]; W >= L-1 means unconstrained;
 *   - every bound is summed over CANDIDATE points c_j, against query-side
 *     envelopes, triangle bounds and boxes;
 *   - a negative triangle lower bound is stored as 0 (a distance is >= 0);
 *   - LB_TI uses the "TIP_TOP" variant: exact distances on query rows with
 *     i mod P == 0 and at the top of each window (orc_lb_ti_var adds the basic,
 *     TOP and TIP variants);
 *   - LB_PC boxes are the tight bounding boxes of each cluster's member points;
 *     cells are ordered lexicographically with dimension 0 most significant; when
 *     there are more than K non-empty cells the first K-1 are kept and the rest
 *     merged into one box; the minimum cell length is 1e-5 (data is z-normalised).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_INF INFINITY

static int imin(int a, int b) { return a < b ? a : b; }
static int imax(int a, int b) { return a > b ? a : b; }
static double dmin2(double a, double b) { return a < b ? a : b; }
static double dmax2(double a, double b) { return a > b ? a : b; }

int orc_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* Point cost d(i,j): squared Euclidean distance between two D-vectors
 * (dependent multivariate DTW, Section 2 "Multivariate DTW"). */
double orc_cost(const float *a, const float *b, int D) {
    double s = 0.0;
    for (int p = 0; p < D; ++p) {
        double t = (double)a[p] - (double)b[p];
        s += t * t;
    }
    return s;
}

/* Unsquared Euclidean distance, used by the triangle bounds (Section 4). */
static double orc_euclid(const float *a, const float *b, int D) {
    return sqrt(orc_cost(a, b, D));
}

/* Row band of row i: [max(0,i-W), min(L-1,i+W)] (Sakoe-Chiba window, Section 2). */
static double band_get(const double *row, int i, int j, int W) {
    if (i < 0 || j < 0) return ORC_INF;
    if (abs(i - j) > W) return ORC_INF;
    return row[j];
}

/*
 * Windowed DTW, Eq. (1) with the Sakoe-Chiba band |i-j| <= W:
 *   R(i,j) = d(i,j) + min(R(i-1,j), R(i,j-1), R(i-1,j-1)),  R(-1,-1) = 0,
 *   R = +inf outside the band and on the other boundary cells.
 * Returns R(L-1, L-1).  If abandon_at is finite, the computation stops as soon
 * as every cell of a row is >= abandon_at (each warping path crosses every row)
 * and returns +inf ("early abandoning", Section 7.1).
 */
double orc_dtw_abandon(const float *a, const float *b, int L, int D, int W, double abandon_at) {
    if (W > L - 1) W = L - 1;
    double *prev = (double *)malloc(sizeof(double) * (size_t)L);
    double *cur = (double *)malloc(sizeof(double) * (size_t)L);
    for (int j = 0; j < L; ++j) prev[j] = ORC_INF;
    for (int i = 0; i < L; ++i) {
        double rowmin = ORC_INF;
        for (int j = imax(0, i - W); j <= imin(L - 1, i + W); ++j) {
            double best;
            if (i == 0 && j == 0) {
                best = 0.0;
            } else {
                double up = band_get(prev, i - 1, j, W);
                double left = band_get(cur, i, j - 1, W);
                double diag = band_get(prev, i - 1, j - 1, W);
                best = dmin2(dmin2(up, left), diag);
            }
            cur[j] = orc_cost(a + (size_t)i * D, b + (size_t)j * D, D) + best;
            rowmin = dmin2(rowmin, cur[j]);
        }
        double *t = prev; prev = cur; cur = t;
        if (rowmin >= abandon_at) {
            free(prev); free(cur);
            return ORC_INF;
        }
    }
    double r = prev[L - 1];
    free(prev); free(cur);
    return r;
}

double orc_dtw(const float *a, const float *b, int L, int D, int W) {
    return orc_dtw_abandon(a, b, L, D, W, ORC_INF);
}

/* Many independent pairs (A[p], B[p]); out[p] = DTW. */
void orc_dtw_pairs(const float *A, const float *B, int64_t P, int L, int D, int W, double *out,
                   int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t p = 0; p < P; ++p)
        out[p] = orc_dtw(A + (size_t)p * L * D, B + (size_t)p * L * D, L, D, W);
}

/*
 * Bounding envelope of a query (Section 3, "Algorithm LB_MV"):
 *   u_{i,p} = max(q_{i-W,p} : q_{i+W,p}),  l_{i,p} = min(...),
 * window clipped to [0, L-1].  U and Lo are [L][D].
 */
void orc_envelope(const float *q, int L, int D, int W, double *U, double *Lo) {
    for (int i = 0; i < L; ++i) {
        for (int p = 0; p < D; ++p) {
            double u = -ORC_INF, l = ORC_INF;
            for (int k = imax(0, i - W); k <= imin(L - 1, i + W); ++k) {
                double v = (double)q[(size_t)k * D + p];
                u = dmax2(u, v);
                l = dmin2(l, v);
            }
            U[(size_t)i * D + p] = u;
            Lo[(size_t)i * D + p] = l;
        }
    }
}

/* LB_MV from a precomputed envelope (Section 3), summed over candidate points,
 * without the outer square root:  sum_j sum_p  (c-u)^2 if c>u, (c-l)^2 if c<l. */
double orc_lb_mv_env(const double *U, const double *Lo, const float *c, int L, int D,
                     double abandon_at) {
    double s = 0.0;
    for (int j = 0; j < L; ++j) {
        for (int p = 0; p < D; ++p) {
            double x = (double)c[(size_t)j * D + p];
            double u = U[(size_t)j * D + p], l = Lo[(size_t)j * D + p];
            if (x > u) s += (x - u) * (x - u);
            else if (x < l) s += (x - l) * (x - l);
        }
        if (s >= abandon_at) return s;
    }
    return s;
}

double orc_lb_mv(const float *q, const float *c, int L, int D, int W) {
    double *U = (double *)malloc(sizeof(double) * (size_t)L * D);
    double *Lo = (double *)malloc(sizeof(double) * (size_t)L * D);
    orc_envelope(q, L, D, W, U, Lo);
    double r = orc_lb_mv_env(U, Lo, c, L, D, ORC_INF);
    free(U); free(Lo);
    return r;
}

/* LB_AD (Section 3): for every candidate point c_j, the smallest cost to a query
 * point in its window; summed over candidate points. */
double orc_lb_ad(const float *q, const float *c, int L, int D, int W) {
    if (W > L - 1) W = L - 1;
    double s = 0.0;
    for (int j = 0; j < L; ++j) {
        double m = ORC_INF;
        for (int i = imax(0, j - W); i <= imin(L - 1, j + W); ++i)
            m = dmin2(m, orc_cost(q + (size_t)i * D, c + (size_t)j * D, D));
        s += m;
    }
    return s;
}

/* Neighbour distances of a query, dq[i] = d(q_{i-1}, q_i) (Section 4.1); dq[0] = 0. */
void orc_query_dq(const float *q, int L, int D, double *dq) {
    dq[0] = 0.0;
    for (int i = 1; i < L; ++i) dq[i] = orc_euclid(q + (size_t)(i - 1) * D, q + (size_t)i * D, D);
}

/*
 * LB_TI, the "TIP_TOP" variant (Section 4.2 (3); P = period):
 * for each query row i, over its window j in [i-W, i+W] (clipped):
 *   - i mod P == 0: Lb = Ub = d(q_i, c_j)  (periodic exact rows; row 0 is exact);
 *   - j == i+W:     Lb = Ub = d(q_i, c_j)  (exact top of the window);
 *   - otherwise, Eqs. (bt_lb), (bt_ub) with dq_i = d(q_{i-1}, q_i):
 *       Lb(i,j) = max(Lb(i-1,j) - dq_i, dq_i - Ub(i-1,j)),  stored as max(.,0),
 *       Ub(i,j) = Ub(i-1,j) + dq_i.
 * Each candidate point's bound is the minimum Lb over the rows of its window; the
 * bound of the pair is the sum over candidate points of the squared minima
 * ("Full algorithm", Section 4.1), matching the squared point cost.
 */
double orc_lb_ti_dq(const float *q, const double *dq, const float *c, int L, int D, int W, int P,
                    double abandon_at) {
    if (W > L - 1) W = L - 1;
    double *Lb_prev = (double *)malloc(sizeof(double) * (size_t)L);
    double *Ub_prev = (double *)malloc(sizeof(double) * (size_t)L);
    double *Lb_cur = (double *)malloc(sizeof(double) * (size_t)L);
    double *Ub_cur = (double *)malloc(sizeof(double) * (size_t)L);
    double *m = (double *)malloc(sizeof(double) * (size_t)L);
    for (int j = 0; j < L; ++j) m[j] = ORC_INF;
    for (int i = 0; i < L; ++i) {
        for (int j = imax(0, i - W); j <= imin(L - 1, i + W); ++j) {
            double lb, ub;
            if (i % P == 0 || j == i + W) {
                lb = ub = orc_euclid(q + (size_t)i * D, c + (size_t)j * D, D);
            } else {
                lb = dmax2(Lb_prev[j] - dq[i], dq[i] - Ub_prev[j]);
                lb = dmax2(lb, 0.0);
                ub = Ub_prev[j] + dq[i];
            }
            Lb_cur[j] = lb;
            Ub_cur[j] = ub;
            m[j] = dmin2(m[j], lb);
        }
        double *t;
        t = Lb_prev; Lb_prev = Lb_cur; Lb_cur = t;
        t = Ub_prev; Ub_prev = Ub_cur; Ub_cur = t;
    }
    double s = 0.0;
    for (int j = 0; j < L; ++j) {
        s += m[j] * m[j];
        if (s >= abandon_at) break;
    }
    free(Lb_prev); free(Ub_prev); free(Lb_cur); free(Ub_cur); free(m);
    return s;
}

/*
 * The other LB_TI variants of Section 4.2 (basic LB_TI, LB_TI_TOP, LB_TIP; `top` and P
 * select them; top = 1 is orc_lb_ti_dq above):
 *   - i mod P == 0: exact row (P >= L: only row 0, the basic algorithm's start);
 *   - j == i+W, top == 1: exact top of the window;
 *   - j == i+W, top == 0, W >= 1: the candidate-side triangle with c_{j-1} (Eqs.
 *     (bt_lb_ir), (bt_ub_ir)), dc_j = d(c_{j-1}, c_j), from row i's value at j-1:
 *       Lb(i,j) = max(Lb(i,j-1) - dc_j, dc_j - Ub(i,j-1)),  stored as max(.,0),
 *       Ub(i,j) = Ub(i,j-1) + dc_j;
 *     (with W = 0 the window is the single point j = i, which has no neighbour in
 *     the window, so it is exact);
 *   - otherwise the query-side recursion with dq_i, as above.
 */
double orc_lb_ti_var(const float *q, const float *c, int L, int D, int W, int P, int top) {
    if (W > L - 1) W = L - 1;
    double *dq = (double *)malloc(sizeof(double) * (size_t)L);
    double *dc = (double *)malloc(sizeof(double) * (size_t)L);
    orc_query_dq(q, L, D, dq);
    orc_query_dq(c, L, D, dc);  /* the same neighbour distance, on the candidate */
    double *Lb_prev = (double *)malloc(sizeof(double) * (size_t)L);
    double *Ub_prev = (double *)malloc(sizeof(double) * (size_t)L);
    double *Lb_cur = (double *)malloc(sizeof(double) * (size_t)L);
    double *Ub_cur = (double *)malloc(sizeof(double) * (size_t)L);
    double *m = (double *)malloc(sizeof(double) * (size_t)L);
    for (int j = 0; j < L; ++j) m[j] = ORC_INF;
    for (int i = 0; i < L; ++i) {
        for (int j = imax(0, i - W); j <= imin(L - 1, i + W); ++j) {
            double lb, ub;
            if (i % P == 0 || (j == i + W && (top || W == 0))) {
                lb = ub = orc_euclid(q + (size_t)i * D, c + (size_t)j * D, D);
            } else if (j == i + W) {
                lb = dmax2(Lb_cur[j - 1] - dc[j], dc[j] - Ub_cur[j - 1]);
                lb = dmax2(lb, 0.0);
                ub = Ub_cur[j - 1] + dc[j];
            } else {
                lb = dmax2(Lb_prev[j] - dq[i], dq[i] - Ub_prev[j]);
                lb = dmax2(lb, 0.0);
                ub = Ub_prev[j] + dq[i];
            }
            Lb_cur[j] = lb;
            Ub_cur[j] = ub;
            m[j] = dmin2(m[j], lb);
        }
        double *t;
        t = Lb_prev; Lb_prev = Lb_cur; Lb_cur = t;
        t = Ub_prev; Ub_prev = Ub_cur; Ub_cur = t;
    }
    double s = 0.0;
    for (int j = 0; j < L; ++j) s += m[j] * m[j];
    free(dq); free(dc); free(Lb_prev); free(Ub_prev); free(Lb_cur); free(Ub_cur); free(m);
    return s;
}

double orc_lb_ti(const float *q, const float *c, int L, int D, int W, int P) {
    double *dq = (double *)malloc(sizeof(double) * (size_t)L);
    orc_query_dq(q, L, D, dq);
    double r = orc_lb_ti_dq(q, dq, c, L, D, W, P, ORC_INF);
    free(dq);
    return r;
}

/* Lexicographic comparison of two cell-id tuples, dimension 0 most significant. */
static const int *g_cells_sort_base;
static int g_cells_sort_D;
static int cmp_cell_rows(const void *x, const void *y) {
    int a = *(const int *)x, b = *(const int *)y;
    const int *ca = g_cells_sort_base + (size_t)a * g_cells_sort_D;
    const int *cb = g_cells_sort_base + (size_t)b * g_cells_sort_D;
    for (int p = 0; p < g_cells_sort_D; ++p) {
        if (ca[p] != cb[p]) return ca[p] < cb[p] ? -1 : 1;
    }
    return a < b ? -1 : (a > b);
}

/*
 * LB_PC bounding boxes of one query (Section 5, "Quantization-based clustering"
 * and "Uniform window grouping").
 * Group g (g = 0 .. ceil(L/w)-1) serves the windows of candidate points
 * j in [g*w, g*w+w-1]; its "expanded window" holds query points
 * [g*w - W, g*w + w - 1 + W] clipped to [0, L-1].  Per dimension p the value range
 * [mn_p, mx_p] of those points is split into Lq segments of length
 * len_p = max((mx_p - mn_p)/Lq, 1e-5); a point's cell along p is
 * min(Lq-1, floor((x - mn_p)/len_p)).  These cell ids are computed in FP32 (IEEE
 * round-to-nearest sub and div) so the discrete clustering is reproducible by any
 * implementation that follows the same FP32 steps.  Each non-empty cell is a
 * cluster whose box is the bounding box of its member points.  Cells are sorted
 * lexicographically; with more than K cells the first K-1 are kept and the rest
 * are combined into box K-1.
 * Output: boxes[g][k][0][p] = lower corner, boxes[g][k][1][p] = upper corner
 * ([G][K][2][D], unused slots untouched), counts[g] = number of boxes.
 * Unused box slots are left as they were.
 */
void orc_pc_boxes(const float *q, int L, int D, int W, int K, int Lq, int w, double *boxes,
                  int *counts) {
    if (W > L - 1) W = L - 1;
    int G = (L + w - 1) / w;
    int maxpts = imin(L, w + 2 * W);
    int *cell = (int *)malloc(sizeof(int) * (size_t)maxpts * D);
    int *order = (int *)malloc(sizeof(int) * (size_t)maxpts);
    float *mn = (float *)malloc(sizeof(float) * (size_t)D);
    float *len = (float *)malloc(sizeof(float) * (size_t)D);
    for (int g = 0; g < G; ++g) {
        int p0 = imax(0, g * w - W), p1 = imin(L - 1, g * w + w - 1 + W);
        int n = p1 - p0 + 1;
        for (int p = 0; p < D; ++p) {
            float lo = q[(size_t)p0 * D + p], hi = lo;
            for (int k = p0; k <= p1; ++k) {
                float v = q[(size_t)k * D + p];
                if (v < lo) lo = v;
                if (v > hi) hi = v;
            }
            volatile float range = hi - lo;              /* FP32, round to nearest */
            volatile float seg = range / (float)Lq;
            mn[p] = lo;
            len[p] = seg > 1e-5f ? seg : 1e-5f;
        }
        for (int k = 0; k < n; ++k) {
            for (int p = 0; p < D; ++p) {
                volatile float off = q[(size_t)(p0 + k) * D + p] - mn[p];
                volatile float r = off / len[p];
                int id = (int)floorf(r);
                if (id > Lq - 1) id = Lq - 1;
                cell[(size_t)k * D + p] = id;
            }
            order[k] = k;
        }
        g_cells_sort_base = cell;
        g_cells_sort_D = D;
        qsort(order, (size_t)n, sizeof(int), cmp_cell_rows);
        /* walk the sorted points; a new cell starts when the tuple changes */
        int nb = 0;
        double *gb = boxes + (size_t)g * K * 2 * D;
        for (int t = 0; t < n; ++t) {
            int k = order[t];
            int newcell = (t == 0) ||
                          memcmp(cell + (size_t)k * D, cell + (size_t)order[t - 1] * D,
                                 sizeof(int) * (size_t)D) != 0;
            if (newcell && nb < K) {
                ++nb;
                for (int p = 0; p < D; ++p) {
                    double v = (double)q[(size_t)(p0 + k) * D + p];
                    gb[(size_t)(nb - 1) * 2 * D + p] = v;
                    gb[(size_t)(nb - 1) * 2 * D + D + p] = v;
                }
                continue;
            }
            /* same cell as the previous point, or beyond K: grow box nb-1 */
            for (int p = 0; p < D; ++p) {
                double v = (double)q[(size_t)(p0 + k) * D + p];
                double *lo = &gb[(size_t)(nb - 1) * 2 * D + p];
                double *hi = &gb[(size_t)(nb - 1) * 2 * D + D + p];
                if (v < *lo) *lo = v;
                if (v > *hi) *hi = v;
            }
        }
        counts[g] = nb;
    }
    free(cell); free(order); free(mn); free(len);
}

/* Squared distance from a point to an axis-aligned box (0 inside). */
static double box_dist2(const float *x, const double *lo, const double *hi, int D) {
    double s = 0.0;
    for (int p = 0; p < D; ++p) {
        double v = (double)x[p];
        if (v < lo[p]) s += (lo[p] - v) * (lo[p] - v);
        else if (v > hi[p]) s += (v - hi[p]) * (v - hi[p]);
    }
    return s;
}

/* LB_PC from precomputed boxes (Section 5): each candidate point c_j is bounded by
 * its nearest box among the boxes of group floor(j/w); the pair's bound is the sum
 * over candidate points. */
double orc_lb_pc_boxes(const double *boxes, const int *counts, const float *c, int L, int D, int K,
                       int w, double abandon_at) {
    double s = 0.0;
    for (int j = 0; j < L; ++j) {
        int g = j / w;
        const double *gb = boxes + (size_t)g * K * 2 * D;
        double m = ORC_INF;
        for (int k = 0; k < counts[g]; ++k)
            m = dmin2(m, box_dist2(c + (size_t)j * D, gb + (size_t)k * 2 * D, gb + (size_t)k * 2 * D + D, D));
        s += m;
        if (s >= abandon_at) return s;
    }
    return s;
}

double orc_lb_pc(const float *q, const float *c, int L, int D, int W, int K, int Lq, int w) {
    int G = (L + w - 1) / w;
    double *boxes = (double *)calloc((size_t)G * K * 2 * D, sizeof(double));
    int *counts = (int *)calloc((size_t)G, sizeof(int));
    orc_pc_boxes(q, L, D, W, K, Lq, w, boxes, counts);
    double r = orc_lb_pc_boxes(boxes, counts, c, L, D, K, w, ORC_INF);
    free(boxes); free(counts);
    return r;
}

/* Brute-force DTW-NN (Section 2 "DTW-NN"): argmin over all candidates of the
 * windowed DTW, ties to the smallest candidate index. */
void orc_nn_brute(const float *Q, int64_t M, const float *C, int64_t N, int L, int D, int W,
                  int64_t *idx, double *dist, int nthreads) {
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads)
#endif
    for (int64_t m = 0; m < M; ++m) {
        double best = ORC_INF;
        int64_t bi = -1;
        for (int64_t n = 0; n < N; ++n) {
            double d = orc_dtw(Q + (size_t)m * L * D, C + (size_t)n * L * D, L, D, W);
            if (d < best) { best = d; bi = n; }
        }
        idx[m] = bi;
        dist[m] = best;
    }
}

/* Counters of the pruned search. */
typedef struct {
    int64_t pairs, pruned_mv, pruned_pc, pruned_ti, dtw_started, dtw_abandoned;
} orc_stats;

/*
 * The paper's pruned DTW-NN (Sections 2, 6 and 7.1), one query at a time, over
 * the candidates in index order:
 *   query-side preparation when the query arrives: envelope, neighbour distances,
 *   LB_PC boxes;
 *   per candidate: LB_MV (abandoned once it reaches best-so-far); skip if
 *   LB >= best-so-far; selective deployment: only if e*bsf < LB_MV < bsf apply
 *   LB_PC and/or LB_TI (use_pc, use_ti), LB = max of the bounds, skip if
 *   LB >= bsf; otherwise DTW with early abandoning; keep the smaller.
 * Strict "<" on improvement and ">=" on pruning keep the smallest index on ties.
 */
void orc_nn_pruned(const float *Q, int64_t M, const float *C, int64_t N, int L, int D, int W,
                   int K, int Lq, int w, int P, int use_pc, int use_ti, double e_pc, double e_ti,
                   int64_t *idx, double *dist, orc_stats *stats, int nthreads) {
    if (W > L - 1) W = L - 1;
    int G = (L + w - 1) / w;
    int64_t s_pairs = 0, s_mv = 0, s_pc = 0, s_ti = 0, s_started = 0, s_aband = 0;
#ifdef _OPENMP
    if (nthreads <= 0) nthreads = omp_get_max_threads();
#pragma omp parallel for schedule(dynamic, 1) num_threads(nthreads) \
    reduction(+ : s_pairs, s_mv, s_pc, s_ti, s_started, s_aband)
#endif
    for (int64_t m = 0; m < M; ++m) {
        const float *q = Q + (size_t)m * L * D;
        double *U = (double *)malloc(sizeof(double) * (size_t)L * D);
        double *Lo = (double *)malloc(sizeof(double) * (size_t)L * D);
        double *dq = (double *)malloc(sizeof(double) * (size_t)L);
        double *boxes = (double *)calloc((size_t)G * K * 2 * D, sizeof(double));
        int *counts = (int *)calloc((size_t)G, sizeof(int));
        orc_envelope(q, L, D, W, U, Lo);
        if (use_ti) orc_query_dq(q, L, D, dq);
        if (use_pc) orc_pc_boxes(q, L, D, W, K, Lq, w, boxes, counts);
        double bsf = ORC_INF;
        int64_t bi = -1;
        for (int64_t n = 0; n < N; ++n) {
            const float *c = C + (size_t)n * L * D;
            ++s_pairs;
            double lb_mv = orc_lb_mv_env(U, Lo, c, L, D, bsf);
            if (lb_mv >= bsf) { ++s_mv; continue; }
            double lb = lb_mv;
            if (use_pc && e_pc * bsf < lb_mv) {
                lb = dmax2(lb, orc_lb_pc_boxes(boxes, counts, c, L, D, K, w, bsf));
                if (lb >= bsf) { ++s_pc; continue; }
            }
            if (use_ti && e_ti * bsf < lb_mv) {
                lb = dmax2(lb, orc_lb_ti_dq(q, dq, c, L, D, W, P, bsf));
                if (lb >= bsf) { ++s_ti; continue; }
            }
            ++s_started;
            double d = orc_dtw_abandon(q, c, L, D, W, bsf);
            if (d == ORC_INF) { ++s_aband; continue; }
            if (d < bsf) { bsf = d; bi = n; }
        }
        idx[m] = bi;
        dist[m] = bsf;
        free(U); free(Lo); free(dq); free(boxes); free(counts);
    }
    if (stats) {
        stats->pairs = s_pairs; stats->pruned_mv = s_mv; stats->pruned_pc = s_pc;
        stats->pruned_ti = s_ti; stats->dtw_started = s_started; stats->dtw_abandoned = s_aband;
    }
}

/*
 * Gradient of the windowed DTW distance (the almost-everywhere derivative of Eq. (1);
 * the paper only names DTW as a loss, Section 1).  The optimal path is recovered by
 * backtracking from (L-1, L-1): the predecessor of (i,j) is the argmin of
 * {(i-1,j-1), (i-1,j), (i,j-1)} over in-band cells, exact ties resolved in that
 * order (diagonal, then up, then left).  Along the path
 *   dDTW/da_i = sum_{(i,j) on path} 2 (a_i - b_j),
 *   dDTW/db_j = sum_{(i,j) on path} 2 (b_j - a_i).
 * path_i/path_j (capacity 2L-1) receive the path from (0,0) to (L-1,L-1); the
 * return value is the distance.  *margin receives the smallest gap, relative to
 * R(i,j), between the chosen predecessor and the next best one along the path
 * (+inf if never ambiguous): a small margin flags a nearly non-unique path.
 */
double orc_dtw_grad(const float *a, const float *b, int L, int D, int W, double *ga, double *gb,
                    int *path_i, int *path_j, int *path_len, double *margin) {
    if (W > L - 1) W = L - 1;
    double *R = (double *)malloc(sizeof(double) * (size_t)L * L);
    for (size_t t = 0; t < (size_t)L * L; ++t) R[t] = ORC_INF;
#define RR(i, j) (((i) < 0 || (j) < 0 || abs((i) - (j)) > W) ? ORC_INF : R[(size_t)(i) * L + (j)])
    for (int i = 0; i < L; ++i) {
        for (int j = imax(0, i - W); j <= imin(L - 1, i + W); ++j) {
            double best = (i == 0 && j == 0) ? 0.0 : dmin2(dmin2(RR(i - 1, j), RR(i, j - 1)), RR(i - 1, j - 1));
            R[(size_t)i * L + j] = orc_cost(a + (size_t)i * D, b + (size_t)j * D, D) + best;
        }
    }
    double dist = R[(size_t)(L - 1) * L + (L - 1)];
    for (size_t t = 0; t < (size_t)L * D; ++t) { ga[t] = 0.0; gb[t] = 0.0; }
    int n = 0;
    int i = L - 1, j = L - 1;
    double mg = ORC_INF;
    int *ti = (int *)malloc(sizeof(int) * (size_t)(2 * L));
    int *tj = (int *)malloc(sizeof(int) * (size_t)(2 * L));
    for (;;) {
        ti[n] = i; tj[n] = j; ++n;
        for (int p = 0; p < D; ++p) {
            double diff = (double)a[(size_t)i * D + p] - (double)b[(size_t)j * D + p];
            ga[(size_t)i * D + p] += 2.0 * diff;
            gb[(size_t)j * D + p] -= 2.0 * diff;
        }
        if (i == 0 && j == 0) break;
        double vd = RR(i - 1, j - 1), vu = RR(i - 1, j), vl = RR(i, j - 1);
        double best = vd; int pi = i - 1, pj = j - 1;
        if (vu < best) { best = vu; pi = i - 1; pj = j; }
        if (vl < best) { best = vl; pi = i; pj = j - 1; }
        /* second best among the three, for the uniqueness margin */
        double vals[3] = {vd, vu, vl};
        double second = ORC_INF; int seen_best = 0;
        for (int k = 0; k < 3; ++k) {
            if (vals[k] == best && !seen_best) { seen_best = 1; continue; }
            second = dmin2(second, vals[k]);
        }
        if (second < ORC_INF) {
            double scale = dmax2(R[(size_t)i * L + j], 1e-300);
            mg = dmin2(mg, (second - best) / scale);
        }
        i = pi; j = pj;
    }
#undef RR
    for (int k = 0; k < n; ++k) { path_i[k] = ti[n - 1 - k]; path_j[k] = tj[n - 1 - k]; }
    *path_len = n;
    *margin = mg;
    free(ti); free(tj); free(R);
    return dist;
}
