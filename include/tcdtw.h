/*
 * tcdtw.h -- C ABI of libtcdtw.so: exact 1-nearest-neighbour search under
 * Sakoe-Chiba-windowed dependent multivariate DTW on one GB300 (sm_103a), after
 * TC-DTW (Shen & Chi): query envelopes, the lower-bound cascade LB_MV -> LB_PC /
 * LB_TI with selective deployment, survivor compaction, banded DTW with early
 * abandoning against a device-resident best-so-far; plus a differentiable DTW
 * distance (forward and adjoint) and a batched search over many uneven sets.
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - Series are float32, C-contiguous, layout [count][L][D] (D innermost).  Unless a
 *    comment says "host", every array pointer is a DEVICE pointer on the current
 *    CUDA device.  The caller owns all inputs and outputs.
 *  - `stream` is a cudaStream_t passed as void* (NULL = legacy default stream).
 *    Calls enqueue work on it and return without synchronising, except where a
 *    host output (stats) is requested.
 *  - W is the half-width of the Sakoe-Chiba band (Section 2, "Window DTW": cells
 *    with j-W <= i <= j+W); W >= L-1 means unconstrained and is clamped to L-1.
 *  - The DTW point cost is the SQUARED Euclidean distance of two D-vectors, summed
 *    along the warping path (Eq. 1 with the dependent multivariate cost of
 *    Section 2); distances are returned without a square root.
 *  - Return value: TCDTW_OK (0) or one of the error codes below; the message is
 *    tcdtw_strerror(code).  On an error no output is guaranteed to be written.
 */
#ifndef TCDTW_H
#define TCDTW_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define TCDTW_OK 0
#define TCDTW_ERR_INVALID 1   /* bad argument: L<1, D<1, W<0, K<1, N<1, null pointer, ... */
#define TCDTW_ERR_NOMEM 2     /* a device allocation failed */
#define TCDTW_ERR_CUDA 3      /* a CUDA runtime call or kernel launch failed */
#define TCDTW_ERR_TIMEOUT 4   /* a device-side wait hit its iteration limit */
#define TCDTW_ERR_NONFINITE 5 /* NaN or Inf found in an input series */
#define TCDTW_ERR_UNSUPPORTED 6 /* shape outside the compiled kernels (e.g. D too large) */

/* Largest number of dimensions the kernels are compiled for. */
#define TCDTW_MAX_D 64

/* Which lower bound tcdtw_lower_bounds computes. */
#define TCDTW_LB_MV 0 /* LB_MV (Section 3), over candidate points, no sqrt            */
#define TCDTW_LB_PC 1 /* LB_PC (Section 5) with uniform window grouping              */
#define TCDTW_LB_TI 2 /* LB_TI in its TIP_TOP form (Section 4.2 (3))                  */
#define TCDTW_LB_MV_REV 3 /* candidate-side LB_MV: the candidate's envelope, summed over
                             query points (Section 3 with the roles exchanged)        */

typedef struct tcdtw_index tcdtw_index; /* opaque; created by tcdtw_build */

/*
 * Search options (Sections 6 and 7.1 give the paper's values).
 *  P       LB_TI period: query rows i with i mod P == 0 use exact distances (5).
 *  Lq      LB_PC quantisation levels per dimension (2).
 *  w       LB_PC window expansion factor: boxes per group of w windows (6).
 *  e_pc, e_ti  selective-deployment thresholds: LB_PC / LB_TI run on a pair only if
 *          e * best-so-far < LB_MV < best-so-far (0.1, 0.1).
 *  use_pc, use_ti  enable the two tight bounds (1, 1).
 *  seed_s  per query, the DTW of the seed_s candidates with the smallest LB_MV is
 *          computed first to start the best-so-far low (4).
 *  qblock  queries per pipeline block (0 = chosen from free memory).
 *  tile    DTW band-tile id (-1 = autotuned; see tcdtw_tile_count()).
 *  check_finite  1 = scan inputs and fail with TCDTW_ERR_NONFINITE on NaN/Inf (1).
 *  no_prune  1 = the "default windowed DTW without lower bounds" the paper measures
 *          its speedups against (Section 7.2): the full DTW of every pair, no bound,
 *          no abandoning; the answer is the same (0).
 *  use_graph  1 = a tcdtw_nn call of at most one query block (M <= qblock) runs on the
 *          index's own query and answer buffers: it copies the queries in, runs the
 *          kernel sequence -- eagerly the first time a given M is seen, then as a CUDA
 *          graph captured on the second call with that M and replayed afterwards --
 *          and copies the answers out, all on `stream`.  The caller may pass different
 *          buffers on every call (1).
 *  select  1 = TC-DTW's data-adaptive choice (Section 6, "TC-DTW"; parameter ranges of
 *          Section 7.1): the first tcdtw_nn call on an index times, on up to 32 of
 *          its queries, LB_MV alone, LB_TI with e_ti in {0.05, 0.1, 0.2} and LB_PC with
 *          e_pc in {0.1, 0.5} and Lq in {2, 3} (within use_ti / use_pc), and keeps the
 *          fastest for the index (1).  The answers do not depend on the choice;
 *          tcdtw_index_opts reports it.
 *  use_rev  1 = also apply the candidate-side LB_MV (TCDTW_LB_MV_REV) to every pair that
 *          survives the query-side LB_MV, before LB_PC / LB_TI; a pair's bound becomes
 *          the larger of the two.  tcdtw_build then computes and keeps the envelopes
 *          of all candidates (2*N*L*D floats) (0).  Not applied by tcdtw_batch_nn.
 *  ti_top  LB_TI's window top c_{i+W}: 1 = exact distance (LB_TI_TOP; with P the
 *          TIP_TOP form, Section 4.2 (3)), 0 = from the candidate-side triangle with
 *          c_{i+W-1} (Eqs. (bt_lb_ir), (bt_ub_ir); with P < L the LB_TIP form, with
 *          P >= L the basic LB_TI, whose only exact row is row 0) (1).  ti_top = 0
 *          needs W <= 127 (else tcdtw_build and tcdtw_lower_bounds return
 *          UNSUPPORTED); tcdtw_batch_nn always uses 1.
 *  mv_abandon  1 = LB_MV with early abandoning (Section 7.1 applies abandoning to the
 *          lower bounds as well as to DTW): a block of at least 32 queries first sums,
 *          for every pair, a sample of its LB_MV elements: s = clamp(C/16, 1, 8) chunks
 *          of 32 spread evenly over the row (chunks 0, C/s, 2C/s, ...; C = ceil(L*D/32)),
 *          a sum over a subset of the terms and hence a lower bound.  It takes seed_s
 *          seeds from those sample sums and runs their DTW, then completes LB_MV only
 *          for the pairs at or under the seeded threshold (the others keep their sample
 *          sum, a lower bound above the threshold), and runs the DTW of a second round
 *          of seed_s seeds, the smallest completed bounds (tcdtw_batch_nn: one round).
 *          Rows of fewer than 128 elements never abandon.  The answers are the same (1).
 */
typedef struct {
    int32_t P;
    int32_t Lq;
    int32_t w;
    float e_pc;
    float e_ti;
    int32_t use_pc;
    int32_t use_ti;
    int32_t seed_s;
    int32_t qblock;
    int32_t tile;
    int32_t check_finite;
    int32_t no_prune;
    int32_t use_graph;
    int32_t select;
    int32_t use_rev;
    int32_t ti_top;
    int32_t mv_abandon;
} tcdtw_opts;

/* Counters of one tcdtw_nn call, summed over its queries. */
typedef struct {
    uint64_t pairs;         /* query-candidate pairs considered (M*N)               */
    uint64_t pruned_mv;     /* pairs whose LB_MV exceeded the best-so-far threshold  */
    uint64_t pruned_pc;     /* ... pruned by LB_PC after passing LB_MV               */
    uint64_t pruned_ti;     /* ... pruned by LB_TI                                   */
    uint64_t dtw_started;   /* DTWs started (seeds included)                         */
    uint64_t dtw_abandoned; /* DTWs stopped early against the best-so-far            */
    uint64_t cells;         /* DTW cells computed in FP32                            */
    uint64_t refined;       /* candidates recomputed in double-float arithmetic
                               because FP32 could not separate them from the best */
    uint64_t refined64;     /* ... of those, recomputed in FP64 because double-float
                               could not separate them either                      */
    uint64_t pruned_rev;    /* ... pruned by the candidate-side LB_MV (use_rev)      */
    uint64_t mv_terms;      /* LB_MV terms summed, one per (element, pair); below
                               pairs*L*D when LB_MV abandons (mv_abandon)          */
} tcdtw_stats;

/* Fill *opts with the defaults listed above. */
void tcdtw_default_opts(tcdtw_opts *opts);

/*
 * tcdtw_build -- prepare a searchable candidate set C (Def. 1: the set C of
 * candidate series; the search is for each query's nearest member of C).
 *   cand  device [N][L][D] float32.  BORROWED: it must stay alive and unchanged
 *         until tcdtw_free (large sets are not copied).
 *   N, L, D, W  set size, series length, dimensions, band half-width.
 *   K     maximum number of LB_PC clusters per expanded window (Section 5).
 *   opts  NULL = defaults.
 *   out   host: receives the new index; it owns its device workspaces.
 * Validates the shapes, scans the candidates for non-finite values (if
 * opts->check_finite), allocates the per-block workspaces and chooses the DTW tile:
 * unless opts->tile is set, every valid (tile, G) of the shape is timed on pairs of the
 * candidates and the fastest kept, per (L, D, W) for the life of the process; with the
 * environment variable TCDTW_TUNE_CACHE naming a file, choices are also read from and
 * appended to that file (lines of another device or build are ignored).
 * LB_PC is switched off (results are unchanged, only pruning) when its cell keys
 * Lq^D do not fit in 63 bits.
 * Errors: INVALID, NOMEM, CUDA, NONFINITE, UNSUPPORTED.
 */
int tcdtw_build(const float *cand, int64_t N, int32_t L, int32_t D, int32_t W, int32_t K,
                const tcdtw_opts *opts, void *stream, tcdtw_index **out);

/*
 * tcdtw_nn -- exact DTW nearest neighbour of each query (Def. 1; Section 2
 * "DTW-NN"; the search loop of Sections 6-7 re-laid out for the GPU).
 *   q     device [M][L][D] float32 queries (same L and D as the index).
 *   idx   device [M] int64: index in C of the nearest candidate; exact ties go to
 *         the smallest index.
 *   dist  device [M] float64: its DTW distance from the double-float recompute
 *         (relative error below ~1e-9; the FP64 value itself when the FP64 step ran
 *         for that query).
 *   stats host, may be NULL; when given, the call synchronises `stream` and fills it.
 * Every bound is a rigorous lower bound in FP32 (directed rounding), pruning uses a
 * margin that covers the FP32 DTW rounding error, candidates whose FP32 DTW cannot
 * be told apart from the best are recomputed in double-float arithmetic with a
 * proven error bound, and the few that this still cannot separate are recomputed in
 * FP64 -- so idx equals the FP64 brute-force argmin (ties: smallest index).
 * Errors: INVALID, NOMEM, CUDA, NONFINITE, TIMEOUT.
 */
int tcdtw_nn(tcdtw_index *index, const float *q, int64_t M, int64_t *idx, double *dist,
             tcdtw_stats *stats, void *stream);

/* The options the index searches with (host output): those given to tcdtw_build,
 * with the bound choice of the first tcdtw_nn call when opts->select was set.
 * Errors: INVALID. */
int tcdtw_index_opts(tcdtw_index *index, tcdtw_opts *out);

/* Release an index and its workspaces (NULL is accepted). */
void tcdtw_free(tcdtw_index *index);

/* The DTW band tile the index uses (autotuned at build unless opts->tile was set),
 * its lanes per pair G, and the query block size (host outputs, each may be NULL).
 * Errors: INVALID. */
int tcdtw_index_info(tcdtw_index *index, int32_t *tile, int32_t *G, int32_t *qblock);

/*
 * Per-stage timing of tcdtw_nn (tracing; not in the paper).  With profiling on,
 * every query block records CUDA events on the caller's stream at the stage
 * boundaries below and tcdtw_nn synchronises at its end to add the elapsed times.
 * Stages: 0 non-finite scan, 1 query preparation (envelope, dq, boxes), 2 LB_MV (with
 * mv_abandon: over the sample), 3 seeds (selection and their DTW), 4 completion of the
 * abandoning LB_MV, 5 second seed round (4 and 5 are empty without abandoning),
 * 6 compaction, 7 LB_PC / LB_TI cascade, 8 DTW of the survivors, 9 refine (double-float,
 * then FP64 where needed) and selection.
 * tcdtw_set_profiling: enable != 0 turns it on; either way the totals are reset.
 * tcdtw_stage_times: host ms[TCDTW_NUM_STAGES] receives the summed milliseconds,
 * host *blocks (may be NULL) the number of query blocks timed.  Errors: INVALID.
 */
#define TCDTW_NUM_STAGES 10
int tcdtw_set_profiling(tcdtw_index *index, int32_t enable);
int tcdtw_stage_times(tcdtw_index *index, double *ms, int64_t *blocks);

/* Number of kernels the library has launched in this process (host counter). */
uint64_t tcdtw_kernel_launches(void);

/*
 * tcdtw_dtw_pairs -- DTW distance of P independent pairs (A[p], B[p]) (Eq. 1 in the
 * Sakoe-Chiba band), no abandoning.
 *   A, B  device [P][L][D] float32.   dist  device [P] float32.
 *   ckpt  device buffer of ckpt_bytes (from tcdtw_dtw_pairs_ckpt_bytes) that
 *         receives band rows every few rows for tcdtw_dtw_pairs_backward, or NULL.
 * Errors: INVALID (also ckpt_bytes too small), CUDA, UNSUPPORTED.
 */
int tcdtw_dtw_pairs(const float *A, const float *B, int64_t P, int32_t L, int32_t D, int32_t W,
                    float *dist, void *ckpt, int64_t ckpt_bytes, void *stream);

/* Bytes of checkpoint storage tcdtw_dtw_pairs needs for P pairs (host *bytes). */
int tcdtw_dtw_pairs_ckpt_bytes(int64_t P, int32_t L, int32_t D, int32_t W, int64_t *bytes);

/*
 * tcdtw_dtw_pairs_backward -- adjoint of tcdtw_dtw_pairs (not in the paper, which
 * only names DTW as a loss, Section 1).  For each pair the optimal warping path is
 * recomputed segment by segment from the checkpointed band rows and backtracked from
 * (L-1, L-1) (exact ties: diagonal, then (i-1, j), then (i, j-1)); then
 *   gA[p][i] = grad_dist[p] * sum_{(i,j) on path} 2 (A[p][i] - B[p][j]),
 *   gB[p][j] = grad_dist[p] * sum_{(i,j) on path} 2 (B[p][j] - A[p][i]).
 *   ckpt  the buffer filled by tcdtw_dtw_pairs on the same A, B, L, D, W.
 *   grad_dist device [P] float32;  gA, gB device [P][L][D] float32 (overwritten).
 * Errors: INVALID, CUDA, UNSUPPORTED.
 */
int tcdtw_dtw_pairs_backward(const float *A, const float *B, const void *ckpt, int64_t ckpt_bytes,
                             const float *grad_dist, int64_t P, int32_t L, int32_t D, int32_t W,
                             float *gA, float *gB, void *stream);

/*
 * Stage entry points (each is one step of the tcdtw_nn pipeline, exposed for
 * checking and for callers who build their own pruning).
 */

/* Query envelopes (Section 3, "Algorithm LB_MV"): U[m][i][p] = max of q[m][k][p] over
 * k in [i-W, i+W] clipped to [0, L-1], Lo likewise with min.  q, U, Lo device
 * [M][L][D] float32.  Exact (min/max).  Errors: INVALID, CUDA. */
int tcdtw_envelope(const float *q, int64_t M, int32_t L, int32_t D, int32_t W, float *U, float *Lo,
                   void *stream);

/* Query neighbour distances d(q_{i-1}, q_i) (Section 4.1) as an interval:
 * dq_lo[m][i] <= exact <= dq_hi[m][i] (FP32 rounded down / up); entry 0 is 0.
 * dq_lo, dq_hi device [M][L] float32.  Errors: INVALID, CUDA. */
int tcdtw_query_dq(const float *q, int64_t M, int32_t L, int32_t D, float *dq_lo, float *dq_hi,
                   void *stream);

/* LB_PC boxes of each query (Section 5): boxes device [M][G][K][2][D] float32
 * (lower corner, upper corner), counts device [M][G] int32, G = ceil(L/w).  Cell ids
 * are taken with FP32 round-to-nearest subtraction and division,
 * id = min(Lq-1, floor((x - min_p) / max((max_p - min_p)/Lq, 1e-5))); cells are
 * ordered lexicographically (dimension 0 most significant); beyond K cells the
 * first K-1 are kept and the rest merged; boxes are tight member bounding boxes.
 * Errors: INVALID (Lq^D must fit in 63 bits), CUDA. */
int tcdtw_pc_boxes(const float *q, int64_t M, int32_t L, int32_t D, int32_t W, int32_t K, int32_t Lq,
                   int32_t w, float *boxes, int32_t *counts, void *stream);

/* All M*N values of one lower bound (which = TCDTW_LB_*), no abandoning, rounded
 * down so that out[m][n] <= the exact bound <= DTW(q[m], c[n]).
 * q device [M][L][D], c device [N][L][D], out device [M][N] float32.
 * opts supplies P, Lq, w and ti_top (NULL = defaults): TCDTW_LB_TI with ti_top = 0 is
 * LB_TIP (the basic LB_TI when P >= L); K is the LB_PC cluster cap.
 * TCDTW_LB_MV_REV computes the candidates' envelopes on the fly (2*N*L*D floats).
 * Synchronous on `stream`.
 * Errors: INVALID, NOMEM, CUDA, TIMEOUT (a bounded device wait of the LB_MV stream ran
 * out), UNSUPPORTED (ti_top = 0 with W > 127). */
int tcdtw_lower_bounds(const float *q, int64_t M, const float *c, int64_t N, int32_t L, int32_t D,
                       int32_t W, int32_t K, const tcdtw_opts *opts, int32_t which, float *out,
                       void *stream);

/* LB_MV with early abandoning against per-query thresholds (Section 7.1): every pair
 * first sums a sample of its elements (the chunks mv_abandon uses); pairs whose sample
 * sum is at most thresh[m] complete the sum, the others stop there.  Hence
 * out[m][n] <= the exact LB_MV <= DTW(q[m], c[n]); where the computed LB_MV (rounded
 * down; summation order as in the search, which may differ from tcdtw_lower_bounds in
 * the last bits) is at most thresh[m], out[m][n] is that value, and elsewhere
 * out[m][n] > thresh[m].  Rows of fewer than 128 elements (L*D) are summed whole.
 * q device [M][L][D], c device [N][L][D], thresh device [M] float32 (+inf: every
 * pair complete), out device [M][N] float32.  Synchronous on `stream`.
 * Errors: INVALID, UNSUPPORTED (D > 64, M*N >= 4.29e9), NOMEM, CUDA, TIMEOUT. */
int tcdtw_lb_mv_abandon(const float *q, int64_t M, const float *c, int64_t N, int32_t L, int32_t D,
                        int32_t W, const float *thresh, float *out, void *stream);

/*
 * tcdtw_lb_mv_noalloc -- the same values as tcdtw_lower_bounds(..., TCDTW_LB_MV, ...)
 * (all M*N LB_MV bounds, rounded down, out device [M][N] float32), but without any
 * device allocation.  The paper has no counterpart: this is a deployment variant.
 * Who needs it: serving loops that must not stall (cudaMalloc / cudaFree can
 * synchronise the whole device), and processes whose device memory is owned by a
 * caching allocator or a fixed budget, where a raw cudaMalloc can fail although the
 * application has memory to spare.
 * The envelope scratch is a fixed array inside the library (8 MiB: two halves of
 * 2^20 floats); each loaded device keeps it until the process exits.  Limit:
 * 2*ceil(M/2) * ceil32(L*D) <= 2^20, else TCDTW_ERR_UNSUPPORTED (no work is done).
 * The first call on a device resolves the array's device address (set-up, with that
 * device current; it is resolved again if the device's context has changed, e.g.
 * after cudaDeviceReset): make that first call before any stream capture.
 * Every call uses the same array and the scratch keeps the last call's contents;
 * each call rewrites, before reading them, the envelope values of all its queries
 * (with odd M the unused half of the last query pair keeps stale values, which feed
 * only a discarded lane of the computation), so nothing needs clearing.  Calls whose
 * kernels overlap on the GPU (different streams, or different host threads) race on
 * the array and must be serialised by the caller.  Asynchronous on `stream`.
 * Errors (checked in the order of tcdtw_lower_bounds): INVALID, UNSUPPORTED (D > 64,
 * M*N >= 4.29e9, or beyond the scratch), CUDA.
 */
int tcdtw_lb_mv_noalloc(const float *q, int64_t M, const float *c, int64_t N, int32_t L, int32_t D, int32_t W,
                        float *out, void *stream);

/* Survivor compaction: for each row m of lb [M][N], the column indices n with
 * lb[m][n] <= thresh[m], in increasing n, written to out_idx[m][0 .. count[m]-1]
 * (out_idx device [M][N] int32, count device [M] int32).  Errors: INVALID, CUDA. */
int tcdtw_compact(const float *lb, int64_t M, int64_t N, const float *thresh, int32_t *out_idx,
                  int32_t *count, void *stream);

/*
 * Batched search: many independent (candidate set, query set) problems of uneven
 * L, D, N, W searched together (not in the paper; a deployment pattern).  Each entry
 * is searched exactly as tcdtw_nn would search it (same bounds, same rounding
 * margins, same refine), so idx/dist are the exact nearest neighbours under Eq. (1)
 * with the band |i-j| <= W.
 *
 * The batch runs as one sequence of persistent launches, each taking work items off
 * a device queue: (1) per query its envelope / neighbour distances / LB_PC boxes, per
 * 32-query x 128-candidate tile its LB_MV bounds, per query its seeds -- items of one
 * set wait for the earlier items they need on device counters, and each wait gives
 * up after about a second (the call then returns TIMEOUT); (2) the seeds' banded DTW,
 * one launch per tile class (D); (3) per query compaction and gated LB_PC / LB_TI;
 * (4) the survivors' DTW with early abandoning, one launch per tile class; (5) per
 * query the refine.  Each set's DTW runs on the band tile the single-set tuner picks for
 * its shape (tcdtw_batch_tiles).  Entries with D > 12 or W > 140 are searched through tcdtw_build
 * / tcdtw_nn, one after another, after the sequence.  The sequence and its workspace
 * are kept per distinct batch (the descriptors and opts, byte for byte; up to 4
 * batches): the second call with the same batch captures the sequence into a CUDA
 * graph (opts->use_graph), later calls replay it.  With opts->check_finite the
 * candidates are scanned when a batch is first seen and the queries on every call.
 * opts->select is not used here: every set runs with the bounds opts enables.
 */
typedef struct {
    const float *cand; /* device [N][L][D], row-major, N >= 1 */
    int64_t N;
    int32_t L, D, W, K; /* L >= 1, 1 <= D <= 64, W >= 0 (clamped to L-1), K >= 1 */
    const float *q;    /* device [M][L][D] */
    int64_t M;         /* M >= 0; M == 0: entry skipped */
    int64_t *idx;      /* device [M], output */
    double *dist;      /* device [M], output */
} tcdtw_dataset;

/* sets: HOST array of nsets descriptors (the library keeps none of the pointers
 * beyond the cached launch, which re-reads the same device buffers on replay).
 * opts: NULL = defaults.  stats: host, may be NULL (summed over all sets).
 * The call is synchronous on `stream` (it reads the launch's device status word).
 * Errors: INVALID, NOMEM, CUDA, NONFINITE, TIMEOUT, UNSUPPORTED (D > 64). */
int tcdtw_batch_nn(const tcdtw_dataset *sets, int32_t nsets, const tcdtw_opts *opts,
                   tcdtw_stats *stats, void *stream);

/* The band tile tcdtw_batch_nn gives each set (host outputs R[k], G[k]: rows per lane
 * and lanes per pair of its DTW launches; 0, 0 for a set searched through tcdtw_nn or
 * with M == 0).  Each set of the batched path takes the (tile, G) that the single-set
 * tuner measures fastest for its (L, D, W) on its own candidates (cached per shape; see
 * TCDTW_TUNE_CACHE at tcdtw_build), when the batched launches compile that tile (R in
 * {4, 8, 16} for D <= 8, {4, 8} for D = 9..12), else 8 rows per lane with the smallest
 * valid G.  May run the tuner (kernels on `stream`, synchronised).
 * Errors: INVALID, NOMEM, CUDA. */
int tcdtw_batch_tiles(const tcdtw_dataset *sets, int32_t nsets, const tcdtw_opts *opts, int32_t *R,
                      int32_t *G, void *stream);

/* Release the batch sequences tcdtw_batch_nn keeps (CUDA graphs and workspaces of
 * up to 4 distinct batches) after waiting for the device; the next call builds its
 * sequence again.  Errors: CUDA. */
int tcdtw_batch_release(void);

/* Failure-detection self-test of the batched launch (no counterpart in the paper):
 * one persistent launch whose only work item waits for a device counter that
 * nothing increments, with a limit of spin_limit sleeps of ~256 ns.  The wait runs
 * out, the launch records TIMEOUT in its status word and returns; the context stays
 * usable.  Returns TIMEOUT on success of the self-test, INVALID for spin_limit < 1,
 * CUDA on a runtime error.  Synchronous on `stream`. */
int tcdtw_batch_selftest_timeout(int64_t spin_limit, void *stream);

/* Failure-detection self-test of the TMA-fed LB_MV stream (no counterpart in the
 * paper): one CTA whose producer warp issues no copy, so the consumers' wait for the
 * first chunk runs out after wait_us microseconds; the launch records TIMEOUT in its
 * status word and returns, and the context stays usable.  Returns TIMEOUT on success
 * of the self-test, INVALID for wait_us outside [1, 10^7], NOMEM, CUDA on a runtime
 * error.  Synchronous on `stream`. */
int tcdtw_lb_mv_selftest_timeout(int64_t wait_us, void *stream);
/* The same test for the bulk-tensor completion kernel of the abandoning LB_MV
 * (tcdtw_lb_mv_abandon, mv_abandon): a launch whose producer issues nothing, so its
 * consumers' first wait runs out after wait_us microseconds.  Synchronous on `stream`.
 * Returns TIMEOUT when the wait limit worked; INVALID (wait_us outside [1, 1e7]),
 * NOMEM, CUDA. */
int tcdtw_lb_mv_rest_selftest_timeout(int64_t wait_us, void *stream);

/* Number of compiled DTW band tiles, and the shape of tile t: G lanes per pair,
 * R rows per lane (host outputs).  Returns INVALID for an unknown t. */
int tcdtw_tile_count(void);
int tcdtw_tile_info(int32_t t, int32_t *G, int32_t *R, int32_t *maxD);

/* Failure injection for tests (host side; not in the paper): after `after` more
 * successful device allocations by the library, every later one fails as if the
 * device were out of memory -- no cudaMalloc is made -- and the calling entry point
 * returns TCDTW_ERR_NOMEM after releasing what it had allocated.  after = -1 turns
 * the injection off (the default); after = 0 fails the next allocation.  The setting
 * is process-wide.  Errors: INVALID (after < -1). */
int tcdtw_inject_alloc_failure(int64_t after);

/* Static message for an error code. */
const char *tcdtw_strerror(int code);

/* Name and message of the last CUDA runtime error this thread's calls returned as
 * TCDTW_ERR_CUDA or TCDTW_ERR_NOMEM ("" if none); valid until the thread's next such error. */
const char *tcdtw_last_error_detail(void);

#ifdef __cplusplus
}
#endif

#endif /* TCDTW_H */
