// lb_kernels.cuh -- launch records and launchers of the preparation, lower-bound,
// compaction and selection kernels (prep.cu, lb.cu).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "common.cuh"

namespace tc {

// prep.cu
cudaError_t launch_check_finite(const float *x, int64_t n, DevStatus *st, int where, cudaStream_t s);
cudaError_t launch_envelope(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo, int ldE,
                            cudaStream_t s);
// envelope in the query-pair interleaved layout of the LB_MV stream:
// element e of query m at ((m/2)*ldE + e)*2 + m%2, entries e >= L*D set to +-inf
cudaError_t launch_envelope_pairs(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo, int ldE,
                                  cudaStream_t s);
// both layouts at once: query-pair interleaved (U, Lo) and one query per row (U2, Lo2:
// element e of query m at m*ldE + e, entries e >= L*D set to +-inf)
cudaError_t launch_envelope_pairs_plain(const float *q, int64_t M, int L, int D, int W, float *U, float *Lo,
                                        float *U2, float *Lo2, int ldE, cudaStream_t s);
cudaError_t launch_query_dq(const float *q, int64_t M, int L, int D, float *dq_lo, float *dq_hi, cudaStream_t s);
size_t pc_boxes_smem(int L, int D, int W, int K, int w, int *npow2_out);
cudaError_t launch_pc_boxes(const float *q, int64_t M, int L, int D, int W, int K, int Lq, int w, float *boxes,
                            int32_t *counts, cudaStream_t s);

// lb.cu -- LB_MV over all (query, candidate) pairs of a block
struct LbMvArgs {
    const float *cand;  // [N][ldC]: rows of Erow valid elements
    int64_t N;
    int E;              // elements the stream sums per pair: ceil(E/32) chunks of 32, chunk k
                        // starting at row element k * cstride * 32
    int64_t ldC = 0;    // row stride of cand in floats (0: E)
    int Erow = 0;       // valid elements per row (0: E)
    int cstride = 1;    // row chunks per stream chunk (1: the first E elements)
    const float *U;     // query-pair interleaved envelope [(Mb+1)/2][ldE][2], +inf beyond E
    const float *Lo;    // likewise, -inf beyond E
    int64_t ldE;        // multiple of 32
    int Mb;
    float *lb;          // [Mb][ldLb]
    int64_t ldLb;
    int sms;
    // device status word for the bounded waits of the TMA stream; null selects the
    // cp.async stream (which has no waits)
    DevStatus *status = nullptr;
    // optional: workspace for the partial sums of split tiles (ws_floats floats) and
    // per-tile arrival counters (tile_cnt_cap ints, zero before the first use; every
    // launch leaves them zero); without them every tile is one work unit
    float *ws = nullptr;
    int64_t ws_floats = 0;
    int *tile_cnt = nullptr;
    int64_t tile_cnt_cap = 0;
};
cudaError_t launch_lb_mv(const LbMvArgs &a, cudaStream_t s);
// lb_tma.cu: the same stream fed by bulk-tensor copies (needs E % 4 == 0, 16-byte
// aligned candidates and envelopes, and a status word); cudaErrorNotSupported when
// the arguments do not qualify
bool lb_mv_tma_ok(const LbMvArgs &a);
// workspace sizes that let the TMA stream split every tile it needs to split
constexpr int64_t kMvWsFloats = (int64_t)1 << 23;
constexpr int64_t kMvTileCounters = 4096;
cudaError_t launch_lb_mv_tma(const LbMvArgs &a, cudaStream_t s);
// whether the LB_MV stream may copy candidate rows 16 bytes at a time
bool lb_mv_vec4(const float *cand, int E);

// lb_rest.cu -- completion of LB_MV, with early abandoning, for the pairs whose sum over
// a sample of their elements (already in lb) is at most their query's threshold; the
// others keep that partial sum.  The sample is samp chunks of 32 elements spread over
// the row, chunk k * sstride for k < samp.  Completed and abandoned values are written
// in place.
constexpr int kRestTC = 224;   // candidates per tile, at most
constexpr int kRestQG = 256;   // queries staged per pass, at most
struct LbMvRestArgs {
    const float *cand;      // [N][ldC], elements [0, E) used
    int64_t N;
    int E;
    int samp, sstride;      // the sampled chunks, already summed (samp >= 1, chunks full)
    int64_t ldC;
    const float *Up, *Lp;   // envelope, one query per row: [Mb][ldP], +inf / -inf beyond E
    int64_t ldP;            // a multiple of 32, >= E
    int Mb;
    float *lb;              // [Mb][ldLb]: sample sums in, bounds out
    int64_t ldLb;
    const float *thresh;    // [Mb] thresholds, or null: prune_threshold(bsf[m], rho)
    const unsigned long long *bsf;
    float rho;
    uint32_t *list;         // scratch: lb_mv_rest_list_entries(N, Mb, sms) entries
    int64_t list_entries;
    int sms;
    unsigned long long *terms = nullptr;  // optional: += the (element, pair) terms summed
    DevStatus *status = nullptr;          // bounded waits of the bulk-tensor form (null: cp.async form)
    uint64_t wait_ns = 0;                 // their limit (0: the library default)
    int stall = 0;                        // self-test: the producer issues nothing
};
int lb_mv_rest_tile(int64_t N, int sms);
int64_t lb_mv_rest_list_entries(int64_t N, int Mb, int sms);
cudaError_t launch_lb_mv_rest(const LbMvRestArgs &a, cudaStream_t s);
// Sample of the abandoning LB_MV for rows of E elements: the number of sampled chunks
// (0: no abandoning, the rows are too short for it to pay) and their stride in chunks.
// Chunks 0, stride, 2*stride, ... lie before the last chunk, so each is whole.  The
// sample spreads over the whole series, so its sums rank candidates much as the full
// bound does (a prefix would rank them by their first few points only).
inline int lb_mv_sample(int E, int *stride) {
    const int nchunks = (E + 31) / 32;
    *stride = 1;
    if (nchunks < 4) return 0;
    int c = nchunks / 16;
    if (c < 1) c = 1;
    if (c > 8) c = 8;
    *stride = nchunks / c;
    return c;
}
// Whether row chunk c belongs to that sample.
__host__ __device__ inline bool lb_mv_sampled(int c, int samp, int sstride) {
    return c % sstride == 0 && c / sstride < samp;
}

// compaction of rows of a bound matrix against per-row thresholds
struct CompactArgs {
    const float *lb;
    int64_t M, N, ldLb;
    const float *thresh;             // [M] or null
    const unsigned long long *bsf;   // used when thresh is null
    float rho;
    int32_t *counts;                 // [M]
    int32_t *offsets;                // [M] flat-list mode, or null for per-row mode
    int32_t *total;                  // flat-list mode
    int64_t ldOut;                   // per-row mode: row stride of idx_out
    uint32_t *pairs;                 // flat-list mode: m*N + n
    float *lbs;                      // flat-list mode: bound of each entry
    int32_t *idx_out;                // per-row mode: n
    unsigned long long *pruned;      // optional counter of dropped entries
};
cudaError_t launch_compact(const CompactArgs &a, cudaStream_t s);
cudaError_t launch_seed_topk(float *lb, int64_t M, int64_t N, int64_t ldLb, int S, uint32_t *seeds, cudaStream_t s);

// tight bounds on listed pairs
struct PairListArgs {
    const float *Q;          // [Mb][L][D]
    const float *C;          // [N][L][D]
    int L, D, W;
    const uint32_t *pairs;   // entry -> m*N + n (UINT32_MAX = empty)
    const int32_t *count;    // device entry count, or null (n_static)
    int64_t n_static;
    int64_t N;
    float *lb;               // in/out bound per entry (+inf = dropped)
};
cudaError_t launch_lb_pc_list(const PairListArgs &a, const float *boxes, const int32_t *counts, int K, int w,
                              const unsigned long long *bsf, float rho, float e_gate, unsigned long long *stat_pruned,
                              int64_t n_hint, int sms, cudaStream_t s);
// LB_TI without the exact window top (basic when P >= L, TIP otherwise): W <= 127
bool lb_ti_rows_supported(int W);
cudaError_t launch_lb_ti_rows_list(const PairListArgs &a, const float *dq_lo, const float *dq_hi, int P,
                                   const unsigned long long *bsf, float rho, float e_gate,
                                   unsigned long long *stat_pruned, int64_t n_hint, int sms, cudaStream_t s);
// candidate-side LB_MV of listed pairs (bsf == null: threshold +inf, every bound kept)
cudaError_t launch_lb_rev_list(const PairListArgs &a, const float *Uc, const float *Lc, const unsigned long long *bsf,
                               float rho, unsigned long long *stat_pruned, int64_t n_hint, int sms, cudaStream_t s);
cudaError_t launch_lb_ti_list(const PairListArgs &a, const float *dq_lo, const float *dq_hi, int P,
                              const unsigned long long *bsf, float rho, float e_gate, unsigned long long *stat_pruned,
                              int64_t n_hint, int sms, cudaStream_t s);

// refine / select
cudaError_t launch_refine_select(const uint32_t *pairs, const float *dtw, const int32_t *count, int64_t n_static,
                                 int64_t N, const unsigned long long *bsf, float rho, uint32_t *out,
                                 int32_t *out_count, int64_t cap, int sms, cudaStream_t s);
cudaError_t launch_refine_pick(const uint32_t *pairs, const double *d64, const int32_t *count, int64_t N,
                               const unsigned long long *best64, unsigned long long *best_idx, int sms,
                               cudaStream_t s);
// double-float refine: per-query count of inseparable entries and the index at the
// best double-float value; entries of queries that need FP64 go to a second list
cudaError_t launch_refine_amb(const uint32_t *pairs, const double *v, const int32_t *count, int64_t N,
                              const unsigned long long *bestdf, double kappa, int32_t *amb,
                              unsigned long long *best_idx_df, int sms, cudaStream_t s);
cudaError_t launch_refine_need64(const uint32_t *pairs, const double *v, const int32_t *count, int64_t N,
                                 const unsigned long long *bestdf, double kappa, const int32_t *amb, uint32_t *out,
                                 int32_t *out_count, int64_t cap, int sms, cudaStream_t s);
cudaError_t launch_finalize(int64_t Mb, const unsigned long long *bestdf, const unsigned long long *best_idx_df,
                            const int32_t *amb, const unsigned long long *best64, const unsigned long long *best_idx,
                            int64_t *idx, double *dist, cudaStream_t s);
cudaError_t launch_init_block(int64_t Mb, unsigned long long *bsf, unsigned long long *best64,
                              unsigned long long *best_idx, unsigned long long *bestdf,
                              unsigned long long *best_idx_df, int32_t *amb, cudaStream_t s);
cudaError_t launch_count_add(unsigned long long *acc, const int32_t *v, cudaStream_t s);
cudaError_t launch_iota_pairs(uint32_t *p, int64_t n, cudaStream_t s);

}  // namespace tc
