// api_batch.cu -- C ABI of the batched search over many independent uneven sets.
#include <cuda_runtime.h>
#include <string.h>

#include "api_internal.h"
#include "common.cuh"

extern "C" {

int tcdtw_batch_nn(const tcdtw_dataset *sets, int32_t nsets, const tcdtw_opts *opts, tcdtw_stats *stats,
                   void *stream) {
    if (nsets < 0 || (nsets > 0 && !sets)) return TCDTW_ERR_INVALID;
    if (stats) memset(stats, 0, sizeof(*stats));
    for (int32_t k = 0; k < nsets; ++k) {
        const tcdtw_dataset &d = sets[k];
        tcdtw_index *x = nullptr;
        int rc = tcdtw_build(d.cand, d.N, d.L, d.D, d.W, d.K, opts, stream, &x);
        if (rc) return rc;
        tcdtw_stats st;
        rc = tcdtw_nn(x, d.q, d.M, d.idx, d.dist, stats ? &st : nullptr, stream);
        tcdtw_free(x);
        if (rc) return rc;
        if (stats) {
            stats->pairs += st.pairs; stats->pruned_mv += st.pruned_mv; stats->pruned_pc += st.pruned_pc;
            stats->pruned_ti += st.pruned_ti; stats->dtw_started += st.dtw_started;
            stats->dtw_abandoned += st.dtw_abandoned; stats->cells += st.cells; stats->refined += st.refined;
        }
    }
    return TCDTW_OK;
}

}  // extern "C"
