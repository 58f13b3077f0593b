// batch.cu -- dupin_peel_batch: many independent graphs.
#include <cuda_runtime.h>

#include <string>

#include "dupin_internal.h"

extern "C" int dupin_peel_batch(dupin_graph *const *graphs, const dupin_params *params, dupin_result *results,
                                int64_t count, void *stream) {
    if (count < 0) return dupin_fail(DUPIN_ERR_INVALID_ARG, "count < 0");
    if (count > 0 && (!graphs || !params || !results))
        return dupin_fail(DUPIN_ERR_INVALID_ARG, "graphs, params and results must be non-NULL");
    for (int64_t j = 0; j < count; j++) {
        int rc = dupin_peel(graphs[j], &params[j], &results[j], stream);
        if (rc) {
            char buf[512];
            dupin_last_error(buf, sizeof(buf));
            return dupin_fail(rc, "graph " + std::to_string(j) + ": " + buf);
        }
    }
    return DUPIN_OK;
}
