// Query request descriptors and launchers shared by the single-batch query,
// the multi-request query, the CUDA-graph batcher and the autotuner.
#pragma once

#include "mk_host.h"

namespace mk {

// One query request (layout identical to the public mk_query_req).
struct QueryReq {
    const uint32_t *src;
    const uint32_t *dst;
    uint64_t n;
    uint32_t *bitmap;
    uint32_t *w;
};

cudaError_t launch_query(mk_graph *g, int group, int block, const uint32_t *src, const uint32_t *dst, uint64_t n,
                         uint32_t *bitmap, uint32_t *w, cudaStream_t s);
cudaError_t launch_query_multi(mk_graph *g, int group, int block, int grid, const QueryReq *reqs,
                               const uint64_t *prefix, uint32_t nreq, const uint64_t *total, cudaStream_t s);

} // namespace mk
