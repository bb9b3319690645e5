// Batching and autotuning.
//
//  * mk_query_multi: many uneven query requests in one persistent launch.
//  * mk_batcher: the same launch captured once in a CUDA graph (descriptor
//    copy + multi-request kernel) and replayed for every later group of
//    requests, so a serving tick costs one graph launch.
//  * mk_autotune: times the query kernel for every slab tile width (4, 8, 16
//    or 32 lanes per chain) and block size, and the persistent round kernel
//    for every number of blocks per SM, on the caller's graph and sample,
//    and keeps the fastest shapes for this graph.
#include "mk_host.h"
#include "mk_query.h"

#include <algorithm>
#include <cstring>
#include <vector>

using namespace mk;

namespace mk {
mk_status time_static_bfs(mk_graph *g, uint32_t source, cudaStream_t s, float *ms);
}

namespace {

int multi_grid(int block)
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    }
    return sms * std::max(1, 2048 / block);
}

// Device layout of one group of requests: requests, chunk prefix (nreq + 1)
// and {total chunks, nreq}.
struct ReqBlock {
    size_t bytes = 0;
    uint32_t cap = 0;
    static size_t size_for(uint32_t cap) { return cap * sizeof(QueryReq) + (cap + 1) * 8 + 16; }
};

// Fills a host image of the block; returns the total chunk count.
uint64_t fill_block(unsigned char *img, uint32_t cap, const mk_query_req *reqs, uint32_t nreq)
{
    QueryReq *r = reinterpret_cast<QueryReq *>(img);
    uint64_t *prefix = reinterpret_cast<uint64_t *>(img + cap * sizeof(QueryReq));
    uint64_t *total = prefix + cap + 1;
    uint64_t acc = 0;
    for (uint32_t i = 0; i < nreq; ++i) {
        r[i].src = reqs[i].d_src;
        r[i].dst = reqs[i].d_dst;
        r[i].n = reqs[i].n;
        r[i].bitmap = reqs[i].d_bitmap;
        r[i].w = reqs[i].d_w;
        prefix[i] = acc;
        acc += (reqs[i].n + 31) / 32;
    }
    prefix[nreq] = acc;
    total[0] = acc;
    total[1] = nreq;
    return acc;
}

} // namespace

struct mk_batcher {
    mk_graph *g = nullptr;
    uint32_t cap = 0;
    size_t bytes = 0;
    cudaStream_t stream = nullptr;        // private stream (capture needs a non-legacy stream)
    unsigned char *h_img[2] = {nullptr, nullptr};
    unsigned char *d_blk[2] = {nullptr, nullptr};
    cudaGraphExec_t exec[2] = {nullptr, nullptr};
    cudaEvent_t done[2] = {nullptr, nullptr};
    cudaEvent_t ready = nullptr;
    int slot = 0;
    int group = 8, block = 256;
    std::vector<mk_query_req> pending;
    uint64_t launches = 0;
};

extern "C" {

mk_status mk_query_multi(mk_graph *g, const mk_query_req *h_reqs, uint32_t nreq, void *stream)
{
    if (!g || (nreq && !h_reqs))
        return MK_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < nreq; ++i)
        if (h_reqs[i].n && (!h_reqs[i].d_src || !h_reqs[i].d_dst || !h_reqs[i].d_bitmap))
            return MK_ERR_INVALID_ARG;
    if (!nreq)
        return MK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<unsigned char> img(ReqBlock::size_for(nreq));
    const uint64_t total = fill_block(img.data(), nreq, h_reqs, nreq);
    if (!total)
        return MK_OK;
    unsigned char *d = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&d, img.size(), s));
    MK_CUDA(cudaMemcpyAsync(d, img.data(), img.size(), cudaMemcpyHostToDevice, s));
    const QueryReq *reqs = reinterpret_cast<const QueryReq *>(d);
    const uint64_t *prefix = reinterpret_cast<const uint64_t *>(d + nreq * sizeof(QueryReq));
    const uint64_t *tot = prefix + nreq + 1;
    const int grid = (int)std::min<uint64_t>((uint64_t)multi_grid(g->tune.query_block),
                                             (total * 32 + g->tune.query_block - 1) / g->tune.query_block);
    mk_status st = timed(g, "query_multi", s, 1, [&]() {
        return launch_query_multi(g, g->tune.query_group, g->tune.query_block, std::max(grid, 1), reqs, prefix, nreq,
                                  tot, s);
    });
    cudaFreeAsync(d, s);
    return st;
}

mk_status mk_batcher_create(mk_graph *g, uint32_t max_requests, mk_batcher **out)
{
    if (!g || !out || !max_requests)
        return MK_ERR_INVALID_ARG;
    mk_batcher *b = new mk_batcher;
    b->g = g;
    b->cap = max_requests;
    b->bytes = ReqBlock::size_for(max_requests);
    b->group = g->tune.query_group;
    b->block = g->tune.query_block;
    bool ok = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->ready, cudaEventDisableTiming) == cudaSuccess;
    for (int k = 0; k < 2 && ok; ++k) {
        ok = cudaMallocHost((void **)&b->h_img[k], b->bytes) == cudaSuccess &&
             cudaMalloc((void **)&b->d_blk[k], b->bytes) == cudaSuccess &&
             cudaEventCreateWithFlags(&b->done[k], cudaEventDisableTiming) == cudaSuccess;
        if (ok) {
            std::memset(b->h_img[k], 0, b->bytes);
            ok = cudaMemset(b->d_blk[k], 0, b->bytes) == cudaSuccess;
        }
    }
    if (!ok) {
        mk_batcher_destroy(b);
        return MK_ERR_NO_MEMORY;
    }
    // capture one graph per slot: descriptor copy, then the multi-request
    // kernel reading sizes from the copied block
    const int grid = multi_grid(b->block);
    for (int k = 0; k < 2; ++k) {
        cudaGraph_t graph = nullptr;
        const QueryReq *reqs = reinterpret_cast<const QueryReq *>(b->d_blk[k]);
        const uint64_t *prefix = reinterpret_cast<const uint64_t *>(b->d_blk[k] + b->cap * sizeof(QueryReq));
        const uint64_t *tot = prefix + b->cap + 1;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            mk_batcher_destroy(b);
            return MK_ERR_CUDA;
        }
        cudaMemcpyAsync(b->d_blk[k], b->h_img[k], b->bytes, cudaMemcpyHostToDevice, b->stream);
        launch_query_multi(g, b->group, b->block, grid, reqs, prefix, b->cap, tot, b->stream);
        cudaError_t e = cudaStreamEndCapture(b->stream, &graph);
        if (e == cudaSuccess)
            e = cudaGraphInstantiate(&b->exec[k], graph, 0);
        if (graph)
            cudaGraphDestroy(graph);
        if (e != cudaSuccess) {
            cudaGetLastError();
            mk_batcher_destroy(b);
            return MK_ERR_CUDA;
        }
    }
    *out = b;
    return MK_OK;
}

mk_status mk_batcher_destroy(mk_batcher *b)
{
    if (!b)
        return MK_ERR_INVALID_ARG;
    if (b->stream)
        cudaStreamSynchronize(b->stream);
    for (int k = 0; k < 2; ++k) {
        if (b->exec[k])
            cudaGraphExecDestroy(b->exec[k]);
        if (b->h_img[k])
            cudaFreeHost(b->h_img[k]);
        if (b->d_blk[k])
            cudaFree(b->d_blk[k]);
        if (b->done[k])
            cudaEventDestroy(b->done[k]);
    }
    if (b->ready)
        cudaEventDestroy(b->ready);
    if (b->stream)
        cudaStreamDestroy(b->stream);
    delete b;
    return MK_OK;
}

mk_status mk_batcher_add_query(mk_batcher *b, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                               uint32_t *d_bitmap, uint32_t *d_w)
{
    if (!b || (n && (!d_src || !d_dst || !d_bitmap)))
        return MK_ERR_INVALID_ARG;
    if (b->pending.size() >= b->cap)
        return MK_ERR_INVALID_ARG;
    b->pending.push_back({d_src, d_dst, n, d_bitmap, d_w});
    return MK_OK;
}

mk_status mk_batcher_launch(mk_batcher *b, void *stream)
{
    if (!b)
        return MK_ERR_INVALID_ARG;
    if (b->pending.empty())
        return MK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const int k = b->slot;
    // the slot's host image may still feed the copy of its previous replay
    MK_CUDA(cudaEventSynchronize(b->done[k]));
    fill_block(b->h_img[k], b->cap, b->pending.data(), (uint32_t)b->pending.size());
    b->pending.clear();
    MK_CUDA(cudaEventRecord(b->ready, s));
    MK_CUDA(cudaStreamWaitEvent(b->stream, b->ready, 0));
    mk_graph *g = b->g;
    MK_TRY(timed(g, "query_graph_tick", b->stream, 1, [&]() { return cudaGraphLaunch(b->exec[k], b->stream); }));
    MK_CUDA(cudaEventRecord(b->done[k], b->stream));
    MK_CUDA(cudaStreamWaitEvent(s, b->done[k], 0));
    b->slot ^= 1;
    b->launches++;
    return MK_OK;
}

mk_status mk_get_tuning(mk_graph *g, mk_tuning *out)
{
    if (!g || !out)
        return MK_ERR_INVALID_ARG;
    std::memset(out, 0, sizeof *out);
    out->query_group = g->tune.query_group;
    out->query_block = g->tune.query_block;
    out->rounds_blocks_per_sm = g->tune.rounds_blocks_per_sm;
    return MK_OK;
}

mk_status mk_set_tuning(mk_graph *g, const mk_tuning *t)
{
    if (!g || !t)
        return MK_ERR_INVALID_ARG;
    const int gr = t->query_group;
    if ((gr != 4 && gr != 8 && gr != 16 && gr != 32) ||
        (t->query_block != 128 && t->query_block != 256 && t->query_block != 512) || t->rounds_blocks_per_sm < 0)
        return MK_ERR_INVALID_ARG;
    g->tune.query_group = gr;
    g->tune.query_block = t->query_block;
    g->tune.rounds_blocks_per_sm = t->rounds_blocks_per_sm;
    return MK_OK;
}

mk_status mk_autotune(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n, uint32_t bfs_source,
                      void *stream, mk_tuning *out)
{
    if (!g || !out || !n || !d_src || !d_dst || bfs_source >= g->v.V)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::memset(out, 0, sizeof *out);
    uint32_t *bm = nullptr;
    MK_CUDA(cudaMalloc((void **)&bm, ((n + 31) / 32) * 4));
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    const int groups[4] = {4, 8, 16, 32}, blocks[3] = {128, 256, 512};
    float best = 1e30f;
    int n_tried = 0;
    for (int gi = 0; gi < 4; ++gi) {
        for (int bi = 0; bi < 3; ++bi) {
            float t_min = 1e30f;
            for (int rep = 0; rep < 4; ++rep) {
                cudaEventRecord(a, s);
                cudaError_t e = launch_query(g, groups[gi], blocks[bi], d_src, d_dst, n, bm, nullptr, s);
                cudaEventRecord(b, s);
                if (e != cudaSuccess || cudaEventSynchronize(b) != cudaSuccess) {
                    cudaFree(bm);
                    return MK_ERR_CUDA;
                }
                float ms = 0.f;
                cudaEventElapsedTime(&ms, a, b);
                if (rep > 0)
                    t_min = std::min(t_min, ms);
            }
            g->launches += 4;
            if (n_tried < 16)
                out->query_ms[n_tried] = t_min;
            ++n_tried;
            if (t_min < best) {
                best = t_min;
                out->query_group = groups[gi];
                out->query_block = blocks[bi];
            }
        }
    }
    out->query_best_ms = best;
    cudaFree(bm);
    g->tune.query_group = out->query_group;
    g->tune.query_block = out->query_block;
    // persistent round kernel: blocks per SM, timed on a static BFS
    const int max_bps = rounds_max_blocks_per_sm();
    float best_r = 1e30f;
    int best_bps = max_bps;
    for (int bps = 1; bps <= max_bps; ++bps) {
        g->tune.rounds_blocks_per_sm = bps;
        float t_min = 1e30f;
        for (int rep = 0; rep < 2; ++rep) {
            float ms = 0.f;
            MK_TRY(time_static_bfs(g, bfs_source, s, &ms));
            t_min = std::min(t_min, ms);
        }
        if (bps - 1 < 8)
            out->rounds_ms[bps - 1] = t_min;
        if (t_min < best_r) {
            best_r = t_min;
            best_bps = bps;
        }
    }
    g->tune.rounds_blocks_per_sm = best_bps;
    out->rounds_blocks_per_sm = best_bps;
    out->rounds_best_ms = best_r;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return MK_OK;
}

} // extern "C"
