// Batched edge query (paper, Sec. "Experimental Evaluation", query: the
// destination is hashed to one bucket of the source and only that chain is
// walked; the walk stops at the key, at the first free pair or at the end).
//
// Queries are independent, so the batch is not sorted.  One warp answers 32
// consecutive queries (a chunk): each lane first fetches the source's bucket
// range for its own query (32 independent gathers in flight), then the warp
// walks 32/G chains at a time, one per G-lane group, each lane loading 32/G
// consecutive words of the 128-byte slab as one vector (G = 8: 16 bytes, two
// pairs per lane; G = 32: one word per lane, the paper's layout).  The warp
// writes one bitmap word per chunk.  G and the block size are picked by the
// autotuner (mk_autotune); the default is G = 8, 256 threads.
//
// The multi-request form runs the chunks of many query requests in one
// persistent grid-stride launch: chunk c belongs to the request whose chunk
// range [prefix[r], prefix[r+1]) contains it, so uneven requests share one
// launch (and one CUDA graph node) instead of one launch each.
#include "mk_host.h"
#include "mk_query.h"

#include <algorithm>
#include <cstring>

using namespace mk;

namespace {

template <int W>
struct Vec;
template <>
struct Vec<1> {
    static __device__ __forceinline__ void load(const uint32_t *p, uint32_t *w) { w[0] = __ldg(p); }
};
template <>
struct Vec<2> {
    static __device__ __forceinline__ void load(const uint32_t *p, uint32_t *w)
    {
        const uint2 x = __ldg(reinterpret_cast<const uint2 *>(p));
        w[0] = x.x;
        w[1] = x.y;
    }
};
template <>
struct Vec<4> {
    static __device__ __forceinline__ void load(const uint32_t *p, uint32_t *w)
    {
        const uint4 x = __ldg(reinterpret_cast<const uint4 *>(p));
        w[0] = x.x;
        w[1] = x.y;
        w[2] = x.z;
        w[3] = x.w;
    }
};
template <>
struct Vec<8> {
    static __device__ __forceinline__ void load(const uint32_t *p, uint32_t *w)
    {
        Vec<4>::load(p, w);
        Vec<4>::load(p + 4, w + 4);
    }
};

// Answers the 32 queries [q0, q0 + 32) (those below n) of one request.
template <int G>
__device__ __forceinline__ void query_chunk(const GView &g, const uint32_t *__restrict__ src,
                                            const uint32_t *__restrict__ dst, uint64_t n, uint64_t q0,
                                            uint32_t *__restrict__ bitmap_word, uint32_t *__restrict__ w_out,
                                            uint32_t max_hops, unsigned long long &loads)
{
    constexpr uint32_t W = 32 / G;        // words per lane
    constexpr uint32_t kGroups = 32 / G;  // chains in flight per warp
    const uint32_t lane = lane_id();
    const uint64_t q = q0 + lane;
    uint32_t my_d = kNil, my_head = kNil;
    bool bad = false;
    if (q < n) {
        const uint32_t s = __ldg(src + q);
        my_d = __ldg(dst + q);
        if (s < g.V && my_d < g.V) {
            const uint2 vi = __ldg(&g.vinfo[s]);
            my_head = vi.x + bucket_of(my_d, vi.y);
        } else {
            bad = true;
        }
    }
    if (__ballot_sync(kFull, bad) && lane == 0)
        set_status(g.st, kErrInvalid);
    const uint32_t gi = lane / G, sub = lane % G;
    const uint32_t gmask = (G == 32 ? kFull : ((1u << G) - 1u)) << (gi * G);
    uint32_t word_bits = 0;
#pragma unroll 1
    for (uint32_t it = 0; it < 32 / kGroups; ++it) {
        const uint32_t who = it * kGroups + gi;
        const uint32_t d = __shfl_sync(kFull, my_d, who);
        uint32_t slab = __shfl_sync(kFull, my_head, who);
        bool active = slab != kNil;
        bool found = false;
        for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
            loads += __popc(__ballot_sync(kFull, active && sub == 0));
            uint32_t w[W];
#pragma unroll
            for (uint32_t k = 0; k < W; ++k)
                w[k] = kFull;
            if (active)
                Vec<W>::load(slab_ptr(g, slab) + sub * W, w);
            bool hit = false, emp = false;
            uint32_t wt = 0;
#pragma unroll
            for (uint32_t k = 0; k < W; ++k) {
                const uint32_t word = sub * W + k;
                if (is_key_lane(word)) {
                    if (w[k] == d && active) {
                        hit = true;
                        if (W > 1)
                            wt = w[k + 1 < W ? k + 1 : k];
                    }
                    emp |= active && w[k] == kEmptyKey;
                }
            }
            if (W == 1) {
                // the weight of a key in word 2p sits in the next lane
                const uint32_t nw = __shfl_down_sync(kFull, w[0], 1);
                if (hit)
                    wt = nw;
            }
            const uint32_t hm = __ballot_sync(kFull, hit) & gmask;
            const uint32_t em = __ballot_sync(kFull, emp) & gmask;
            const uint32_t nxt = __shfl_sync(kFull, w[W - 1], gi * G + G - 1);
            if (hit && w_out)
                w_out[q0 + who] = wt;
            if (hm)
                found = true;
            if (active && (hm || em || nxt == kNil || hop >= max_hops))
                active = false;
            else if (active)
                slab = nxt;
        }
        const uint32_t fb = __ballot_sync(kFull, sub == 0 && found);
        uint32_t packed = 0;
#pragma unroll
        for (uint32_t k = 0; k < kGroups; ++k)
            packed |= ((fb >> (k * G)) & 1u) << k;
        word_bits |= packed << (it * kGroups);
        if (w_out && sub == 0 && !found && q0 + who < n)
            w_out[q0 + who] = 0;
    }
    if (lane == 0)
        *bitmap_word = word_bits;
}

template <int G>
__global__ void __launch_bounds__(512) k_query(GView g, const uint32_t *__restrict__ src,
                                               const uint32_t *__restrict__ dst, uint64_t n,
                                               uint32_t *__restrict__ bitmap, uint32_t *__restrict__ w_out,
                                               uint32_t max_hops)
{
    const unsigned long long warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t base = warp * 32;
    if (base >= n || status_hint(g.st) != 0)
        return;
    unsigned long long loads = 0;
    query_chunk<G>(g, src, dst, n, base, bitmap + warp, w_out, max_hops, loads);
    count_add(g.st, kCtrQuerySlabs, loads);
}

// Chunks of many requests, grid-stride.  total[0] = number of chunks and
// total[1] = number of requests, read on the device so that a captured graph
// can be replayed with other requests.
template <int G>
__global__ void __launch_bounds__(512) k_query_multi(GView g, const QueryReq *__restrict__ reqs,
                                                     const uint64_t *__restrict__ prefix, uint32_t nreq_max,
                                                     const uint64_t *__restrict__ total, uint32_t max_hops)
{
    if (status_hint(g.st) != 0)
        return;
    const uint64_t nchunks = total[0];
    const uint32_t nreq = total[1] < nreq_max ? (uint32_t)total[1] : nreq_max;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long loads = 0;
    for (uint64_t c = warp0; c < nchunks; c += nwarps) {
        // request r with prefix[r] <= c < prefix[r + 1]
        uint32_t lo = 0, hi = nreq;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (prefix[mid] <= c)
                lo = mid;
            else
                hi = mid;
        }
        const QueryReq r = reqs[lo];
        const uint64_t local = c - prefix[lo];
        query_chunk<G>(g, r.src, r.dst, r.n, local * 32, r.bitmap + local, r.w, max_hops, loads);
    }
    count_add(g.st, kCtrQuerySlabs, loads);
}

} // namespace

namespace mk {

cudaError_t launch_query(mk_graph *g, int group, int block, const uint32_t *src, const uint32_t *dst, uint64_t n,
                         uint32_t *bitmap, uint32_t *w, cudaStream_t s)
{
    const uint32_t max_hops = g->v.P + 2;
    const uint32_t grid = grid_for(n, (uint32_t)block);
    switch (group) {
    case 4: k_query<4><<<grid, block, 0, s>>>(g->v, src, dst, n, bitmap, w, max_hops); break;
    case 16: k_query<16><<<grid, block, 0, s>>>(g->v, src, dst, n, bitmap, w, max_hops); break;
    case 32: k_query<32><<<grid, block, 0, s>>>(g->v, src, dst, n, bitmap, w, max_hops); break;
    default: k_query<8><<<grid, block, 0, s>>>(g->v, src, dst, n, bitmap, w, max_hops); break;
    }
    return cudaGetLastError();
}

cudaError_t launch_query_multi(mk_graph *g, int group, int block, int grid, const QueryReq *reqs,
                               const uint64_t *prefix, uint32_t nreq, const uint64_t *total, cudaStream_t s)
{
    const uint32_t max_hops = g->v.P + 2;
    switch (group) {
    case 4: k_query_multi<4><<<grid, block, 0, s>>>(g->v, reqs, prefix, nreq, total, max_hops); break;
    case 16: k_query_multi<16><<<grid, block, 0, s>>>(g->v, reqs, prefix, nreq, total, max_hops); break;
    case 32: k_query_multi<32><<<grid, block, 0, s>>>(g->v, reqs, prefix, nreq, total, max_hops); break;
    default: k_query_multi<8><<<grid, block, 0, s>>>(g->v, reqs, prefix, nreq, total, max_hops); break;
    }
    return cudaGetLastError();
}

} // namespace mk

extern "C" mk_status mk_query_batch(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                                    uint32_t *d_bitmap, uint32_t *d_w, void *stream)
{
    if (!g || (n > 0 && (!d_src || !d_dst || !d_bitmap)) || n >= 0xFFFFFFFFull)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 0)
        return MK_OK;
    return timed(g, "query", s, 1, [&]() {
        return launch_query(g, g->tune.query_group, g->tune.query_block, d_src, d_dst, n, d_bitmap, d_w, s);
    });
}
