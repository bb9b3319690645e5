// Graph analytics on the slab store beyond BFS/SSSP/WCC: PageRank (paper,
// Sec. "Dynamic PageRank", Algorithm "Page Rank - Static / Incremental /
// Decremental", Eq. 1) and triangle counting (paper, Sec. "Dynamic Triangle
// Counting", Algorithms "Triangle Counting - Incremental / Decremental" and
// the Count kernel).
//
// PageRank.  The paper's Compute kernel pulls over a graph object that
// stores in-edges; this store keeps out-edges, so each super-step pushes
// instead: every live edge u -> v adds u's contribution PR[u] / out[u] to
// v's accumulator, reading the slab array in address order (the per-slab
// owner names u), which keeps every slab read coalesced.  To make the pushes
// order-independent the ranks, contributions and accumulators are 64-bit
// fixed-point numbers (value * 2^48) added with integer atomics, so a
// result does not depend on the order in which the atomics land; the L1
// delta of a super-step is summed the same way.  The teleport term for
// zero-out-degree vertices is added as in the paper (FindTeleportProb).
// The host reads the delta after every super-step, as in the paper's loop.
//
// Triangle counting.  Count(G1, G2, edges) adds, for every edge (u, v), the
// size of the intersection of u's neighbours in G1 and v's neighbours in
// G2.  The paper walks v's slabs in G2 with a warp and lets each lane search
// G1 for (u, w); since an intersection is symmetric, this kernel walks the
// side with fewer buckets (the bucket count grows with the degree) and
// searches the other, which bounds the work of an edge between a hub and a
// leaf by the leaf's degree.
#include "mk_host.h"

#include <algorithm>
#include <cmath>
#include <cstring>
#include <vector>

using namespace mk;

namespace {

constexpr double kFix = 281474976710656.0; // 2^48: fixed-point scale of ranks
constexpr double kInvFix = 1.0 / 281474976710656.0;

// Adds the lanes' values v to *dst with one atomic per warp.
__device__ __forceinline__ void warp_add_u64(unsigned long long *dst, unsigned long long v)
{
    for (int o = 16; o; o >>= 1)
        v += __shfl_xor_sync(kFull, v, o);
    if (lane_id() == 0 && v)
        atomicAdd(dst, v);
}

} // namespace

// ----------------------------------------------------------------- PageRank

// out[u] += live pairs of every slab in use owned by u (one warp per slab,
// grid-stride; one atomic per slab).
__global__ void __launch_bounds__(256) k_pr_outdeg(GView g, uint32_t *out)
{
    const uint64_t total = (uint64_t)g.H + g.P;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t lane = lane_id();
    for (uint64_t s = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; s < total; s += stride) {
        const uint32_t own = __ldg(&g.owner[s]);
        if (own == kNil)
            continue;
        const uint32_t word = __ldcg(slab_ptr(g, (uint32_t)s) + lane);
        const uint32_t live = __ballot_sync(kFull, is_key_lane(lane) && word < kTombKey);
        if (lane == 0 && live)
            atomicAdd(&out[own], (uint32_t)__popc(live));
    }
}

// Start vector: 1 / V for every vertex (static), or the caller's ranks
// (incremental / decremental: the ranks before the batch).
__global__ void k_pr_init(unsigned long long *pr, const float *init, uint32_t V)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V)
        pr[v] = init ? __double2ull_rn((double)fmaxf(init[v], 0.f) * kFix) : __double2ull_rn(kFix / (double)V);
}

// FindContributionPerVertex: contrib[u] = PR[u] / out[u] (0 for a vertex
// without out-edges, whose rank goes to the teleport sum); clears the
// accumulators.  ctr[0] receives the teleport sum of this super-step.
__global__ void k_pr_contrib(const unsigned long long *pr, const uint32_t *out, uint32_t V,
                             unsigned long long *contrib, unsigned long long *acc, unsigned long long *ctr)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long dangling = 0;
    if (v < V) {
        const unsigned long long p = pr[v];
        const uint32_t o = out[v];
        contrib[v] = o ? p / o : 0ull;
        dangling = o ? 0ull : p;
        acc[v] = 0;
    }
    warp_add_u64(ctr, dangling);
}

// Pushes contrib[u] along every live edge u -> v.  A warp takes
// 4 * kPushHalves consecutive slabs a step, four at a time: eight lanes a
// slab, each lane one 16-byte block (two pairs; the last lane of a slab one
// pair and the unused and next words); the owners, slab parts and
// contributions of every group of four are loaded before any atomic, so
// kPushHalves independent load chains are in flight per lane.
constexpr int kPushHalves = 2;

__global__ void __launch_bounds__(256) k_pr_push(GView g, const unsigned long long *__restrict__ contrib,
                                                 unsigned long long *acc)
{
    const uint64_t nslab = (uint64_t)g.H + g.P;
    const uint32_t lane = lane_id(), part = lane & 7u, sub = lane >> 3;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t s0 = warp * (4 * kPushHalves); s0 < nslab; s0 += nwarps * (4 * kPushHalves)) {
        uint32_t own[kPushHalves];
        uint4 q[kPushHalves];
#pragma unroll
        for (int h = 0; h < kPushHalves; ++h) {
            const uint64_t s = s0 + h * 4 + sub;
            own[h] = s < nslab ? __ldg(&g.owner[s]) : kNil;
            q[h] = s < nslab ? __ldcg(reinterpret_cast<const uint4 *>(slab_ptr(g, (uint32_t)s)) + part)
                             : make_uint4(kEmptyKey, 0u, kEmptyKey, 0u);
        }
        unsigned long long c[kPushHalves];
#pragma unroll
        for (int h = 0; h < kPushHalves; ++h)
            c[h] = own[h] != kNil ? __ldg(&contrib[own[h]]) : 0ull; // an unused pool slab holds stale keys
#pragma unroll
        for (int h = 0; h < kPushHalves; ++h) {
            if (!c[h])
                continue;
            if (q[h].x < kTombKey)
                atomicAdd(&acc[q[h].x], c[h]);
            if (part != 7u && q[h].z < kTombKey)
                atomicAdd(&acc[q[h].z], c[h]);
        }
    }
}

// Compute + teleport (Eq. 1): PR[v] = (1 - d) / V + d * (acc[v] + teleport
// / V); ctr[1] receives the L1 delta of the super-step.
__global__ void k_pr_finish(unsigned long long *pr, const unsigned long long *acc, uint32_t V, double d,
                            unsigned long long base, unsigned long long *ctr)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long diff = 0;
    if (v < V) {
        const unsigned long long tele = __ldcg(&ctr[0]) / V;
        const unsigned long long nv = base + __double2ull_rn(d * (double)(acc[v] + tele));
        const unsigned long long ov = pr[v];
        diff = nv > ov ? nv - ov : ov - nv;
        pr[v] = nv;
    }
    warp_add_u64(&ctr[1], diff);
}

__global__ void k_pr_out(const unsigned long long *pr, uint32_t V, float *out)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V)
        out[v] = __double2float_rn((double)pr[v] * kInvFix);
}

// ------------------------------------------------------- triangle counting

namespace {

// Whether edge (u, w) is in g: the lane walks the chain of w's bucket among
// u's buckets, eight 16-byte loads per slab issued together.
__device__ __forceinline__ bool lane_has_edge(const GView &g, uint32_t u, uint32_t w, uint32_t max_hops)
{
    const uint2 vi = __ldg(&g.vinfo[u]);
    uint32_t slab = vi.x + bucket_of(w, vi.y);
    for (uint32_t hop = 0; hop < max_hops && slab != kNil; ++hop) {
        const uint4 *p = reinterpret_cast<const uint4 *>(slab_ptr(g, slab));
        uint4 x[8];
#pragma unroll
        for (int q = 0; q < 8; ++q)
            x[q] = __ldcg(p + q);
        bool hit = false;
#pragma unroll
        for (int q = 0; q < 8; ++q)
            hit |= x[q].x == w || (q < 7 && x[q].z == w);
        if (hit)
            return true;
        slab = x[7].w;
    }
    return false;
}

// |N_g1(u) ∩ N_g2(v)| spread over the warp's lanes (each lane returns its
// share; the full warp calls it with warp-uniform u, v).  The side with
// fewer buckets is walked (one list: slab by slab, a word a lane; several:
// eight lists at a time in 4-lane groups) and each key lane searches the
// other side for its neighbour.
__device__ __forceinline__ uint32_t warp_edge_count(const GView &g1, const GView &g2, uint32_t u, uint32_t v,
                                                    uint32_t mh1, uint32_t mh2, unsigned long long &slabs)
{
    const uint32_t lane = lane_id();
    const uint2 vu = __ldg(&g1.vinfo[u]), vv = __ldg(&g2.vinfo[v]);
    // walk N_g2(v) and search g1 for (u, w), or walk N_g1(u) and search g2 for (v, w)
    const bool walk_u = vu.y < vv.y;
    const GView &gw = walk_u ? g1 : g2;
    const GView &gs = walk_u ? g2 : g1;
    const uint2 vw = walk_u ? vu : vv;
    const uint32_t probe = walk_u ? v : u;
    const uint32_t mh = walk_u ? mh1 : mh2, mhs = walk_u ? mh2 : mh1;
    uint32_t count = 0;
    if (vw.y == 1) {
        // one list: the warp reads it slab by slab, one word a lane
        uint32_t slab = vw.x;
        for (uint32_t hop = 0; hop < mh && slab != kNil; ++hop) {
            const uint32_t word = __ldcg(slab_ptr(gw, slab) + lane);
            ++slabs;
            if (is_key_lane(lane) && word < kTombKey)
                count += lane_has_edge(gs, probe, word, mhs) ? 1u : 0u;
            slab = __shfl_sync(kFull, word, kNextLane);
        }
        return count;
    }
    // several lists: eight at a time, one per 4-lane group (bucket b by
    // group b % 8), each lane holding 32 bytes of the slab (four pairs; the
    // group's last lane three and the unused and next words)
    const uint32_t g4 = lane >> 2, s4 = lane & 3u, gbase = lane & ~3u;
    for (uint32_t b0 = 0; b0 < vw.y; b0 += 8) {
        uint32_t slab = b0 + g4 < vw.y ? vw.x + b0 + g4 : kNil;
        bool active = slab != kNil;
        for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
            uint4 lo = make_uint4(kEmptyKey, 0u, kEmptyKey, 0u), hi = lo;
            if (active) {
                const uint4 *q = reinterpret_cast<const uint4 *>(slab_ptr(gw, slab) + s4 * 8);
                lo = __ldcg(q);
                hi = __ldcg(q + 1);
                if (s4 == 0)
                    ++slabs;
            }
            const uint32_t key[4] = {lo.x, lo.z, hi.x, s4 == 3u ? kEmptyKey : hi.z};
#pragma unroll
            for (int k = 0; k < 4; ++k)
                if (active && key[k] < kTombKey)
                    count += lane_has_edge(gs, probe, key[k], mhs) ? 1u : 0u;
            const uint32_t nxt = __shfl_sync(kFull, hi.w, gbase + 3);
            if (active) {
                if (nxt == kNil || hop + 1 >= mh)
                    active = false;
                else
                    slab = nxt;
            }
        }
    }
    return count;
}

} // namespace

// Count(G1, G2, edges): total += |N_G1(u) ∩ N_G2(v)| over the n edges
// (u, v); a persistent grid whose warps take the edges one at a time from a
// shared counter (*next, zero at launch), so a few edges between two large
// neighbourhoods do not hold up a whole chunk of others.
__global__ void __launch_bounds__(256) k_tc_count(GView g1, GView g2, const uint32_t *__restrict__ src,
                                                  const uint32_t *__restrict__ dst, uint64_t n, uint32_t mh1,
                                                  uint32_t mh2, unsigned long long *total,
                                                  unsigned long long *next)
{
    const uint32_t lane = lane_id();
    unsigned long long count = 0, slabs = 0;
    for (;;) {
        unsigned long long e = 0;
        if (lane == 0)
            e = atomicAdd(next, 1ull);
        e = __shfl_sync(kFull, e, 0);
        if (e >= n)
            break;
        const uint32_t u = __ldg(src + e), v = __ldg(dst + e);
        if (u >= g1.V || v >= g2.V) {
            if (lane == 0)
                set_status(g1.st, kErrInvalid);
            continue;
        }
        count += warp_edge_count(g1, g2, u, v, mh1, mh2, slabs);
    }
    warp_add_u64(total, count);
}

namespace {

// Rank of a vertex for the oriented static count: (bucket count, id), a
// strict total order in which vertices with more buckets (higher degree at
// sizing) come later.
__device__ __forceinline__ unsigned long long tc_rank(uint32_t buckets, uint32_t x)
{
    return ((unsigned long long)buckets << 32) | x;
}

} // namespace

// Static count, each triangle once: with the vertices ranked by tc_rank, a
// triangle a < b < c is counted on its edge (a, b) as the common neighbour
// c.  One warp per slab in use (address order, owner u); each live edge
// (u, v) with rank(u) < rank(v) walks N(u) (u ranks lower, so it has no
// more buckets than v) slab by slab, and a key lane w with rank(w) > rank(v)
// looks (v, w) up.  Needs both directions of every edge stored.
__global__ void __launch_bounds__(256) k_tc_static(GView g, uint32_t mh, unsigned long long *total)
{
    const uint32_t lane = lane_id();
    const uint64_t all = (uint64_t)g.H + g.P;
    const uint64_t stride = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long count = 0;
    for (uint64_t s = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5; s < all; s += stride) {
        const uint32_t u = __ldg(&g.owner[s]);
        if (u == kNil)
            continue;
        const uint2 vu = __ldg(&g.vinfo[u]);
        const unsigned long long ru = tc_rank(vu.y, u);
        const uint32_t word = __ldcg(slab_ptr(g, (uint32_t)s) + lane);
        bool up = false;
        unsigned long long rv = 0;
        if (is_key_lane(lane) && word < kTombKey) {
            rv = tc_rank(__ldg(&g.vinfo[word]).y, word);
            up = rv > ru;
        }
        uint32_t todo = __ballot_sync(kFull, up);
        while (todo) {
            const uint32_t j = __ffs(todo) - 1;
            todo &= todo - 1;
            const uint32_t v = __shfl_sync(kFull, word, j);
            const unsigned long long rvj = __shfl_sync(kFull, rv, j);
            for (uint32_t b = 0; b < vu.y; ++b) {
                uint32_t slab = vu.x + b;
                for (uint32_t hop = 0; hop < mh && slab != kNil; ++hop) {
                    const uint32_t w = __ldcg(slab_ptr(g, slab) + lane);
                    if (is_key_lane(lane) && w < kTombKey && tc_rank(__ldg(&g.vinfo[w]).y, w) > rvj)
                        count += lane_has_edge(g, v, w, mh) ? 1u : 0u;
                    slab = __shfl_sync(kFull, w, kNextLane);
                }
            }
        }
    }
    warp_add_u64(total, count);
}

// ---------------------------------------------------------------- host side

extern "C" {

mk_status mk_pagerank(mk_graph *g, float *d_pr, int warm_start, float damping, float eps, uint32_t max_iter,
                      uint32_t *h_iters, float *h_delta, void *stream)
{
    if (!g || !d_pr || !(damping > 0.f && damping < 1.f) || !(eps > 0.f) || max_iter == 0)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t V = g->v.V;
    const uint64_t words = ((uint64_t)g->v.H + g->v.P) * 32;
    unsigned long long *pr = nullptr, *acc = nullptr, *contrib = nullptr, *ctr = nullptr;
    uint32_t *out = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&pr, (size_t)V * 8, s));
    MK_CUDA(cudaMallocAsync((void **)&acc, (size_t)V * 8, s));
    MK_CUDA(cudaMallocAsync((void **)&contrib, (size_t)V * 8, s));
    MK_CUDA(cudaMallocAsync((void **)&out, (size_t)V * 4, s));
    MK_CUDA(cudaMallocAsync((void **)&ctr, 16, s));
    MK_CUDA(cudaMemsetAsync(out, 0, (size_t)V * 4, s));
    mk_status st = timed(g, "pr_outdeg", s, 2, [&]() {
        k_pr_outdeg<<<resident_grid(k_pr_outdeg, 256), 256, 0, s>>>(g->v, out);
        k_pr_init<<<grid_for(V, 256), 256, 0, s>>>(pr, warm_start ? d_pr : nullptr, V);
        return cudaSuccess;
    });
    const double d = damping;
    const unsigned long long base = (unsigned long long)std::llround((1.0 - d) / (double)V * kFix);
    uint32_t it = 0;
    double delta = 0;
    // 4 * kPushHalves slabs per warp step
    const uint32_t push_grid = std::min<uint64_t>(grid_for(words / (4 * kPushHalves), 256),
                                                  (uint64_t)resident_grid(k_pr_push, 256) * 4);
    while (st == MK_OK && it < max_iter) {
        if (cudaMemsetAsync(ctr, 0, 16, s) != cudaSuccess) {
            st = MK_ERR_CUDA;
            break;
        }
        st = timed(g, "pr_step", s, 3, [&]() {
            k_pr_contrib<<<grid_for(V, 256), 256, 0, s>>>(pr, out, V, contrib, acc, ctr);
            k_pr_push<<<push_grid, 256, 0, s>>>(g->v, contrib, acc);
            k_pr_finish<<<grid_for(V, 256), 256, 0, s>>>(pr, acc, V, d, base, ctr);
            return cudaSuccess;
        });
        if (st != MK_OK)
            break;
        ++it;
        unsigned long long dfx = 0;
        if (cudaMemcpyAsync(g->h_pinned, ctr + 1, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = MK_ERR_CUDA;
            break;
        }
        std::memcpy(&dfx, g->h_pinned, 8);
        delta = (double)dfx * kInvFix;
        if (delta <= eps)
            break;
    }
    if (st == MK_OK)
        st = timed(g, "pr_out", s, 1, [&]() {
            k_pr_out<<<grid_for(V, 256), 256, 0, s>>>(pr, V, d_pr);
            return cudaSuccess;
        });
    cudaFreeAsync(pr, s);
    cudaFreeAsync(acc, s);
    cudaFreeAsync(contrib, s);
    cudaFreeAsync(out, s);
    cudaFreeAsync(ctr, s);
    if (h_iters)
        *h_iters = it;
    if (h_delta)
        *h_delta = (float)delta;
    return st;
}

mk_status mk_tc_count(mk_graph *g1, mk_graph *g2, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                      unsigned long long *d_total, void *stream)
{
    if (!g1 || !g2 || !d_total || (n && (!d_src || !d_dst)) || g1->v.V != g2->v.V)
        return MK_ERR_INVALID_ARG;
    if (!n)
        return MK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t grid = std::min<uint64_t>(grid_for(n * 32, 256), (uint64_t)resident_grid(k_tc_count, 256));
    unsigned long long *next = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&next, 8, s));
    MK_CUDA(cudaMemsetAsync(next, 0, 8, s));
    const mk_status st = timed(g1, "tc_count", s, 1, [&]() {
        k_tc_count<<<grid, 256, 0, s>>>(g1->v, g2->v, d_src, d_dst, n, g1->v.P + 2, g2->v.P + 2, d_total, next);
        return cudaSuccess;
    });
    cudaFreeAsync(next, s);
    return st;
}

mk_status mk_tc_static(mk_graph *g, uint64_t *h_triangles, void *stream)
{
    if (!g || !h_triangles)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&d, 8, s));
    MK_CUDA(cudaMemsetAsync(d, 0, 8, s));
    mk_status st = timed(g, "tc_static", s, 1, [&]() {
        k_tc_static<<<resident_grid(k_tc_static, 256), 256, 0, s>>>(g->v, g->v.P + 2, d);
        return cudaSuccess;
    });
    unsigned long long total = 0;
    if (st == MK_OK && (cudaMemcpyAsync(&total, d, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = MK_ERR_CUDA;
    cudaFreeAsync(d, s);
    *h_triangles = total;
    return st;
}

mk_status mk_tc_update(mk_graph *g_post, mk_graph *g_upd, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                       int deletion, int64_t *h_delta, void *stream)
{
    if (!g_post || !g_upd || !h_delta || g_post->v.V != g_upd->v.V || (n && (!d_src || !d_dst)))
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&d, 24, s));
    MK_CUDA(cudaMemsetAsync(d, 0, 24, s));
    mk_status st = mk_tc_count(g_post, g_post, d_src, d_dst, n, d + 0, stream);
    if (st == MK_OK)
        st = mk_tc_count(g_post, g_upd, d_src, d_dst, n, d + 1, stream);
    if (st == MK_OK)
        st = mk_tc_count(g_upd, g_upd, d_src, d_dst, n, d + 2, stream);
    unsigned long long S[3] = {0, 0, 0};
    if (st == MK_OK && (cudaMemcpyAsync(S, d, 24, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                        cudaStreamSynchronize(s) != cudaSuccess))
        st = MK_ERR_CUDA;
    cudaFreeAsync(d, s);
    if (st != MK_OK)
        return st;
    // S1 = 2 T1 + 4 T2 + 6 T3 and S2 = 2 T2 + 6 T3 (insertion) or S1 = 2 T1,
    // S2 = 2 T2 (deletion); S3 = 6 T3 in both
    const long long s1 = (long long)S[0], s2 = (long long)S[1], s3 = (long long)S[2];
    if (s1 % 2 || s2 % 2 || s3 % 6)
        return MK_ERR_INTERNAL;
    *h_delta = deletion ? -(s1 / 2 + s2 / 2 + s3 / 6) : (s1 / 2 - s2 / 2 + s3 / 6);
    return MK_OK;
}

} // extern "C"
