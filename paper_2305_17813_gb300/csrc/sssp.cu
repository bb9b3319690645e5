// Incremental / decremental single-source shortest paths and BFS (paper,
// Algorithm "SSSP - Incremental / Decremental" and Sec. "Dynamic Single
// Source Shortest Path and Breadth First Search").
//
// Every vertex holds a 64-bit tree node <distance:32, parent:32>, updated
// with one 64-bit atomicMin so both halves change together (footnote on the
// tree-node packing); at the fixpoint the parent is the smallest-id tight
// predecessor.  Frontiers hold slab LISTS rather than edges or vertices: when
// a vertex improves, all its lists are enqueued (once per round, deduplicated
// by a per-vertex round stamp), and one warp then relaxes every live edge of
// one list.  Lists are short and evenly sized by the bucket rule, so the work
// is balanced even for high-degree vertices (the motivation of the paper's
// BucketIterator, Algorithm "Iteration Scheme 2").
//
// Decremental prologue: deleted tree edges (parent(v) = u) invalidate v; the
// invalidation then spreads down the tree through the children of every
// invalidated vertex (a top-down traversal of the affected subtrees instead
// of the paper's per-vertex walk up to the source, so the cost follows the
// invalidated region); then every edge from a valid vertex into an invalid
// one is relaxed.  Incremental prologue: the edges inserted since the last
// commit, read with the UpdateIterator, are relaxed.  Common epilogue: rounds
// until no distance improves.
#include "mk_host.h"
#include "walk.cuh"

#include <algorithm>

using namespace mk;

namespace {

constexpr uint32_t kInf32 = 0xFFFFFFFFu;

__device__ __forceinline__ uint32_t node_dist(unsigned long long d) { return (uint32_t)(d >> 32); }
__device__ __forceinline__ uint32_t node_parent(unsigned long long d) { return (uint32_t)d; }

// Relaxes edge (x, y, w) given x's distance dx; returns true if D[y] dropped.
__device__ __forceinline__ bool relax(unsigned long long *D, uint32_t x, uint32_t dx, uint32_t y, uint32_t w)
{
    const unsigned long long nd = (unsigned long long)dx + w;
    if (nd >= kInf32)
        return false;
    const unsigned long long cand = (nd << 32) | x;
    if (cand >= __ldcg(&D[y]))
        return false;
    return cand < atomicMin(&D[y], cand);
}

// Vertex-level dedup for one round: true for the first lane that stamps y.
__device__ __forceinline__ bool first_this_round(uint32_t *stamp, uint32_t y, uint32_t round)
{
    return atomicExch(&stamp[y], round) != round;
}

} // namespace

__global__ void k_sssp_init(unsigned long long *D, uint32_t V, uint32_t source, uint32_t *front, uint32_t *count,
                            const uint2 *vinfo)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V)
        D[v] = v == source ? ((unsigned long long)0 << 32 | source) : kInfNode;
    if (v == 0) {
        const uint2 vi = vinfo[source];
        for (uint32_t b = 0; b < vi.y; ++b)
            front[b] = vi.x + b;
        *count = vi.y;
    }
}

// One round of the epilogue: warp per 32 frontier lists.
__global__ void __launch_bounds__(256) k_relax_round(GView g, unsigned long long *D, const uint32_t *__restrict__ F,
                                                     uint32_t n, uint32_t *Fn, uint32_t *cnt, uint32_t cap,
                                                     uint32_t *stamp, uint32_t round, int unit, uint32_t max_hops,
                                                     int *overflow)
{
    const uint32_t lane = lane_id();
    const uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull;
    if (base >= n)
        return;
    const uint64_t i = base + lane;
    bool todo = i < n;
    const uint32_t mine = todo ? F[i] : 0;
    unsigned long long lists = 0, slabs = 0, edges = 0, improved = 0;
    uint32_t q;
    while ((q = __ballot_sync(kFull, todo)) != 0) {
        const uint32_t leader = __ffs(q) - 1;
        if (lane == leader)
            todo = false;
        const uint32_t L = __shfl_sync(kFull, mine, leader);
        const uint32_t x = g.list_src[L];
        const uint32_t dx = __shfl_sync(kFull, node_dist(__ldcg(&D[x])), 0);
        ++lists;
        if (dx == kInf32)
            continue;
        slabs += walk_list(g, L, 0, max_hops, [&](uint32_t y, uint32_t w, bool live) {
            edges += __popc(__ballot_sync(kFull, live));
            bool up = live && relax(D, x, dx, y, unit ? 1u : w);
            up = up && first_this_round(stamp, y, round);
            improved += __popc(__ballot_sync(kFull, up));
            enqueue_lists(g, y, up, Fn, cnt, cap, overflow);
        });
    }
    count_add(g.st, kCtrRelaxLists, lists);
    count_add(g.st, kCtrRelaxSlabs, slabs);
    count_add(g.st, kCtrRelaxEdges, edges);
    count_add(g.st, kCtrRelaxImproved, improved);
}

// Decremental seeds: a deleted edge (u, v) that is v's tree edge invalidates v.
__global__ void k_invalidate(const unsigned long long *dlog, const DevState *st, unsigned long long *D, uint32_t source,
                             GView g, uint32_t *Fn, uint32_t *cnt, uint32_t cap, int *overflow, uint32_t *total,
                             uint32_t *inv)
{
    const uint32_t n = st->dlog_count;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    const uint64_t lim = ((uint64_t)n + 31) & ~31ull;
    if ((uint64_t)(i & ~31u) >= lim)
        return;
    bool hit = false;
    uint32_t v = 0;
    if (i < n) {
        const unsigned long long e = dlog[i];
        const uint32_t u = (uint32_t)(e >> 32);
        v = (uint32_t)e;
        const unsigned long long dv = __ldcg(&D[v]);
        if (v != source && dv != kInfNode && node_parent(dv) == u)
            hit = atomicCAS(&D[v], dv, kInfNode) == dv;
    }
    if (hit) {
        atomicAdd(total, 1u);
        atomicOr(&inv[v >> 5], 1u << (v & 31));
    }
    enqueue_lists(g, v, hit, Fn, cnt, cap, overflow);
}

// Spreads invalidation to the tree children of invalidated vertices.
__global__ void __launch_bounds__(256) k_invalidate_round(GView g, unsigned long long *D, const uint32_t *__restrict__ F,
                                                          uint32_t n, uint32_t *Fn, uint32_t *cnt, uint32_t cap,
                                                          uint32_t source, uint32_t max_hops, int *overflow,
                                                          uint32_t *total, uint32_t *inv)
{
    const uint32_t lane = lane_id();
    const uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull;
    if (base >= n)
        return;
    const uint64_t i = base + lane;
    bool todo = i < n;
    const uint32_t mine = todo ? F[i] : 0;
    unsigned long long slabs = 0;
    uint32_t q;
    while ((q = __ballot_sync(kFull, todo)) != 0) {
        const uint32_t leader = __ffs(q) - 1;
        if (lane == leader)
            todo = false;
        const uint32_t L = __shfl_sync(kFull, mine, leader);
        const uint32_t x = g.list_src[L];
        slabs += walk_list(g, L, 0, max_hops, [&](uint32_t y, uint32_t, bool live) {
            bool hit = false;
            if (live && y != source) {
                const unsigned long long dy = __ldcg(&D[y]);
                if (dy != kInfNode && node_parent(dy) == x)
                    hit = atomicCAS(&D[y], dy, kInfNode) == dy;
            }
            if (hit) {
                atomicAdd(total, 1u);
                atomicOr(&inv[y >> 5], 1u << (y & 31));
            }
            enqueue_lists(g, y, hit, Fn, cnt, cap, overflow);
        });
    }
    count_add(g.st, kCtrInvalidSlabs, slabs);
}

// After invalidation: relax every edge out of a valid vertex into a vertex
// invalidated by this call (warp per 32 lists over all lists).  The target
// test reads the invalidation bitmap, which stays fixed during the pass, so
// every such edge is relaxed even after another in-neighbour has already
// given its target a finite distance.
__global__ void __launch_bounds__(256) k_relax_into_invalid(GView g, unsigned long long *D, uint32_t *Fn, uint32_t *cnt,
                                                            uint32_t cap, uint32_t *stamp, uint32_t round, int unit,
                                                            uint32_t max_hops, int *overflow, const uint32_t *inv)
{
    const uint32_t lane = lane_id();
    const uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull;
    if (base >= g.H)
        return;
    const uint64_t l = base + lane;
    bool todo = false;
    uint32_t x = 0;
    if (l < g.H) {
        x = g.list_src[l];
        todo = node_dist(__ldcg(&D[x])) != kInf32;
    }
    unsigned long long lists = 0, slabs = 0, edges = 0, improved = 0;
    uint32_t q;
    while ((q = __ballot_sync(kFull, todo)) != 0) {
        const uint32_t leader = __ffs(q) - 1;
        if (lane == leader)
            todo = false;
        const uint32_t L = (uint32_t)(base + leader);
        const uint32_t src = __shfl_sync(kFull, x, leader);
        const uint32_t dx = __shfl_sync(kFull, node_dist(__ldcg(&D[src])), 0);
        ++lists;
        slabs += walk_list(g, L, 0, max_hops, [&](uint32_t y, uint32_t w, bool live) {
            edges += __popc(__ballot_sync(kFull, live));
            const bool target = live && ((inv[y >> 5] >> (y & 31)) & 1u);
            bool up = target && relax(D, src, dx, y, unit ? 1u : w);
            up = up && first_this_round(stamp, y, round);
            improved += __popc(__ballot_sync(kFull, up));
            enqueue_lists(g, y, up, Fn, cnt, cap, overflow);
        });
    }
    count_add(g.st, kCtrRelaxLists, lists);
    count_add(g.st, kCtrRelaxSlabs, slabs);
    count_add(g.st, kCtrRelaxEdges, edges);
    count_add(g.st, kCtrRelaxImproved, improved);
}

// Incremental seeds: relax the entries inserted since the last commit
// (UpdateIterator over the lists flagged as updated).
__global__ void __launch_bounds__(256) k_relax_updated(GView g, unsigned long long *D, uint32_t *Fn, uint32_t *cnt,
                                                       uint32_t cap, uint32_t *stamp, uint32_t round, int unit,
                                                       uint32_t max_hops, int *overflow)
{
    const uint32_t lane = lane_id();
    const uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull;
    if (base >= g.H)
        return;
    const uint64_t l = base + lane;
    bool todo = l < g.H && g.lupd[l];
    unsigned long long lists = 0, slabs = 0, edges = 0, improved = 0;
    uint32_t q;
    while ((q = __ballot_sync(kFull, todo)) != 0) {
        const uint32_t leader = __ffs(q) - 1;
        if (lane == leader)
            todo = false;
        const uint32_t L = (uint32_t)(base + leader);
        const uint32_t src = g.list_src[L];
        const uint32_t dx = __shfl_sync(kFull, node_dist(__ldcg(&D[src])), 0);
        if (dx == kInf32)
            continue;
        uint32_t first_lane = 0;
        const uint32_t start = update_begin(g, L, &first_lane);
        ++lists;
        slabs += walk_list(g, start, first_lane, max_hops, [&](uint32_t y, uint32_t w, bool live) {
            edges += __popc(__ballot_sync(kFull, live));
            bool up = live && relax(D, src, dx, y, unit ? 1u : w);
            up = up && first_this_round(stamp, y, round);
            improved += __popc(__ballot_sync(kFull, up));
            enqueue_lists(g, y, up, Fn, cnt, cap, overflow);
        });
    }
    count_add(g.st, kCtrRelaxLists, lists);
    count_add(g.st, kCtrRelaxSlabs, slabs);
    count_add(g.st, kCtrRelaxEdges, edges);
    count_add(g.st, kCtrRelaxImproved, improved);
}

__global__ void k_unpack(const unsigned long long *D, uint32_t V, uint32_t *dist, uint32_t *parent)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V)
        return;
    const unsigned long long d = D[v];
    if (dist)
        dist[v] = node_dist(d);
    if (parent)
        parent[v] = node_parent(d);
}

__global__ void k_flag_overflow(const int *overflow, DevState *st)
{
    if (*overflow)
        set_status(st, kErrTimeout);
}

// ---------------------------------------------------------------- host side

namespace {

// counters layout (device words)
enum { kCntA = 0, kCntB = 1, kInvTotal = 2, kOverflow = 3 };

mk_status get_consumer(mk_graph *g, int kind, uint32_t source, Consumer **out)
{
    auto key = std::make_pair(kind, source);
    auto it = g->consumers.find(key);
    if (it != g->consumers.end()) {
        *out = it->second;
        return MK_OK;
    }
    Consumer *c = new Consumer;
    c->kind = kind;
    c->source = source;
    const size_t V = g->v.V, H = g->v.H;
    mk_status st = device_alloc(g, (void **)&c->D, V * 8);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->front[0], H * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->front[1], H * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->stamp, V * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->inv, (V + 31) / 32 * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->counters, 64);
    if (st == MK_OK && (cudaMemset(c->stamp, 0, V * 4) != cudaSuccess || cudaMemset(c->counters, 0, 64) != cudaSuccess))
        st = MK_ERR_CUDA;
    if (st != MK_OK) {
        device_free(g, c->D, V * 8);
        device_free(g, c->front[0], H * 4);
        device_free(g, c->front[1], H * 4);
        device_free(g, c->stamp, V * 4);
        device_free(g, c->inv, (V + 31) / 32 * 4);
        device_free(g, c->counters, 64);
        delete c;
        return st;
    }
    g->consumers[key] = c;
    *out = c;
    return MK_OK;
}

mk_status read_word(mk_graph *g, const uint32_t *d_word, uint32_t *out, cudaStream_t s)
{
    MK_CUDA(cudaMemcpyAsync(g->h_pinned, d_word, 4, cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    *out = g->h_pinned[0];
    return MK_OK;
}

// Runs rounds of `kernel_launch(cur, n, next)` until the frontier is empty.
// The frontier in front[*cur] holds `n` lists; returns with n == 0.
template <typename Launch>
mk_status run_rounds(mk_graph *g, Consumer *c, int *cur, uint32_t n, cudaStream_t s, const char *name,
                     Launch &&launch)
{
    const uint64_t limit = (uint64_t)g->v.V + 2;
    for (uint64_t r = 0; n != 0; ++r) {
        if (r > limit) {
            mk_status st = MK_ERR_TIMEOUT;
            return st;
        }
        const int nxt = *cur ^ 1;
        MK_CUDA(cudaMemsetAsync(c->counters + nxt, 0, 4, s));
        MK_TRY(timed(g, name, s, 1, [&]() { return launch(*cur, n, nxt); }));
        MK_TRY(read_word(g, c->counters + nxt, &n, s));
        *cur = nxt;
    }
    return MK_OK;
}

mk_status run_sssp(mk_graph *g, int kind, uint32_t source, uint32_t *d_dist, uint32_t *d_parent, cudaStream_t s)
{
    if (!g || source >= g->v.V)
        return MK_ERR_INVALID_ARG;
    g->last_stream = s;
    Consumer *c = nullptr;
    MK_TRY(get_consumer(g, kind, source, &c));
    const int unit = kind == kBfs ? 1 : 0;
    const uint32_t V = g->v.V, H = g->v.H, cap = H;
    const uint32_t max_hops = g->v.P + 2;
    int *overflow = (int *)(c->counters + kOverflow);
    int cur = 0;
    uint32_t n = 0;
    const bool incremental = c->epoch == g->epoch;
    MK_CUDA(cudaMemsetAsync(c->counters, 0, 64, s));
    auto relax_launch = [&](int a, uint32_t na, int b) {
        k_relax_round<<<grid_for((uint64_t)na, 256), 256, 0, s>>>(g->v, c->D, c->front[a], na, c->front[b],
                                                                  c->counters + b, cap, c->stamp, ++c->round, unit,
                                                                  max_hops, overflow);
        return cudaSuccess;
    };
    if (!incremental) {
        MK_TRY(timed(g, "sssp_init", s, 1, [&]() {
            k_sssp_init<<<grid_for(V, 256), 256, 0, s>>>(c->D, V, source, c->front[0], c->counters + 0, g->v.vinfo);
            return cudaSuccess;
        }));
        MK_TRY(read_word(g, c->counters + 0, &n, s));
    } else {
        // both prologues seed the first epilogue frontier under one round stamp
        const uint32_t seeds_round = ++c->round;
        if (g->epoch_has_deletes) {
            // decremental prologue: invalidate, spread down the tree
            MK_CUDA(cudaMemsetAsync(c->counters, 0, 16, s));
            MK_CUDA(cudaMemsetAsync(c->inv, 0, (size_t)(V + 31) / 32 * 4, s));
            MK_TRY(timed(g, "sssp_invalidate", s, 1, [&]() {
                k_invalidate<<<grid_for(std::max<uint64_t>(g->dlog_bound, 1), 256), 256, 0, s>>>(
                    g->d_dlog, g->d_state, c->D, source, g->v, c->front[0], c->counters + 0, cap, overflow,
                    c->counters + kInvTotal, c->inv);
                return cudaSuccess;
            }));
            MK_TRY(read_word(g, c->counters + 0, &n, s));
            MK_TRY(run_rounds(g, c, &cur, n, s, "sssp_invalidate_round", [&](int a, uint32_t na, int b) {
                k_invalidate_round<<<grid_for((uint64_t)na, 256), 256, 0, s>>>(
                    g->v, c->D, c->front[a], na, c->front[b], c->counters + b, cap, source, max_hops, overflow,
                    c->counters + kInvTotal, c->inv);
                return cudaSuccess;
            }));
            uint32_t invalidated = 0;
            MK_TRY(read_word(g, c->counters + kInvTotal, &invalidated, s));
            cur = 0;
            MK_CUDA(cudaMemsetAsync(c->counters, 0, 8, s));
            if (invalidated) {
                const uint32_t round = seeds_round;
                MK_TRY(timed(g, "sssp_relax_into_invalid", s, 1, [&]() {
                    k_relax_into_invalid<<<grid_for((uint64_t)H, 256), 256, 0, s>>>(
                        g->v, c->D, c->front[0], c->counters + 0, cap, c->stamp, round, unit, max_hops, overflow,
                        c->inv);
                    return cudaSuccess;
                }));
            }
        } else {
            MK_CUDA(cudaMemsetAsync(c->counters, 0, 8, s));
        }
        // incremental prologue: edges inserted since the last commit
        const uint32_t round = seeds_round;
        MK_TRY(timed(g, "sssp_relax_updated", s, 1, [&]() {
            k_relax_updated<<<grid_for((uint64_t)H, 256), 256, 0, s>>>(g->v, c->D, c->front[0], c->counters + 0, cap,
                                                                       c->stamp, round, unit, max_hops, overflow);
            return cudaSuccess;
        }));
        MK_TRY(read_word(g, c->counters + 0, &n, s));
    }
    // common epilogue
    MK_TRY(run_rounds(g, c, &cur, n, s, "sssp_round", relax_launch));
    MK_TRY(timed(g, "sssp_unpack", s, 2, [&]() {
        k_flag_overflow<<<1, 1, 0, s>>>(overflow, g->d_state);
        if (d_dist || d_parent)
            k_unpack<<<grid_for(V, 256), 256, 0, s>>>(c->D, V, d_dist, d_parent);
        return cudaSuccess;
    }));
    c->epoch = g->epoch;
    c->seq = g->change_seq;
    return MK_OK;
}

} // namespace

extern "C" {

mk_status mk_incr_sssp(mk_graph *g, uint32_t source, uint32_t *d_dist, uint32_t *d_parent, void *stream)
{
    return run_sssp(g, kSssp, source, d_dist, d_parent, (cudaStream_t)stream);
}

mk_status mk_incr_bfs(mk_graph *g, uint32_t source, uint32_t *d_dist, uint32_t *d_parent, void *stream)
{
    return run_sssp(g, kBfs, source, d_dist, d_parent, (cudaStream_t)stream);
}

} // extern "C"
