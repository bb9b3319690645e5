// Static and incremental weakly connected components (paper, Sec.
// "Incremental WCC" and Sec. "Auxiliary Data Structures", Union-Find).
//
// Union-Async: to unite sets, find their roots and hook the larger root under
// the smaller with one CAS, retrying with fresh roots when the CAS loses.
// Parents therefore never exceed their child's id, the root of every tree is
// its smallest vertex, and after full path compression each label is the
// smallest vertex id of its component.  Finds use path halving.  A warp unites
// a whole slab at once: the source and the slab's live destinations are
// hooked under the smallest of their roots (one parallel round of finds and
// CASes per slab instead of one union per edge on the same source root).
//
// Static pass: every live edge of every list.  Incremental pass (insert-only
// epochs): only the entries written since the last commit, read with the
// UpdateIterator from each updated list's marker (the paper's
// ApplyUnionUpdate, which skips lanes before the first updated lane).
#include "mk_host.h"
#include "walk.cuh"

using namespace mk;

namespace {

__device__ __forceinline__ uint32_t uf_find(uint32_t *p, uint32_t x)
{
    for (;;) {
        const uint32_t px = __ldcg(&p[x]);
        if (px == x)
            return x;
        const uint32_t ppx = __ldcg(&p[px]);
        if (ppx != px)
            p[x] = ppx; // path halving: ppx is an ancestor of x
        x = ppx;
    }
}

// Warp-wide union of the sets of every active lane's element: all roots are
// found in parallel, the warp's smallest root m is the anchor, and every
// other root is hooked under it with one CAS on its parent (m is smaller, so
// parents keep decreasing).  A lane whose CAS loses (its root was hooked by
// another warp meanwhile) retries with fresh roots of its element and of the
// anchor, hooking the larger under the smaller.  Returns false if the retry
// bound was hit.  Must be called by the full warp.
__device__ __forceinline__ bool warp_union(uint32_t *p, uint32_t e, bool active, uint32_t limit)
{
    uint32_t r = active ? uf_find(p, e) : kNil;
    uint32_t m = r;
#pragma unroll
    for (uint32_t o = 16; o; o >>= 1)
        m = min(m, __shfl_xor_sync(kFull, m, o));
    bool pending = active && r != m;
    for (uint32_t it = 0; it < limit; ++it) {
        if (!__any_sync(kFull, pending))
            return true;
        if (pending) {
            const uint32_t a = uf_find(p, m);
            r = uf_find(p, r);
            if (r == a) {
                pending = false;
            } else {
                const uint32_t hi = max(r, a), lo = min(r, a);
                if (atomicCAS(&p[hi], hi, lo) == hi)
                    pending = false;
            }
        }
    }
    return false;
}

} // namespace

__global__ void k_uf_init(uint32_t *p, uint32_t V)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V)
        p[v] = v;
}

// Unites src with every live destination of the selected lists; warp per 32
// lists.  all_lists: every list from its head; otherwise only updated lists
// from their UpdateIterator start.
__global__ void __launch_bounds__(256) k_uf_hook(GView g, uint32_t *p, int all_lists, uint32_t max_hops, int *failed)
{
    const uint32_t lane = lane_id();
    const uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull;
    if (base >= g.H)
        return;
    const uint64_t l = base + lane;
    bool todo = l < g.H && (all_lists || g.lupd[l]);
    unsigned long long slabs = 0, edges = 0;
    uint32_t q;
    while ((q = __ballot_sync(kFull, todo)) != 0) {
        const uint32_t leader = __ffs(q) - 1;
        if (lane == leader)
            todo = false;
        const uint32_t L = (uint32_t)(base + leader);
        const uint32_t src = g.list_src[L];
        uint32_t first_lane = 0, start = L;
        if (!all_lists)
            start = update_begin(g, L, &first_lane);
        // lane 30 (no key) carries the list's source into each slab's union
        slabs += walk_list(g, start, first_lane, max_hops, [&](uint32_t y, uint32_t, bool live) {
            edges += __popc(__ballot_sync(kFull, live));
            const bool act = live || lane == 30;
            if (!warp_union(p, lane == 30 ? src : y, act, 1u << 20) && lane == 0)
                *failed = 1;
        });
    }
    count_add(g.st, kCtrWccSlabs, slabs);
    count_add(g.st, kCtrWccEdges, edges);
}

__global__ void k_uf_compress(uint32_t *p, uint32_t V, uint32_t *label)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V)
        return;
    const uint32_t r = uf_find(p, v);
    p[v] = r;
    if (label)
        label[v] = r;
}

__global__ void k_uf_failed(const int *failed, DevState *st)
{
    if (*failed)
        set_status(st, kErrTimeout);
}

extern "C" mk_status mk_incr_wcc(mk_graph *g, uint32_t *d_label, void *stream)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    const uint32_t V = g->v.V, H = g->v.H;
    auto key = std::make_pair((int)kWcc, 0u);
    Consumer *c = nullptr;
    auto it = g->consumers.find(key);
    if (it == g->consumers.end()) {
        c = new Consumer;
        c->kind = kWcc;
        mk_status st = device_alloc(g, (void **)&c->uf, (size_t)V * 4);
        if (st == MK_OK)
            st = device_alloc(g, (void **)&c->counters, 64);
        if (st != MK_OK) {
            device_free(g, c->uf, (size_t)V * 4);
            device_free(g, c->counters, 64);
            delete c;
            return st;
        }
        g->consumers[key] = c;
    } else {
        c = it->second;
    }
    // the paper has no decremental WCC: an epoch with deletions recomputes
    const bool incremental = c->epoch == g->epoch && !g->epoch_has_deletes;
    const uint32_t max_hops = g->v.P + 2;
    int *failed = (int *)c->counters;
    MK_CUDA(cudaMemsetAsync(c->counters, 0, 64, s));
    if (!incremental) {
        MK_TRY(timed(g, "wcc_init", s, 1, [&]() {
            k_uf_init<<<grid_for(V, 256), 256, 0, s>>>(c->uf, V);
            return cudaSuccess;
        }));
    }
    MK_TRY(timed(g, incremental ? "wcc_hook_updated" : "wcc_hook_all", s, 1, [&]() {
        k_uf_hook<<<grid_for((uint64_t)H, 256), 256, 0, s>>>(g->v, c->uf, incremental ? 0 : 1, max_hops, failed);
        return cudaSuccess;
    }));
    MK_TRY(timed(g, "wcc_compress", s, 2, [&]() {
        k_uf_compress<<<grid_for(V, 256), 256, 0, s>>>(c->uf, V, d_label);
        k_uf_failed<<<1, 1, 0, s>>>(failed, g->d_state);
        return cudaSuccess;
    }));
    c->epoch = g->epoch;
    c->seq = g->change_seq;
    return MK_OK;
}
