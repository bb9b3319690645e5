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
// CASes per slab instead of one union per edge on the same source root), and
// a warp walks four lists at a time.
//
// Static pass: every live edge of every list.  Incremental pass (insert-only
// epochs): only the entries written since the last commit, read with the
// UpdateIterator from each updated list's marker (the paper's
// ApplyUnionUpdate, which skips lanes before the first updated lane).
#include "mk_host.h"
#include "walk.cuh"

#include <algorithm>

using namespace mk;

namespace {

__device__ __forceinline__ uint32_t uf_find(uint32_t *p, uint32_t x)
{
    for (;;) {
        const uint32_t px = __ldcg(&p[x]);
        if (px == x)
            return x;
        const uint32_t ppx = __ldcg(&p[px]);
        if (ppx == px)
            return px; // px is the root: no third load
        p[x] = ppx;    // path halving: ppx is an ancestor of x
        x = ppx;
    }
}

// Parent loads.  The coherent form reads L2 (the point of coherence); the
// cached form may also hit a stale line in the SM's L1.  A stale parent is
// still a correct one from an earlier moment: parents only ever move to
// smaller ids of the same set (a hook replaces a root's self-link, path
// halving replaces a parent by an ancestor), and a vertex that is not a root
// never becomes one again.  So a find on cached loads returns a vertex that
// is, or was, the root of the element's set -- always a member of that set.
// Path halving may then store a parent older than the current one, which
// is still an ancestor in the same set.  The union below only acts on a
// found root through a CAS that succeeds while it is still a root, and
// retries on coherent loads.  The cached form
// keeps the roots that every find ends at (above all the giant component's
// vertex 0) in L1 instead of sending every find's last load to the same L2
// line.
template <bool kCached>
__device__ __forceinline__ uint32_t uf_load(const uint32_t *p, uint32_t x)
{
    return kCached ? p[x] : __ldcg(&p[x]);
}

// Two finds in lockstep, so that their dependent loads overlap; kNil
// entries are left alone.  Parents strictly decrease along every path
// (p[x] < x except at roots), so both walks end.
template <bool kCached>
__device__ __forceinline__ void uf_find2(uint32_t *p, uint32_t &x, uint32_t &y)
{
    bool dx = x == kNil, dy = y == kNil;
    while (!(dx && dy)) {
        uint32_t px = x, py = y;
        if (!dx)
            px = uf_load<kCached>(p, x);
        if (!dy)
            py = uf_load<kCached>(p, y);
        dx = dx || px == x;
        dy = dy || py == y;
        uint32_t ppx = px, ppy = py;
        if (!dx)
            ppx = uf_load<kCached>(p, px);
        if (!dy)
            ppy = uf_load<kCached>(p, py);
        if (!dx) {
            if (ppx == px) {
                x = px;
                dx = true;
            } else {
                p[x] = ppx; // path halving: ppx is an ancestor of x
                x = ppx;
            }
        }
        if (!dy) {
            if (ppy == py) {
                y = py;
                dy = true;
            } else {
                p[y] = ppy;
                y = ppy;
            }
        }
    }
}

// Union of the sets of up to 16 elements held by one 8-lane group, two per
// lane: all roots are found in parallel, the group's smallest root m is the
// anchor, and every other root r is hooked under it with one CAS on p[r]
// from r to m.  The CAS succeeds only while r is still a root; m need not be
// one any more, because any vertex with a smaller id lies in another tree
// (ids never increase towards a root), so the hook joins the two sets and
// keeps parents decreasing.  An element whose CAS loses (its root was
// hooked by another warp meanwhile) retries with fresh roots of itself and
// of the anchor, hooking the larger under the smaller.  Returns false if the
// retry bound was hit.  Must be called by the full warp.
__device__ __forceinline__ bool group_union2(uint32_t *p, uint32_t e0, bool a0, uint32_t e1, bool a1,
                                             uint32_t limit)
{
    uint32_t r0 = a0 ? e0 : kNil;
    uint32_t r1 = a1 ? e1 : kNil;
    uf_find2<true>(p, r0, r1);
    uint32_t m = min(r0, r1);
    m = min(m, __shfl_xor_sync(kFull, m, 4));
    m = min(m, __shfl_xor_sync(kFull, m, 2));
    m = min(m, __shfl_xor_sync(kFull, m, 1));
    bool p0 = a0 && r0 != m, p1 = a1 && r1 != m;
    // first attempt with the roots just found (r > m for every pending r)
    if (p0 && atomicCAS(&p[r0], r0, m) == r0)
        p0 = false;
    if (p1) {
        if (a0 && r1 == r0)
            p1 = p0; // the same root: decided by the CAS above
        else if (atomicCAS(&p[r1], r1, m) == r1)
            p1 = false;
    }
    for (uint32_t it = 0; it < limit; ++it) {
        if (!__any_sync(kFull, p0 || p1))
            return true;
        uint32_t a = (p0 || p1) ? m : kNil, unused = kNil;
        uf_find2<false>(p, a, unused);
        uint32_t x0 = p0 ? r0 : kNil, x1 = p1 ? r1 : kNil;
        uf_find2<false>(p, x0, x1);
        if (p0) {
            r0 = x0;
            if (r0 == a || atomicCAS(&p[max(r0, a)], max(r0, a), min(r0, a)) == max(r0, a))
                p0 = false;
        }
        if (p1) {
            r1 = x1;
            if (r1 == a || atomicCAS(&p[max(r1, a)], max(r1, a), min(r1, a)) == max(r1, a))
                p1 = false;
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

// Unites src with every live destination of the selected lists.  Each warp
// owns 32 consecutive lists and walks the selected ones four at a time, one
// per 8-lane group with 16-byte loads (pairs 2*sub and 2*sub+1 per lane); the
// unused slot of lane 7 (slab lane 30) carries the list's source, so each
// slab's source and destinations are united in one group_union2.
// all_lists: every list from its head; otherwise only updated lists from
// their UpdateIterator start.
__global__ void __launch_bounds__(256, 6) k_uf_hook(GView g, uint32_t *p, int all_lists, uint32_t max_hops, int *failed)
{
    const uint32_t lane = lane_id(), gi = lane >> 3, sub = lane & 7u, gbase = lane & ~7u;
    const uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull;
    if (base >= g.H)
        return;
    const uint64_t l = base + lane;
    const bool todo = l < g.H && (all_lists || g.lupd[l]);
    // each lane fetches its own list's source and walk start up front
    uint32_t my_src = 0, my_first = 0, my_start = kNil;
    if (todo) {
        my_src = g.list_src[l];
        my_start = all_lists ? (uint32_t)l : update_begin(g, (uint32_t)l, &my_first);
    }
    const uint32_t q = __ballot_sync(kFull, todo);
    unsigned long long slabs = 0, edges = 0;
    for (uint32_t pass = 0; pass * 4 < (uint32_t)__popc(q); ++pass) {
        const uint32_t owner = group_item(q, pass, gi);
        const bool has = owner < 32;
        const uint32_t src = __shfl_sync(kFull, my_src, owner & 31);
        uint32_t first_lane = __shfl_sync(kFull, my_first, owner & 31);
        const uint32_t start0 = __shfl_sync(kFull, my_start, owner & 31);
        uint32_t slab = has ? start0 : kNil;
        bool active = slab != kNil;
        for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
            uint4 x = make_uint4(kEmptyKey, kFull, kFull, kFull);
            if (active)
                x = __ldcg(reinterpret_cast<const uint4 *>(slab_ptr(g, slab) + sub * 4));
            slabs += __popc(__ballot_sync(kFull, active && sub == 0));
            const bool last = sub == 7u;
            const bool a0 = active && x.x < kTombKey && 4 * sub >= first_lane;
            const bool a1 = last ? active : (active && x.z < kTombKey && 4 * sub + 2 >= first_lane);
            edges += __popc(__ballot_sync(kFull, a0)) + __popc(__ballot_sync(kFull, a1 && !last));
            if (!group_union2(p, x.x, a0, last ? src : x.z, a1, 1u << 20) && lane == 0)
                *failed = 1;
            const uint32_t nxt = __shfl_sync(kFull, x.w, gbase + 7);
            if (active) {
                if (nxt == kNil || hop + 1 >= max_hops)
                    active = false;
                else
                    slab = nxt;
            }
            first_lane = 0;
        }
    }
    count_add(g.st, all_lists ? kCtrWccSlabs : kCtrWccUpdSlabs, slabs);
    count_add(g.st, all_lists ? kCtrWccEdges : kCtrWccUpdEdges, edges);
}

// Static pass as a streaming scan over every slab in use (heads and linked
// pool slabs, found through the per-slab owner array) instead of chain
// walks.  A warp takes 32 consecutive slabs at a time: one coalesced load of
// their owners, the slabs in use compacted in shared memory, then four slabs
// per step, one per 8-lane group (16-byte loads), with the next step's slabs
// loaded before this step's finds so that the slab stream overlaps the
// union-find latency.  Each slab's owner and its live destinations are
// united in one group_union2, exactly as in the list walk.
__global__ void __launch_bounds__(256, 6) k_uf_hook_slabs(GView g, uint32_t *p, int *failed)
{
    __shared__ uint8_t comp[8][32];
    const uint32_t lane = lane_id(), gi = lane >> 3, sub = lane & 7u, w = threadIdx.x >> 5;
    const uint64_t total = (uint64_t)g.H + g.P;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint4 none = make_uint4(kEmptyKey, kFull, kFull, kFull);
    unsigned long long slabs = 0, edges = 0;
    for (uint64_t c = warp0 * 32; c < total; c += nwarps * 32) {
        const uint32_t own_l = c + lane < total ? __ldcg(&g.owner[c + lane]) : kNil;
        const uint32_t live = __ballot_sync(kFull, own_l != kNil);
        const uint32_t n = __popc(live);
        if (own_l != kNil)
            comp[w][__popc(live & ((1u << lane) - 1))] = (uint8_t)lane;
        __syncwarp();
        uint32_t it = gi < n ? comp[w][gi] : 32u;
        uint4 x = none;
        if (it < 32)
            x = __ldcg(reinterpret_cast<const uint4 *>(slab_ptr(g, (uint32_t)(c + it)) + sub * 4));
        for (uint32_t k = gi; k - gi < n; k += 4) {
            // prefetch the next step's slab
            const uint32_t nit = k + 4 < n ? comp[w][k + 4] : 32u;
            uint4 nx = none;
            if (nit < 32)
                nx = __ldcg(reinterpret_cast<const uint4 *>(slab_ptr(g, (uint32_t)(c + nit)) + sub * 4));
            const bool active = it < 32;
            const uint32_t own = __shfl_sync(kFull, own_l, it & 31);
            slabs += __popc(__ballot_sync(kFull, active && sub == 0));
            const bool last = sub == 7u;
            const bool a0 = active && x.x < kTombKey;
            const bool a1 = last ? active : (active && x.z < kTombKey);
            edges += __popc(__ballot_sync(kFull, a0)) + __popc(__ballot_sync(kFull, a1 && !last));
            if (!group_union2(p, x.x, a0, last ? own : x.z, a1, 1u << 20) && lane == 0)
                *failed = 1;
            x = nx;
            it = nit;
        }
        __syncwarp();
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
    if (incremental) {
        MK_TRY(timed(g, "wcc_hook_updated", s, 1, [&]() {
            k_uf_hook<<<grid_for((uint64_t)H, 256), 256, 0, s>>>(g->v, c->uf, 0, max_hops, failed);
            return cudaSuccess;
        }));
    } else {
        MK_TRY(timed(g, "wcc_hook_all", s, 1, [&]() {
            const uint64_t warps = ((uint64_t)H + g->v.P + 31) / 32;
            const uint32_t grid = (uint32_t)std::min<uint64_t>(grid_for(warps * 32, 256), (uint64_t)num_sms() * 16);
            k_uf_hook_slabs<<<grid, 256, 0, s>>>(g->v, c->uf, failed);
            return cudaSuccess;
        }));
    }
    MK_TRY(timed(g, "wcc_compress", s, 2, [&]() {
        k_uf_compress<<<grid_for(V, 256), 256, 0, s>>>(c->uf, V, d_label);
        k_uf_failed<<<1, 1, 0, s>>>(failed, g->d_state);
        return cudaSuccess;
    }));
    c->epoch = g->epoch;
    c->seq = g->change_seq;
    return MK_OK;
}
