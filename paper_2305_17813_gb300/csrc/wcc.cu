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
// a warp walks eight lists at a time (incremental pass) or eight slabs (static
// pass).
//
// Static pass: every live edge of every list.  Incremental pass (insert-only
// epochs): only the entries written since the last commit, read with the
// UpdateIterator from each updated list's marker (the paper's
// ApplyUnionUpdate, which skips lanes before the first updated lane).
#include "mk_host.h"
#include "uf.cuh"
#include "walk.cuh"

#include <algorithm>

using namespace mk;

namespace {

__device__ __forceinline__ uint32_t uf_find(uint32_t *p, uint32_t x)
{
    for (;;) {
        const uint32_t px = __ldcg(&p[x]);
        if (px == x || px == 0) // vertex 0 is always a root
            return px;
        const uint32_t ppx = __ldcg(&p[px]);
        if (ppx == px)
            return px; // px is the root: no third load
        p[x] = ppx;    // path halving: ppx is an ancestor of x
        x = ppx;
    }
}


} // namespace

__global__ void k_uf_init(uint32_t *p, uint32_t V)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V)
        p[v] = v;
}

// Incremental pass: unites the source of every list in the updated-list log
// with the destinations inserted since the last commit, read with the
// UpdateIterator from the list's marker (the marker slab's lanes before the
// marker lane are skipped; a full marker slab is skipped entirely).  Every
// 4-lane group of every warp takes one list at a time (group index + k *
// groups in the grid; eight lists per warp) and walks it with two 16-byte
// loads per lane (pairs 4*s4 .. 4*s4+3); the unused slot of lane 3 (slab
// lane 30) carries the list's source, so each slab's source and
// destinations are united in one group_union.  The next list's log entry,
// source and marker are loaded a step ahead.
__global__ void __launch_bounds__(256, 5) k_uf_hook(GView g, uint32_t *p, uint32_t max_hops, int *failed)
{
    const uint32_t lane = lane_id(), gi = lane >> 2, s4 = lane & 3u, gbase = lane & ~3u;
    const uint32_t n = min(__ldg(&g.st->ulog_count), g.H);
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t gs = (((uint64_t)gridDim.x * blockDim.x) >> 5) * 8;
    unsigned long long slabs = 0, edges = 0;
    uint64_t i = warp0 * 8 + gi;
    uint32_t L = i < n ? g.ulog[i] : kNil;
    uint32_t nL = i + gs < n ? g.ulog[i + gs] : kNil;
    uint32_t src = L != kNil ? g.list_src[L] : 0;
    unsigned long long mk = L != kNil ? g.lmark[L] : 0;
    for (uint64_t base = warp0 * 8; base < n; base += gs, i += gs) {
        const uint32_t nnL = i + 2 * gs < n ? g.ulog[i + 2 * gs] : kNil;
        const uint32_t nsrc = nL != kNil ? g.list_src[nL] : 0;
        const unsigned long long nmk = nL != kNil ? g.lmark[nL] : 0;
        const uint32_t mlane = (uint32_t)(mk & 0xFF);
        uint32_t first_lane = mlane == kInvalidLane ? 32u : mlane;
        uint32_t slab = L != kNil ? (uint32_t)(mk >> 32) : kNil;
        bool active = slab != kNil;
        for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
            uint4 lo = make_uint4(kEmptyKey, kFull, kFull, kFull), hi = lo;
            if (active) {
                const uint4 *q = reinterpret_cast<const uint4 *>(slab_ptr(g, slab) + s4 * 8);
                lo = __ldcg(q);
                hi = __ldcg(q + 1);
            }
            slabs += __popc(__ballot_sync(kFull, active && s4 == 0));
            const bool last = s4 == 3u;
            const uint32_t w0 = 8 * s4;
            const uint32_t e[4] = {lo.x, lo.z, hi.x, last ? src : hi.z};
            const bool act[4] = {active && lo.x < kTombKey && w0 >= first_lane,
                                 active && lo.z < kTombKey && w0 + 2 >= first_lane,
                                 active && hi.x < kTombKey && w0 + 4 >= first_lane,
                                 last ? active : (active && hi.z < kTombKey && w0 + 6 >= first_lane)};
            edges += __popc(__ballot_sync(kFull, act[0])) + __popc(__ballot_sync(kFull, act[1])) +
                     __popc(__ballot_sync(kFull, act[2])) + __popc(__ballot_sync(kFull, act[3] && !last));
            if (!group_union<4, 4>(p, e, act, 1u << 20) && lane == 0)
                *failed = 1;
            const uint32_t nxt = __shfl_sync(kFull, hi.w, gbase + 3);
            if (active) {
                if (nxt == kNil || hop + 1 >= max_hops)
                    active = false;
                else
                    slab = nxt;
            }
            first_lane = 0;
        }
        L = nL;
        nL = nnL;
        src = nsrc;
        mk = nmk;
    }
    count_add(g.st, kCtrWccUpdSlabs, slabs);
    count_add(g.st, kCtrWccUpdEdges, edges);
}

// Incremental pass from the inserted-edge log (insert-only epochs, so every
// logged edge is live): each lane unites the two ends of one logged edge
// (a one-lane group_union: both roots found in lockstep, the larger hooked
// under the smaller).
__global__ void __launch_bounds__(256) k_uf_hook_log(DevState *st, const uint4 *__restrict__ ilog, uint32_t cap,
                                                     uint32_t *p, int *failed)
{
    const uint32_t n = min(__ldg(&st->ilog_count), cap);
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long entries = 0;
    for (uint64_t wb = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull; wb < n; wb += stride) {
        const uint64_t i = wb + lane_id();
        const uint4 e = i < n ? __ldcs(&ilog[i]) : make_uint4(0, 0, 0, 0);
        const uint32_t x[2] = {e.x, e.y};
        const bool act[2] = {i < n, i < n};
        entries += __popc(__ballot_sync(kFull, i < n));
        if (!group_union<1, 2>(p, x, act, 1u << 20) && lane_id() == 0)
            *failed = 1;
    }
    count_add(st, kCtrWccLog, entries);
    count_add(st, kCtrWccUpdEdges, entries);
}

// Static pass as a streaming scan over the whole slab array instead of chain
// walks.  A warp takes 32 consecutive slabs at a time: one coalesced load of
// their owners (per-slab source, kNil for an unused pool slab; read a chunk
// ahead), the slabs in use compacted in shared memory, then eight slabs per
// step, one per 4-lane group (lane s4 holds words 8*s4 .. 8*s4+7, i.e. pairs
// 4*s4 .. 4*s4+3, as two 16-byte loads), the next step's slabs loaded before
// this step's finds.  Each slab's owner (in the last lane's fourth slot: the
// unused lane and the next lane) and its live destinations are united with
// one group_union (four elements per lane, found in lockstep).  The scan
// keeps the slabs in registers rather than staging them in shared memory:
// the finds' parent loads depend on L1, which shared-memory buffers would
// take away.
__global__ void __launch_bounds__(256) k_uf_hook_slabs(GView g, uint32_t *p, int *failed)
{
    __shared__ uint8_t comp[8][32];
    const uint32_t lane = lane_id(), g4 = lane >> 2, s4 = lane & 3u, w = threadIdx.x >> 5;
    const uint64_t total = (uint64_t)g.H + g.P;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) * 32;
    const uint4 none = make_uint4(kEmptyKey, kFull, kFull, kFull);
    auto part = [&](uint64_t s, int h) {
        return __ldcg(reinterpret_cast<const uint4 *>(slab_ptr(g, (uint32_t)s) + s4 * 8 + h * 4));
    };
    unsigned long long slabs = 0, edges = 0;
    uint64_t c = warp0 * 32;
    uint32_t own_next = c + lane < total ? __ldcg(&g.owner[c + lane]) : kNil;
    for (; c < total; c += stride) {
        const uint32_t own_l = own_next;
        own_next = c + stride + lane < total ? __ldcg(&g.owner[c + stride + lane]) : kNil;
        const uint32_t live = __ballot_sync(kFull, own_l != kNil);
        const uint32_t n = __popc(live);
        if (own_l != kNil)
            comp[w][__popc(live & ((1u << lane) - 1))] = (uint8_t)lane;
        __syncwarp();
        uint32_t it = g4 < n ? comp[w][g4] : 32u;
        uint4 lo = none, hi = none;
        if (it < 32) {
            lo = part(c + it, 0);
            hi = part(c + it, 1);
        }
        for (uint32_t j = g4; j - g4 < n; j += 8) {
            // the next step's slabs
            const uint32_t nit = j + 8 < n ? comp[w][j + 8] : 32u;
            uint4 nlo = none, nhi = none;
            if (nit < 32) {
                nlo = part(c + nit, 0);
                nhi = part(c + nit, 1);
            }
            const bool active = it < 32;
            const uint32_t own = __shfl_sync(kFull, own_l, it & 31);
            slabs += __popc(__ballot_sync(kFull, active && s4 == 0));
            const bool last = s4 == 3u;
            const uint32_t e[4] = {lo.x, lo.z, hi.x, last ? own : hi.z};
            const bool act[4] = {active && lo.x < kTombKey, active && lo.z < kTombKey, active && hi.x < kTombKey,
                                 last ? active : (active && hi.z < kTombKey)};
            edges += __popc(__ballot_sync(kFull, act[0])) + __popc(__ballot_sync(kFull, act[1])) +
                     __popc(__ballot_sync(kFull, act[2])) + __popc(__ballot_sync(kFull, act[3] && !last));
            if (!group_union<4, 4>(p, e, act, 1u << 20) && lane == 0)
                *failed = 1;
            lo = nlo;
            hi = nhi;
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
    if (incremental && g->ilog_ok && g->d_ilog) {
        MK_TRY(timed(g, "wcc_hook_updated", s, 1, [&]() {
            const uint64_t threads = std::max<uint64_t>(g->ilog_bound, 1);
            k_uf_hook_log<<<std::min<uint32_t>(grid_for(threads, 256), num_sms() * 8), 256, 0, s>>>(
                g->d_state, g->d_ilog, (uint32_t)g->ilog_cap, c->uf, failed);
            return cudaSuccess;
        }));
    } else if (incremental) {
        MK_TRY(timed(g, "wcc_hook_updated", s, 1, [&]() {
            // one 4-lane group per logged list
            const uint64_t threads = std::max<uint64_t>(g->ulog_bound, 1) * 4;
            k_uf_hook<<<std::min<uint32_t>(grid_for(threads, 256), num_sms() * 12), 256, 0, s>>>(g->v, c->uf, max_hops,
                                                                                               failed);
            return cudaSuccess;
        }));
    } else {
        MK_TRY(timed(g, "wcc_hook_all", s, 1, [&]() {
            static const uint32_t grid = resident_grid(k_uf_hook_slabs, 256);
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
