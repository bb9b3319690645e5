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
// invalidation then spreads to every tree descendant of such a v (the
// paper's per-vertex walk up the parent chain, done here as a union-find
// style find with path halving so that the walks share their work); then
// every edge from a valid vertex into an invalidated one is relaxed.  Incremental prologue: the edges inserted since
// the last commit, read with the UpdateIterator, are relaxed.  Common
// epilogue: rounds until no distance improves.
//
// The round loops run on the device: one persistent cooperative kernel
// executes all rounds of a phase and separates them with a grid barrier whose
// waits are bounded, so the host never reads a frontier size (the paper's
// host loop reads it every round).  If the cooperative launch is refused, the
// same round body runs as one launch per round driven by the host.
#include "mk_host.h"
#include "walk.cuh"

#include <algorithm>

using namespace mk;

namespace {

constexpr uint32_t kInf32 = 0xFFFFFFFFu;
constexpr uint32_t kBarrierSpins = 1u << 24;

// consumer counter words
enum {
    kCnt0 = 0,        // kCnt0..kCnt0+2: rotating frontier sizes
    kOverflow = 3,
    kInvTotal = 4,
    kRoundsDone = 5,
    kClearWords = 8,  // words [0, 8) are cleared at the start of every call
    kSoloR = 6,       // round index reached by a solo phase of block 0
    kRid = 8,         // last round stamp used (kept across calls)
    kBar = 10         // grid barrier: arrival count, generation
};
// A frontier of at most kSoloLists lists is processed by block 0 alone, with
// block-level barriers between rounds, for at most kSoloRounds rounds in a
// row (so the other blocks' bounded wait at the grid barrier never expires).
constexpr uint32_t kSoloLists = 1024;
constexpr uint32_t kSoloRounds = 4096;

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

__device__ __forceinline__ uint32_t ld_volatile(const uint32_t *p) { return *(volatile const uint32_t *)p; }

} // namespace

// Arguments of the round loops (one struct so the cooperative launch passes
// a single pointer).
struct RoundArgs {
    GView g;
    unsigned long long *D;
    uint2 *front[2];      // list frontiers: <list, source of the list>
    uint32_t *ctr;        // consumer counter words
    uint32_t *stamp;
    uint32_t *inv;
    uint32_t cap;
    uint32_t max_hops;
    uint32_t max_rounds;
    uint32_t source;
    int unit;
    uint32_t *anc;        // decremental prologue: tree ancestor of each vertex (pointer jumping)
};

namespace {

// One round over frontier F[0, n): warps stride over groups of 32 lists and
// walk them four at a time (8-lane groups, walk_lists_g8_from), the head
// slabs of the next four loaded before the current four are walked.
__device__ void relax_body(const RoundArgs &a, const uint2 *F, uint32_t n, uint2 *Fn, uint32_t *cnt,
                           uint32_t round, uint64_t warp0, uint64_t nwarps)
{
    const GView &g = a.g;
    const uint32_t lane = lane_id(), gi = lane >> 3;
    int *overflow = (int *)(a.ctr + kOverflow);
    unsigned long long lists = 0, slabs = 0, edges = 0, improved = 0;
    for (uint64_t base = warp0 * 32; base < n; base += nwarps * 32) {
        const uint64_t i = base + lane;
        bool todo = i < n;
        // each lane fetches its own entry and the source's distance up front
        const uint2 e = todo ? F[i] : make_uint2(0, 0);
        const uint32_t mine = e.x, my_x = e.y;
        const uint32_t my_dx = todo ? node_dist(__ldcg(&a.D[my_x])) : kInf32;
        lists += __popc(__ballot_sync(kFull, todo));
        todo = todo && my_dx != kInf32;
        const uint32_t q = __ballot_sync(kFull, todo);
        const uint32_t np = ((uint32_t)__popc(q) + 3) / 4;
        uint32_t owner = group_item(q, 0, gi);
        const uint32_t L0 = __shfl_sync(kFull, mine, owner & 31);
        uint4 x0 = group_load(g, owner < 32 ? L0 : kNil);
        for (uint32_t pass = 0; pass < np; ++pass) {
            const uint32_t L = __shfl_sync(kFull, mine, owner & 31);
            const bool has = owner < 32;
            const uint32_t x = __shfl_sync(kFull, my_x, owner & 31);
            const uint32_t dx0 = __shfl_sync(kFull, my_dx, owner & 31);
            const uint32_t dx = has ? dx0 : kInf32;
            // the next pass's head slabs
            const uint32_t nowner = group_item(q, pass + 1, gi);
            const uint32_t nL = __shfl_sync(kFull, mine, nowner & 31);
            const uint4 nx0 = group_load(g, nowner < 32 ? nL : kNil);
            slabs += walk_lists_g8_from(g, has ? L : kNil, true, x0, 0, a.max_hops,
                                        [&](uint32_t y, uint32_t w, bool live) {
                                            edges += __popc(__ballot_sync(kFull, live));
                                            bool up = live && relax(a.D, x, dx, y, a.unit ? 1u : w);
                                            up = up && first_this_round(a.stamp, y, round);
                                            improved += __popc(__ballot_sync(kFull, up));
                                            enqueue_lists(g, y, up, Fn, cnt, a.cap, overflow);
                                        });
            owner = nowner;
            x0 = nx0;
        }
    }
    count_add(g.st, kCtrRelaxLists, lists);
    count_add(g.st, kCtrRelaxSlabs, slabs);
    count_add(g.st, kCtrRelaxEdges, edges);
    count_add(g.st, kCtrRelaxImproved, improved);
}

// Round r of a phase: reads the size in cnts[r % 3], appends to
// cnts[(r+1) % 3] and clears cnts[(r+2) % 3] for round r+1 (cnts: the three
// global counters, or block 0's shared copies during a solo phase).
// Frontier r is front[r & 1].
__device__ __forceinline__ void round_step(const RoundArgs &a, uint32_t *cnts, uint32_t r, uint32_t n, uint64_t warp0,
                                           uint64_t nwarps, uint32_t rid)
{
    const uint32_t in = r & 1;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        cnts[(r + 2) % 3] = 0;
    uint32_t *cnt = cnts + (r + 1) % 3;
    relax_body(a, a.front[in], n, a.front[in ^ 1], cnt, rid + 2 + r, warp0, nwarps);
}

// Bounded sense-counting grid barrier for a co-resident (cooperative) grid.
// Returns false when a wait gave up.
__device__ bool grid_barrier(uint32_t *bar)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile uint32_t *gen = bar + 1;
        const uint32_t g0 = *gen;
        __threadfence();
        int ok = 1;
        if (atomicAdd(&bar[0], 1u) == gridDim.x - 1) {
            atomicExch(&bar[0], 0u);
            __threadfence();
            atomicAdd(&bar[1], 1u);
        } else {
            uint32_t spins = 0;
            while (*gen == g0) {
                if (++spins > kBarrierSpins) {
                    ok = 0;
                    break;
                }
                __nanosleep(64);
            }
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

} // namespace

// All rounds of one phase in one cooperative launch.  The phase input is
// front[0] with its size in ctr[kCnt0]; ctr[kCnt0 + 1] must be zero.  Large
// frontiers are processed by the whole grid, one grid barrier per round.
// While the frontier stays small, block 0 runs the rounds alone (its warps
// striding over the frontier, its frontier sizes in shared memory,
// __syncthreads between rounds) for at most kSoloRounds rounds; the solo
// phase sits between two grid barriers, so no block reads a global size
// while block 0 changes them, and the others wait at one barrier instead of
// one per round.
__global__ void __launch_bounds__(256, 3) k_rounds(RoundArgs a)
{
    __shared__ uint32_t solo_cnt[3];
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t rid = ld_volatile(a.ctr + kRid);
    uint32_t *gcnt = a.ctr + kCnt0;
    uint32_t r = 0, bars = 0;
    bool ok = true;
    while (r < a.max_rounds) {
        uint32_t n = ld_volatile(gcnt + r % 3);
        if (n == 0)
            break;
        if (n > kSoloLists) {
            round_step(a, gcnt, r, n, warp0, nwarps, rid);
            ++bars;
            if (!grid_barrier(a.ctr + kBar)) {
                ok = false;
                break;
            }
            ++r;
            continue;
        }
        // every block has read n: block 0 may now change the global sizes
        bars += 2;
        if (!grid_barrier(a.ctr + kBar)) {
            ok = false;
            break;
        }
        if (blockIdx.x == 0) {
            const uint64_t bw0 = threadIdx.x >> 5, bnw = blockDim.x >> 5;
            if (threadIdx.x == 0) {
                solo_cnt[r % 3] = n;
                solo_cnt[(r + 1) % 3] = 0;
                solo_cnt[(r + 2) % 3] = 0;
            }
            __syncthreads();
            uint32_t steps = 0;
            do {
                round_step(a, solo_cnt, r, n, bw0, bnw, rid);
                __syncthreads();
                ++r;
                ++steps;
                n = *(volatile uint32_t *)&solo_cnt[r % 3];
                __syncthreads();
            } while (n > 0 && n <= kSoloLists && steps < kSoloRounds && r < a.max_rounds);
            if (threadIdx.x == 0) {
                gcnt[r % 3] = n;
                gcnt[(r + 1) % 3] = 0;
                gcnt[(r + 2) % 3] = 0;
                a.ctr[kSoloR] = r;
            }
        }
        if (!grid_barrier(a.ctr + kBar)) {
            ok = false;
            break;
        }
        r = ld_volatile(a.ctr + kSoloR);
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctr[kRoundsDone] = r;
        atomicAdd(&a.g.st->ctr[kCtrRounds], (unsigned long long)r);
        atomicAdd(&a.g.st->ctr[kCtrGridBarriers], (unsigned long long)bars);
        if (!ok || r >= a.max_rounds)
            set_status(a.g.st, kErrTimeout);
    }
}

// One round, for the host-driven fallback.
__global__ void __launch_bounds__(256) k_round_once(RoundArgs a, uint32_t r, uint32_t n)
{
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    round_step(a, a.ctr + kCnt0, r, n, warp0, nwarps, ld_volatile(a.ctr + kRid));
    if (blockIdx.x == 0 && threadIdx.x == 0)
        a.ctr[kRoundsDone] = r + 1;
}

__global__ void k_sssp_init(unsigned long long *D, uint32_t V, uint32_t source, uint2 *front, uint32_t *count,
                            const uint2 *vinfo)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V)
        D[v] = v == source ? ((unsigned long long)0 << 32 | source) : kInfNode;
    if (v == 0) {
        const uint2 vi = vinfo[source];
        for (uint32_t b = 0; b < vi.y; ++b)
            front[b] = make_uint2(vi.x + b, source);
        *count = vi.y;
    }
}

// Decremental seeds: a deleted edge (u, v) that is v's tree edge invalidates
// v (its tree node becomes <INF, INVALID> and its bit is set in `inv`).
__global__ void k_invalidate(const unsigned long long *dlog, const DevState *st, RoundArgs a)
{
    const uint32_t n = st->dlog_count;
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n)
        return;
    const unsigned long long e = dlog[i];
    const uint32_t u = (uint32_t)(e >> 32), v = (uint32_t)e;
    const unsigned long long dv = __ldcg(&a.D[v]);
    if (v != a.source && dv != kInfNode && node_parent(dv) == u && atomicCAS(&a.D[v], dv, kInfNode) == dv) {
        atomicAdd(a.ctr + kInvTotal, 1u);
        atomicOr(&a.inv[v >> 5], 1u << (v & 31));
        atomicAdd(&a.g.st->ctr[kCtrInvalidated], 1ull);
    }
}

// The invalidation spreads to every tree descendant of the seeds: a vertex
// is invalid iff the path from it up the shortest-path tree reaches a seed
// before the source.  The paper walks each vertex up to the source; here the
// walks share their work by pointer jumping on a copy of the parent pointers
// (the union-find "find" with path halving): anc[v] starts as v's tree
// parent, and as v itself at the source, at the seeds and at unreached
// vertices, which are the roots of the forest.  Tree parents have strictly
// smaller distances (weights are >= 1), so the forest has no cycles.
__global__ void k_inv_anc_init(RoundArgs a)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= a.g.V)
        return;
    const unsigned long long d = __ldcg(&a.D[v]);
    a.anc[v] = (v == a.source || d == kInfNode) ? v : node_parent(d);
}

// Each reached vertex finds its root (path halving on anc) and is invalidated
// when the root is not the source.  The invalidated vertices of one warp set
// their bits with one atomicOr (32 consecutive vertices share a bitmap word).
__global__ void k_inv_jump(RoundArgs a)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if ((v & ~31u) >= a.g.V)
        return;
    bool bad = false;
    if (v < a.g.V && v != a.source && __ldcg(&a.D[v]) != kInfNode) {
        uint32_t x = v, hops = 0;
        bool ok = true;
        // plain (L1-cacheable) loads: a stale anc value is an older ancestor,
        // and roots never change, so every walk still ends at v's root
        // while the source's line, where most walks end, stays in L1
        for (;;) {
            const uint32_t px = a.anc[x];
            if (px == x)
                break;
            const uint32_t ppx = a.anc[px];
            if (ppx == px) {
                x = px;
                break;
            }
            a.anc[x] = ppx; // path halving: ppx is an ancestor of x
            x = ppx;
            if (++hops > a.max_rounds) { // parent pointers not a forest: corrupted state
                ok = false;
                break;
            }
        }
        if (!ok)
            set_status(a.g.st, kErrTimeout);
        bad = ok && x != a.source;
    }
    if (bad)
        a.D[v] = kInfNode;
    const uint32_t mask = __ballot_sync(kFull, bad);
    if (lane_id() == 0 && mask) {
        atomicOr(&a.inv[v >> 5], mask);
        atomicAdd(a.ctr + kInvTotal, (uint32_t)__popc(mask));
        count_add(a.g.st, kCtrInvalidated, __popc(mask));
    }
}

// After invalidation: relax every edge out of a valid vertex into a vertex
// invalidated by this call.  The target test reads the invalidation bitmap,
// which stays fixed during the pass, so every such edge is relaxed even after
// another in-neighbour has already given its target a finite distance; does
// nothing if nothing was invalidated.  A streaming scan over every slab in
// use (through the per-slab owner array): a warp takes 32 consecutive slabs,
// reads their owners in one coalesced load and the owners' tree nodes in one
// gather, compacts the slabs whose source has a finite distance, and reads
// those four per step, one per 8-lane group, loading the next step's slabs
// before relaxing this step's edges.
__global__ void __launch_bounds__(256) k_relax_into_invalid_slabs(RoundArgs a)
{
    __shared__ uint8_t comp[8][32];
    const GView &g = a.g;
    if (ld_volatile(a.ctr + kInvTotal) == 0)
        return;
    const uint32_t lane = lane_id(), gi = lane >> 3, sub = lane & 7u, w = threadIdx.x >> 5;
    const uint64_t total = (uint64_t)g.H + g.P;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t round = ld_volatile(a.ctr + kRid) + 1;
    int *overflow = (int *)(a.ctr + kOverflow);
    const uint4 none = make_uint4(kEmptyKey, kFull, kFull, kFull);
    unsigned long long slabs = 0, edges = 0, improved = 0;
    for (uint64_t c = warp0 * 32; c < total; c += nwarps * 32) {
        // 32 consecutive slabs: owners (one coalesced load), then the owners'
        // distances; only slabs of reachable, valid sources are read
        const uint32_t own_l = c + lane < total ? __ldcg(&g.owner[c + lane]) : kNil;
        const uint32_t dx_l = own_l != kNil ? node_dist(__ldcg(&a.D[own_l])) : kInf32;
        const uint32_t live = __ballot_sync(kFull, dx_l != kInf32);
        const uint32_t n = __popc(live);
        if (dx_l != kInf32)
            comp[w][__popc(live & ((1u << lane) - 1))] = (uint8_t)lane;
        __syncwarp();
        uint32_t it = gi < n ? comp[w][gi] : 32u;
        uint4 x = none;
        if (it < 32)
            x = __ldcg(reinterpret_cast<const uint4 *>(slab_ptr(g, (uint32_t)(c + it)) + sub * 4));
        for (uint32_t k = gi; k - gi < n; k += 4) {
            const uint32_t nit = k + 4 < n ? comp[w][k + 4] : 32u;
            uint4 nx = none;
            if (nit < 32)
                nx = __ldcg(reinterpret_cast<const uint4 *>(slab_ptr(g, (uint32_t)(c + nit)) + sub * 4));
            const bool active = it < 32;
            const uint32_t own = __shfl_sync(kFull, own_l, it & 31);
            const uint32_t dx = __shfl_sync(kFull, dx_l, it & 31);
            slabs += __popc(__ballot_sync(kFull, active && sub == 0));
            const bool last = sub == 7u;
#pragma unroll
            for (int k2 = 0; k2 < 2; ++k2) {
                const uint32_t y = k2 ? x.z : x.x, wt = k2 ? x.w : x.y;
                const bool live_e = active && !(k2 && last) && y < kTombKey;
                edges += __popc(__ballot_sync(kFull, live_e));
                const bool target = live_e && ((__ldg(&a.inv[y >> 5]) >> (y & 31)) & 1u); // fixed during the pass
                bool up = target && relax(a.D, own, dx, y, a.unit ? 1u : wt);
                up = up && first_this_round(a.stamp, y, round);
                improved += __popc(__ballot_sync(kFull, up));
                enqueue_lists(g, y, up, a.front[0], a.ctr + kCnt0, a.cap, overflow);
            }
            x = nx;
            it = nit;
        }
        __syncwarp();
    }
    count_add(g.st, kCtrSeedLists, slabs);
    count_add(g.st, kCtrSeedSlabs, slabs);
    count_add(g.st, kCtrSeedEdges, edges);
    count_add(g.st, kCtrSeedImproved, improved);
}

// Incremental seeds: relax the entries inserted since the last commit
// (UpdateIterator over the lists flagged as updated).
__global__ void __launch_bounds__(256) k_relax_updated(RoundArgs a)
{
    const GView &g = a.g;
    const uint32_t lane = lane_id(), gi = lane >> 3;
    const uint64_t base = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull;
    if (base >= g.H)
        return;
    const uint32_t round = ld_volatile(a.ctr + kRid) + 1;
    int *overflow = (int *)(a.ctr + kOverflow);
    const uint64_t l = base + lane;
    bool todo = false;
    uint32_t x = 0, dx = kInf32, my_first = 0, my_start = kNil;
    if (l < g.H && g.lupd[l]) {
        x = g.list_src[l];
        dx = node_dist(__ldcg(&a.D[x]));
        todo = dx != kInf32;
        if (todo)
            my_start = update_begin(g, (uint32_t)l, &my_first);
    }
    const uint32_t q = __ballot_sync(kFull, todo);
    const uint32_t np = ((uint32_t)__popc(q) + 3) / 4;
    unsigned long long slabs = 0, edges = 0, improved = 0;
    // the first slab of each walk is loaded one pass ahead
    uint32_t owner = group_item(q, 0, gi);
    const uint32_t s0 = __shfl_sync(kFull, my_start, owner & 31);
    uint4 x0 = group_load(g, owner < 32 ? s0 : kNil);
    for (uint32_t pass = 0; pass < np; ++pass) {
        const bool has = owner < 32;
        const uint32_t src = __shfl_sync(kFull, x, owner & 31);
        const uint32_t dsrc = __shfl_sync(kFull, dx, owner & 31);
        const uint32_t first_lane = __shfl_sync(kFull, my_first, owner & 31);
        const uint32_t start0 = __shfl_sync(kFull, my_start, owner & 31);
        const uint32_t start = has ? start0 : kNil;
        const uint32_t nowner = group_item(q, pass + 1, gi);
        const uint32_t ns = __shfl_sync(kFull, my_start, nowner & 31);
        const uint4 nx0 = group_load(g, nowner < 32 ? ns : kNil);
        slabs += walk_lists_g8_from(g, start, true, x0, first_lane, a.max_hops, [&](uint32_t y, uint32_t w, bool live) {
            edges += __popc(__ballot_sync(kFull, live));
            bool up = live && relax(a.D, src, dsrc, y, a.unit ? 1u : w);
            up = up && first_this_round(a.stamp, y, round);
            improved += __popc(__ballot_sync(kFull, up));
            enqueue_lists(g, y, up, a.front[0], a.ctr + kCnt0, a.cap, overflow);
        });
        owner = nowner;
        x0 = nx0;
    }
    count_add(g.st, kCtrSeedLists, __popc(q));
    count_add(g.st, kCtrSeedSlabs, slabs);
    count_add(g.st, kCtrSeedEdges, edges);
    count_add(g.st, kCtrSeedImproved, improved);
}

// Ends a call: advances the round stamp past every id used, reports an
// overflowed frontier.
__global__ void k_sssp_finish(uint32_t *ctr, DevState *st)
{
    ctr[kRid] += ctr[kRoundsDone] + 2;
    if (ctr[kOverflow])
        set_status(st, kErrTimeout);
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

// ---------------------------------------------------------------- host side

namespace {

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
        st = device_alloc(g, (void **)&c->front[0], H * 8);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->front[1], H * 8);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->stamp, V * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->inv, (V + 31) / 32 * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->anc, V * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&c->counters, 64);
    if (st == MK_OK && (cudaMemset(c->stamp, 0, V * 4) != cudaSuccess || cudaMemset(c->counters, 0, 64) != cudaSuccess))
        st = MK_ERR_CUDA;
    if (st != MK_OK) {
        device_free(g, c->D, V * 8);
        device_free(g, c->front[0], H * 8);
        device_free(g, c->front[1], H * 8);
        device_free(g, c->stamp, V * 4);
        device_free(g, c->inv, (V + 31) / 32 * 4);
        device_free(g, c->anc, V * 4);
        device_free(g, c->counters, 64);
        delete c;
        return st;
    }
    g->consumers[key] = c;
    *out = c;
    return MK_OK;
}

} // namespace

namespace mk {

// Co-resident grid of k_rounds: SMs x blocks per SM, the latter the
// occupancy limit or the tuned value if smaller.
int rounds_grid(int blocks_per_sm)
{
    static int sms = 0, per_sm_max = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm_max, k_rounds, 256, 0);
        per_sm_max = std::max(per_sm_max, 1);
    }
    const int per = blocks_per_sm > 0 ? std::min(blocks_per_sm, per_sm_max) : per_sm_max;
    return std::max(1, sms * per);
}

int rounds_max_blocks_per_sm()
{
    rounds_grid(0);
    int dev = 0, per = 0;
    cudaGetDevice(&dev);
    cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rounds, 256, 0);
    return std::max(per, 1);
}

} // namespace mk

namespace {

// Runs every round of one phase.  Input: front[0], size in ctr[kCnt0],
// ctr[kCnt0 + 1] zero.
mk_status run_phase(mk_graph *g, RoundArgs a, const char *name, cudaStream_t s)
{
    const int grid = rounds_grid(g->tune.rounds_blocks_per_sm);
    void *args[] = {&a};
    mk_status st = timed(g, name, s, 1, [&]() {
        return cudaLaunchCooperativeKernel((const void *)k_rounds, dim3(grid), dim3(256), args, 0, s);
    });
    if (st == MK_OK)
        return MK_OK;
    cudaGetLastError();
    // fallback: one launch per round, the host reads each size
    for (uint32_t r = 0;; ++r) {
        if (r > a.max_rounds)
            return MK_ERR_TIMEOUT;
        MK_CUDA(cudaMemcpyAsync(g->h_pinned, a.ctr + kCnt0 + r % 3, 4, cudaMemcpyDeviceToHost, s));
        MK_CUDA(cudaStreamSynchronize(s));
        const uint32_t n = g->h_pinned[0];
        if (n == 0)
            return MK_OK;
        MK_TRY(timed(g, name, s, 1, [&]() {
            k_round_once<<<grid_for((uint64_t)n, 256), 256, 0, s>>>(a, r, n);
            return cudaSuccess;
        }));
    }
}

mk_status run_sssp(mk_graph *g, int kind, uint32_t source, uint32_t *d_dist, uint32_t *d_parent, cudaStream_t s)
{
    if (!g || source >= g->v.V)
        return MK_ERR_INVALID_ARG;
    Consumer *c = nullptr;
    MK_TRY(get_consumer(g, kind, source, &c));
    const uint32_t V = g->v.V, H = g->v.H;
    RoundArgs a{};
    a.g = g->v;
    a.D = c->D;
    a.front[0] = c->front[0];
    a.front[1] = c->front[1];
    a.ctr = c->counters;
    a.stamp = c->stamp;
    a.inv = c->inv;
    a.anc = c->anc;
    a.cap = H;
    a.max_hops = g->v.P + 2;
    a.max_rounds = V + 2;
    a.source = source;
    a.unit = kind == kBfs ? 1 : 0;
    const bool incremental = c->epoch == g->epoch;
    MK_CUDA(cudaMemsetAsync(c->counters, 0, kClearWords * 4, s));
    MK_CUDA(cudaMemsetAsync(c->counters + kBar, 0, 8, s));
    if (!incremental) {
        MK_TRY(timed(g, "sssp_init", s, 1, [&]() {
            k_sssp_init<<<grid_for(V, 256), 256, 0, s>>>(c->D, V, source, c->front[0], c->counters + kCnt0,
                                                         g->v.vinfo);
            return cudaSuccess;
        }));
    } else {
        if (g->epoch_has_deletes) {
            // decremental prologue: invalidate, spread down the tree, then
            // relax the edges from valid into invalidated vertices
            MK_CUDA(cudaMemsetAsync(c->inv, 0, (size_t)(V + 31) / 32 * 4, s));
            MK_TRY(timed(g, "sssp_invalidate", s, 1, [&]() {
                k_invalidate<<<grid_for(std::max<uint64_t>(g->dlog_bound, 1), 256), 256, 0, s>>>(g->d_dlog,
                                                                                                 g->d_state, a);
                return cudaSuccess;
            }));
            MK_TRY(timed(g, "sssp_invalidate_jump", s, 2, [&]() {
                k_inv_anc_init<<<grid_for(V, 256), 256, 0, s>>>(a);
                k_inv_jump<<<grid_for(V, 256), 256, 0, s>>>(a);
                return cudaSuccess;
            }));
            MK_TRY(timed(g, "sssp_relax_into_invalid", s, 1, [&]() {
                const uint64_t warps = ((uint64_t)H + g->v.P + 31) / 32;
                const uint32_t grid = (uint32_t)std::min<uint64_t>(grid_for(warps * 32, 256), (uint64_t)num_sms() * 16);
                k_relax_into_invalid_slabs<<<grid, 256, 0, s>>>(a);
                return cudaSuccess;
            }));
        }
        // incremental prologue: edges inserted since the last commit
        MK_TRY(timed(g, "sssp_relax_updated", s, 1, [&]() {
            k_relax_updated<<<grid_for((uint64_t)H, 256), 256, 0, s>>>(a);
            return cudaSuccess;
        }));
    }
    // common epilogue: rounds until no distance improves
    MK_TRY(run_phase(g, a, "sssp_rounds", s));
    MK_TRY(timed(g, "sssp_unpack", s, 2, [&]() {
        k_sssp_finish<<<1, 1, 0, s>>>(c->counters, g->d_state);
        if (d_dist || d_parent)
            k_unpack<<<grid_for(V, 256), 256, 0, s>>>(c->D, V, d_dist, d_parent);
        return cudaSuccess;
    }));
    c->epoch = g->epoch;
    c->seq = g->change_seq;
    return MK_OK;
}

} // namespace

namespace mk {

// Duration of one static BFS from `source` (CUDA events on s), for the
// autotuner; leaves a valid BFS state for that source.
mk_status time_static_bfs(mk_graph *g, uint32_t source, cudaStream_t s, float *ms)
{
    Consumer *c = nullptr;
    MK_TRY(get_consumer(g, kBfs, source, &c));
    c->epoch = ~0ull;
    cudaEvent_t a, b;
    MK_CUDA(cudaEventCreate(&a));
    MK_CUDA(cudaEventCreate(&b));
    cudaEventRecord(a, s);
    mk_status st = run_sssp(g, kBfs, source, nullptr, nullptr, s);
    cudaEventRecord(b, s);
    cudaEventSynchronize(b);
    cudaEventElapsedTime(ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return st;
}

} // namespace mk

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
