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
#include "tma.cuh"
#include "walk.cuh"

#include <algorithm>

using namespace mk;

namespace {

constexpr uint32_t kInf32 = 0xFFFFFFFFu;
constexpr uint32_t kRoundsMaxThreads = 1024; // block size limit of the persistent round kernel
constexpr uint32_t kBarrierSpins = 1u << 24;

// consumer counter words
enum {
    kCnt0 = 0,        // kCnt0..kCnt0+2: rotating frontier sizes
    kOverflow = 3,
    kInvTotal = 4,    // nonzero once this call invalidated a vertex
    kRoundsDone = 5,
    kClearWords = 8,  // words [0, 8) are cleared at the start of every call
    kSoloR = 6,       // round index reached by a solo phase of block 0
    kRid = 8,         // last round stamp used (kept across calls)
    kPhase = 9,       // Near-Far: last far-pile phase stamp used (kept across calls)
    kBar = 10,        // grid barrier: arrivals of the launch so far
    kFarCnt0 = 11,    // Near-Far ordering: sizes of the two far piles (11, 12),
    kFarMin0 = 13,    // the smallest distance pushed to each (13, 14)
    kThresh = 15      // and the smallest source distance of the first frontier
};
// A frontier of at most kSoloLists lists is processed by block 0 alone, with
// block-level barriers between rounds, for at most kSoloRounds rounds in a
// row (so the other blocks' bounded wait at the grid barrier never expires).
// Block 0 (one SM) has up to 192 four-lane groups: a frontier of up to
// about one list per group costs block 0 one load chain a round, less than
// a grid barrier plus one chain; a larger one is faster on the whole grid.
constexpr uint32_t kSoloLists = 192;
constexpr uint32_t kSoloRounds = 4096;
// Near-Far ordering: the far pile is split into the frontier whenever the
// frontier holds fewer lists than this (a smaller frontier costs a round
// about as much as a larger one).
constexpr uint32_t kNearMin = 2048;

__device__ __forceinline__ uint32_t node_dist(unsigned long long d) { return (uint32_t)(d >> 32); }
__device__ __forceinline__ uint32_t node_parent(unsigned long long d) { return (uint32_t)d; }

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
    uint32_t barrier_spins; // polls before a grid-barrier wait gives up
    uint32_t source;
    int unit;
    uint32_t *dist;       // the caller's outputs (nullable), written when the phase ends
    uint32_t *parent;
    uint32_t delta;       // Near-Far bucket width (0: plain frontier rounds)
    uint32_t *far[2];     // Near-Far: the two far piles (V vertices each)
    uint32_t *fstamp;     // Near-Far: phase in which a vertex last joined a pile
};

namespace {

// Near-Far ordering of the rounds (an addition to the paper's frontier
// rounds, for graphs of large diameter and weight range): an improvement
// to a distance at or above the split distance T does not enqueue the
// vertex's lists; the vertex joins the far pile instead (once per phase,
// through its pile stamp), and whenever the frontier is small the pile is
// split at a larger T.  Only the order of the relaxations changes: the rounds
// still run until no distance improves, so the result is the same fixpoint.
struct NearFar {
    uint32_t T = kInf32;      // split distance of this phase
    uint32_t phase = 0;       // pile stamp of this phase
    uint32_t *pile = nullptr; // the pile this phase appends to
    uint32_t *count = nullptr;
    uint32_t *dmin = nullptr; // smallest distance pushed to it
};

// Appends y (lanes with pred) to the far pile once per phase.  Must be
// called by the full warp.
__device__ __forceinline__ void far_push(const RoundArgs &a, const NearFar &nf, uint32_t y, bool pred, uint32_t d)
{
    const bool take = pred && atomicExch(&a.fstamp[y], nf.phase) != nf.phase;
    const uint32_t m = __ballot_sync(kFull, take);
    if (!m)
        return;
    const uint32_t dm = __reduce_min_sync(kFull, take ? d : kInf32);
    uint32_t base = 0;
    if (lane_id() == 0) {
        base = atomicAdd(nf.count, (uint32_t)__popc(m));
        atomicMin(nf.dmin, dm);
    }
    base = __shfl_sync(kFull, base, 0);
    if (take) {
        const uint32_t at = base + __popc(m & lanemask_lt());
        if (at < a.g.V)
            nf.pile[at] = y;
        else
            *(int *)(a.ctr + kOverflow) = 1;
    }
}

// Relaxes the lane's four edges (x, y[k], w[k]) with live[k] and enqueues
// the lists of each vertex whose distance this lane lowered first in this
// round (staged in the block's frontier buffer).  The accesses of the four
// edges go out together, step by step: the four targets' tree nodes are
// read, then the atomic minima of the candidates that beat them are issued,
// then the improved targets' vinfo entries are read and their round stamps
// exchanged, so a slab costs three memory round trips per lane instead of
// three per edge.  Must be called by the full warp.
template <bool kNF = false>
__device__ __forceinline__ void relax_edges4(const RoundArgs &a, uint32_t x, uint32_t dx, const uint32_t (&y)[4],
                                             const uint32_t (&w)[4], const bool (&live)[4], uint32_t round,
                                             BlockFrontier &bq, uint2 *Fn, uint32_t *cnt, int *overflow,
                                             unsigned long long &edges, unsigned long long &improved,
                                             const NearFar *nf = nullptr)
{
    // candidate of edge k: <nd[k], x>
    auto cand = [&](uint32_t d) { return ((unsigned long long)d << 32) | x; };
    uint32_t nd[4];
    unsigned long long cur[4];
    bool up[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        edges += __popc(__ballot_sync(kFull, live[k]));
        const unsigned long long d = (unsigned long long)dx + (a.unit ? 1u : w[k]);
        up[k] = live[k] && d < kInf32;
        nd[k] = (uint32_t)d;
    }
#pragma unroll
    for (int k = 0; k < 4; ++k)
        cur[k] = up[k] ? __ldcg(&a.D[y[k]]) : 0ull;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        if (up[k] && cand(nd[k]) < cur[k])
            cur[k] = atomicMin(&a.D[y[k]], cand(nd[k]));
        else
            up[k] = false;
#pragma unroll
    for (int k = 0; k < 4; ++k)
        up[k] = up[k] && cand(nd[k]) < cur[k];
    if (kNF) {
        // improvements at or beyond the split distance wait in the far pile
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const bool fp = up[k] && nd[k] >= nf->T;
            up[k] = up[k] && !fp;
            far_push(a, *nf, y[k], fp, nd[k]);
        }
    }
    uint2 vi[4];
    uint32_t st[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        vi[k] = make_uint2(0, 0);
        st[k] = round;
        if (up[k]) {
            vi[k] = a.g.vinfo[y[k]];
            st[k] = atomicExch(&a.stamp[y[k]], round);
        }
    }
#pragma unroll
    for (int k = 0; k < 4; ++k) {
        up[k] = up[k] && st[k] != round;
        improved += __popc(__ballot_sync(kFull, up[k]));
        enqueue_lists_block(bq, y[k], up[k], vi[k], Fn, cnt, a.cap, overflow);
    }
}

// One round over frontier F[0, n): every 4-lane group of every warp takes
// one list at a time (group index + k * groups in the grid; eight lists per
// warp in flight), so a round's lists are spread over all warps; each
// group's entry, source distance and head slab are loaded one step ahead
// (the entry two steps ahead) while the current list is relaxed.
template <bool kNF = false>
__device__ void relax_body(const RoundArgs &a, const uint2 *F, uint32_t n, uint2 *Fn, uint32_t *cnt,
                           uint32_t round, uint64_t warp0, uint64_t nwarps, BlockFrontier &bq,
                           const NearFar *nf = nullptr)
{
    const GView &g = a.g;
    const uint32_t s4 = lane_id() & 3u, g4 = lane_id() >> 2;
    int *overflow = (int *)(a.ctr + kOverflow);
    unsigned long long lists = 0, slabs = 0, edges = 0, improved = 0;
    const uint64_t gs = nwarps * 8; // groups in the grid
    const uint2 none = make_uint2(kNil, 0);
    uint64_t i = warp0 * 8 + g4;
    // pipeline: entry e with its distance dx and head slab (lo, hi) (this
    // step), entry ne (next step)
    uint2 e = i < n ? F[i] : none;
    uint2 ne = i + gs < n ? F[i + gs] : none;
    uint32_t dx = e.x != kNil ? node_dist(__ldcg(&a.D[e.y])) : kInf32;
    uint4 lo, hi;
    group4_load(g, e.x, lo, hi);
    for (uint64_t base = warp0 * 8; base < n; base += gs, i += gs) {
        const uint2 nne = i + 2 * gs < n ? F[i + 2 * gs] : none;
        const uint32_t ndx = ne.x != kNil ? node_dist(__ldcg(&a.D[ne.y])) : kInf32;
        uint4 nlo, nhi;
        group4_load(g, ne.x, nlo, nhi);
        lists += __popc(__ballot_sync(kFull, e.x != kNil && s4 == 0));
        const uint32_t L = dx != kInf32 ? e.x : kNil;
        const uint32_t x = e.y, d = dx;
        slabs += walk_lists_g4_from(g, L, true, lo, hi, 0, a.max_hops,
                                    [&](const uint32_t(&y)[4], const uint32_t(&w)[4], const bool(&live)[4]) {
                                        relax_edges4<kNF>(a, x, d, y, w, live, round, bq, Fn, cnt, overflow,
                                                          edges, improved, nf);
                                    });
        e = ne;
        ne = nne;
        dx = ndx;
        lo = nlo;
        hi = nhi;
    }
    count_add(g.st, kCtrRelaxLists, lists);
    count_add(g.st, kCtrRelaxSlabs, slabs);
    count_add(g.st, kCtrRelaxEdges, edges);
    count_add(g.st, kCtrRelaxImproved, improved);
}

// Round r of a phase: reads the size in cnts[r % 3], appends to
// cnts[(r+1) % 3] and clears cnts[(r+2) % 3] for round r+1 (cnts: the three
// global counters, or block 0's shared copies during a solo phase).
// Frontier r is front[r & 1].  Called by whole blocks: the block's staged
// entries are flushed at the end.
template <bool kNF = false>
__device__ __forceinline__ void round_step(const RoundArgs &a, uint32_t *cnts, uint32_t r, uint32_t n, uint64_t warp0,
                                           uint64_t nwarps, uint32_t rid, BlockFrontier &bq,
                                           const NearFar *nf = nullptr)
{
    const uint32_t in = r & 1;
    if (blockIdx.x == 0 && threadIdx.x == 0)
        cnts[(r + 2) % 3] = 0;
    uint32_t *cnt = cnts + (r + 1) % 3;
    relax_body<kNF>(a, a.front[in], n, a.front[in ^ 1], cnt, rid + 2 + r, warp0, nwarps, bq, nf);
    bq_flush(bq, a.front[in ^ 1], cnt, a.cap, (int *)(a.ctr + kOverflow));
}

// Bounded grid barrier for a co-resident (cooperative) grid on one counter
// that only grows: barrier k of a launch is passed once the counter reaches
// k * gridDim.x, so a block arrives with one atomicAdd and polls; nothing is
// reset between barriers (the counter is zeroed before each launch).
// `passed` is the block's count of barriers so far (thread 0's copy is the
// one used).  Returns false when the wait gave up.
__device__ bool grid_barrier(uint32_t *bar, uint32_t &passed, uint32_t max_spins)
{
    __shared__ int ok_s;
    __syncthreads();
    if (threadIdx.x == 0) {
        const uint32_t target = (++passed) * gridDim.x;
        __threadfence();
        atomicAdd(bar, 1u);
        int ok = 1;
        uint32_t spins = 0;
        while ((int)(ld_volatile(bar) - target) < 0) {
            if (++spins > max_spins) {
                ok = 0;
                break;
            }
            __nanosleep(32);
        }
        __threadfence();
        ok_s = ok;
    }
    __syncthreads();
    return ok_s != 0;
}

// Splits the far pile pile[0, fc) at T2 before round r: a vertex whose
// distance is now below T2 has its lists appended to frontier r (under the
// stamp of the entries already there, rid + 1 + r, so a vertex queued
// there already is not queued twice), every other one moves to the pile of
// `next` under its phase stamp.  Called by every thread of every block.
__device__ __forceinline__ void far_split(const RoundArgs &a, const uint32_t *pile, uint32_t fc, const NearFar &next,
                                          uint32_t T2, uint32_t r, uint32_t rid, uint64_t warp0, uint64_t nwarps,
                                          BlockFrontier &bq)
{
    uint2 *out = a.front[r & 1];
    uint32_t *cnt = a.ctr + kCnt0 + r % 3;
    const uint32_t stampv = rid + 1 + r;
    int *overflow = (int *)(a.ctr + kOverflow);
    for (uint64_t wb = warp0 * 32; wb < fc; wb += nwarps * 32) {
        const uint64_t i = wb + lane_id();
        const bool valid = i < fc;
        uint32_t y = 0, dy = kInf32;
        if (valid) {
            y = __ldcg(&pile[i]);
            dy = node_dist(__ldcg(&a.D[y]));
        }
        bool near = valid && dy < T2;
        uint2 vi = make_uint2(0, 0);
        uint32_t st = stampv;
        if (near) {
            vi = a.g.vinfo[y];
            st = atomicExch(&a.stamp[y], stampv);
        }
        near = near && st != stampv;
        enqueue_lists_block(bq, y, near, vi, out, cnt, a.cap, overflow);
        far_push(a, next, y, valid && dy >= T2, dy);
    }
    bq_flush(bq, out, cnt, a.cap, overflow);
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
template <bool kNF>
__global__ void __launch_bounds__(kRoundsMaxThreads, 1) k_rounds(RoundArgs a)
{
    __shared__ uint32_t solo_cnt[3];
    __shared__ BlockFrontier bq;
    bq_init(bq);
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint32_t rid = __ldg(a.ctr + kRid);
    uint32_t *gcnt = a.ctr + kCnt0;
    uint32_t r = 0, bars = 0, passed = 0;
    bool ok = true;
    __shared__ uint32_t s_word, s_fc, s_fm;
    // Near-Far: the first split distance is delta above the smallest source
    // distance of the first frontier (ctr[kThresh] starts at INF)
    NearFar nf;
    uint32_t cur = 0, splits = 0, burst = 0;
    const uint32_t phase0 = kNF ? __ldg(a.ctr + kPhase) + 1 : 0;
    if (kNF) {
        const uint32_t n0 = min(ld_volatile(gcnt), a.cap);
        uint32_t m = kInf32;
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n0;
             i += (uint64_t)gridDim.x * blockDim.x)
            m = min(m, node_dist(__ldcg(&a.D[__ldcg(&a.front[0][i].y)])));
        m = __reduce_min_sync(kFull, m);
        if ((threadIdx.x & 31) == 0 && m != kInf32)
            atomicMin(a.ctr + kThresh, m);
        ++bars;
        ok = grid_barrier(a.ctr + kBar, passed, a.barrier_spins);
        const uint32_t t0 = ld_volatile(a.ctr + kThresh);
        nf.T = t0 >= kInf32 - a.delta ? kInf32 : t0 + a.delta;
        nf.phase = phase0;
        nf.pile = a.far[0];
        nf.count = a.ctr + kFarCnt0;
        nf.dmin = a.ctr + kFarMin0;
    }
    while (ok && r < a.max_rounds) {
        // one read of the frontier size per block (the grid's warps would
        // otherwise all read the same word)
        if (threadIdx.x == 0) {
            s_word = ld_volatile(gcnt + r % 3);
            if (kNF) {
                s_fc = ld_volatile(a.ctr + kFarCnt0 + cur);
                s_fm = ld_volatile(a.ctr + kFarMin0 + cur);
            }
        }
        __syncthreads();
        // a frontier never holds more than `cap` entries; a larger count
        // (entries dropped on overflow, reported below) is read as cap
        uint32_t n = min(s_word, a.cap);
        if (kNF && n < kNearMin && s_fc != 0) {
            // the near frontier is small: move the far pile's vertices below
            // the next split distance into it, once every block has read
            // the sizes above; the distance grows with each split in a row
            const uint32_t fc = min(s_fc, a.g.V), fm = s_fm;
            ++bars;
            if (!grid_barrier(a.ctr + kBar, passed, a.barrier_spins)) {
                ok = false;
                break;
            }
            const uint32_t base = max(nf.T, fm);
            const uint64_t width = (uint64_t)a.delta << min(burst, 16u);
            NearFar next;
            next.T = (uint64_t)base + width >= kInf32 ? kInf32 : (uint32_t)(base + width);
            next.phase = phase0 + ++splits;
            next.pile = a.far[cur ^ 1];
            next.count = a.ctr + kFarCnt0 + (cur ^ 1);
            next.dmin = a.ctr + kFarMin0 + (cur ^ 1);
            far_split(a, nf.pile, fc, next, next.T, r, rid, warp0, nwarps, bq);
            ++bars;
            if (!grid_barrier(a.ctr + kBar, passed, a.barrier_spins)) {
                ok = false;
                break;
            }
            // the old pile is empty again; no block reads its words before
            // the next split, two grid barriers on
            if (blockIdx.x == 0 && threadIdx.x == 0) {
                a.ctr[kFarCnt0 + cur] = 0;
                a.ctr[kFarMin0 + cur] = kInf32;
            }
            cur ^= 1;
            nf = next;
            ++burst;
            if (splits > a.max_rounds) {
                ok = false;
                break;
            }
            continue;
        }
        burst = 0;
        if (n == 0)
            break;
        if (n > kSoloLists) {
            round_step<kNF>(a, gcnt, r, n, warp0, nwarps, rid, bq, &nf);
            ++bars;
            if (!grid_barrier(a.ctr + kBar, passed, a.barrier_spins)) {
                ok = false;
                break;
            }
            ++r;
            continue;
        }
        // every block has read n: block 0 may now change the global sizes
        bars += 2;
        if (!grid_barrier(a.ctr + kBar, passed, a.barrier_spins)) {
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
                round_step<kNF>(a, solo_cnt, r, n, bw0, bnw, rid, bq, &nf);
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
        if (!grid_barrier(a.ctr + kBar, passed, a.barrier_spins)) {
            ok = false;
            break;
        }
        if (threadIdx.x == 0)
            s_word = ld_volatile(a.ctr + kSoloR);
        __syncthreads();
        r = s_word;
        __syncthreads(); // every thread has read s_word before thread 0 rewrites it
    }
    // The phase is over: every block left the loop at the same round, after
    // the grid barrier that ended the last relaxation, so D is final.  The
    // call's epilogue runs here instead of in two more launches: the tree
    // nodes go to the caller's arrays, and the round stamp moves past every
    // id this call used.
    if (a.dist || a.parent) {
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < a.g.V; v += stride) {
            const unsigned long long d = __ldcg(&a.D[v]);
            if (a.dist)
                a.dist[v] = node_dist(d);
            if (a.parent)
                a.parent[v] = node_parent(d);
        }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        a.ctr[kRoundsDone] = r;
        a.ctr[kRid] += r + 2;
        if (kNF)
            a.ctr[kPhase] = phase0 + splits;
        atomicAdd(&a.g.st->ctr[kCtrRounds][0], (unsigned long long)r);
        atomicAdd(&a.g.st->ctr[kCtrGridBarriers][0], (unsigned long long)bars);
        if (a.dist || a.parent)
            atomicAdd(&a.g.st->ctr[kCtrUnpacked][0], (unsigned long long)a.g.V);
        if (!ok || r >= a.max_rounds || ld_volatile(a.ctr + kOverflow) != 0)
            set_status(a.g.st, kErrTimeout);
    }
}

// One round, for the host-driven fallback.
__global__ void __launch_bounds__(256) k_round_once(RoundArgs a, uint32_t r, uint32_t n)
{
    __shared__ BlockFrontier bq;
    bq_init(bq);
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    round_step(a, a.ctr + kCnt0, r, n, warp0, nwarps, __ldg(a.ctr + kRid), bq);
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
    if ((i & ~31u) >= n)
        return;
    bool hit = false;
    uint32_t v = 0;
    if (i < n) {
        const unsigned long long e = dlog[i];
        const uint32_t u = (uint32_t)(e >> 32);
        v = (uint32_t)e;
        const unsigned long long dv = __ldcg(&a.D[v]);
        hit = v != a.source && dv != kInfNode && node_parent(dv) == u && atomicCAS(&a.D[v], dv, kInfNode) == dv;
    }
    if (hit)
        atomicOr(&a.inv[v >> 5], 1u << (v & 31));
    const uint32_t m = __ballot_sync(kFull, hit);
    if (m && lane_id() == 0)
        a.ctr[kInvTotal] = 1; // a flag: something was invalidated
    count_add(a.g.st, kCtrInvalidated, __popc(m));
}

// The invalidation spreads to every tree descendant of the seeds: a vertex
// is invalid iff the path from it up the shortest-path tree reaches a seed
// before the source.  As in the paper, each reached vertex walks its tree
// parents up until it meets the source (valid) or a vertex without a tree
// node (invalid: a seed, or a vertex this pass has already invalidated);
// invalid vertices get <INF, INVALID> at once, so later walks through them
// stop there.  Tree parents have strictly smaller distances (weights are
// >= 1), so every walk ends.  The loads are plain (L1-cacheable): the upper
// part of the tree, where most walks pass, stays in L1, and a stale line can
// only hide an invalidation made by this pass, whose walk went on up the
// same parents to the same seed, so the outcome is the same.  The
// invalidated vertices of one warp set their bits with one atomicOr (32
// consecutive vertices share a bitmap word).
__global__ void k_inv_walk(RoundArgs a)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if ((v & ~31u) >= a.g.V)
        return;
    count_add(a.g.st, kCtrWalkVertices, __popc(__ballot_sync(kFull, v < a.g.V)));
    bool bad = false;
    const unsigned long long dv = v < a.g.V && v != a.source ? a.D[v] : kInfNode;
    if (dv != kInfNode) {
        // only parents are read: a tree node's parent word is kNil exactly
        // when the node is <INF, INVALID> (every finite node names a
        // vertex), so one 4-byte load and one compare decide a hop; four
        // hops an iteration, the bound checked once per four
        const uint32_t *par = reinterpret_cast<const uint32_t *>(a.D); // low word of node x: par[2x]
        uint32_t x = node_parent(dv), hops = 0;
        while (x != a.source) {
            uint32_t p = par[2 * (uint64_t)x];
            if (p == kNil) {
                bad = true;
                break;
            }
            if (p == a.source)
                break;
            p = par[2 * (uint64_t)p];
            if (p == kNil) {
                bad = true;
                break;
            }
            if (p == a.source)
                break;
            p = par[2 * (uint64_t)p];
            if (p == kNil) {
                bad = true;
                break;
            }
            if (p == a.source)
                break;
            p = par[2 * (uint64_t)p];
            if (p == kNil) {
                bad = true;
                break;
            }
            x = p;
            if ((hops += 4) > a.max_rounds) { // parent pointers not a tree: corrupted state
                set_status(a.g.st, kErrTimeout);
                break;
            }
        }
    }
    if (bad)
        a.D[v] = kInfNode;
    const uint32_t mask = __ballot_sync(kFull, bad);
    if (lane_id() == 0 && mask) {
        atomicOr(&a.inv[v >> 5], mask);
        a.ctr[kInvTotal] = 1;
        count_add(a.g.st, kCtrInvalidated, __popc(mask));
    }
}

// After invalidation: relax every edge out of a valid vertex into a vertex
// invalidated by this call.  The target test reads the invalidation bitmap,
// which stays fixed during the pass, so every such edge is relaxed even after
// another in-neighbour has already given its target a finite distance; does
// nothing if nothing was invalidated.  A streaming scan over the whole slab
// array (scan_slab_chunks: 32-slab chunks, of which only the slabs whose
// source has a finite distance are staged in shared memory by bulk copies;
// the owners' tree nodes are gathered two chunks ahead); each kept slab is
// relaxed by one lane.  Only
// distances change here (64-bit atomic minima whose results are not needed);
// the improved targets are enqueued by k_enqueue_invalid.
__global__ void __launch_bounds__(kScanWarps * 32) k_relax_into_invalid_slabs(RoundArgs a)
{
    __shared__ ScanSmem sm;
    const GView &g = a.g;
    if (__ldg(a.ctr + kInvTotal) == 0) // set by the kernels before this one
        return;
    const uint32_t lane = lane_id();
    // per-lane tallies, summed over the warp once at the end
    uint32_t slabs = 0, edges = 0, owners = 0, targets = 0;
    const bool ok = scan_slab_chunks(
        g, sm,
        [&](uint32_t own) {
            owners += own != kNil;
            return own != kNil ? node_dist(__ldcg(&a.D[own])) : kInf32;
        },
        [](uint32_t dx) { return dx != kInf32; }, // slabs of unreached or invalidated sources are not read
        [&](const uint4 *buf, const uint8_t *comp, uint32_t n, uint32_t own_l, uint32_t dx_l) {
            // lane j takes the chunk's j-th slab in use whole: first the
            // bitmap words of all its 15 destinations (loads in flight
            // together), keeping the keys in registers and the live pairs
            // as bits of a mask; then the bit tests, reading a weight from
            // shared memory only for a relaxed edge.  The slab's 16-byte
            // parts are read in a lane-rotated order, so the eight lanes of
            // each shared-memory phase hit distinct banks.
            const bool active = lane < n; // every kept slab's source has a finite distance
            const uint32_t it = active ? comp[lane] : 0u;
            const uint32_t own = __shfl_sync(kFull, own_l, it);
            const uint32_t dx = __shfl_sync(kFull, dx_l, it);
            slabs += active;
            if (!__any_sync(kFull, active))
                return;
            const uint32_t *mine = reinterpret_cast<const uint32_t *>(buf + (active ? lane : 0) * 8);
            uint32_t key[16], word[16];
            uint32_t live = 0; // bit k: pair k of the rotated order is a live edge
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t qq = (q + lane) & 7u;
                const uint4 v = reinterpret_cast<const uint4 *>(mine)[qq];
                const bool l0 = active && v.x < kTombKey, l1 = active && qq != 7u && v.z < kTombKey;
                key[2 * q] = v.x;
                key[2 * q + 1] = v.z;
                live |= (l0 ? 1u : 0u) << (2 * q) | (l1 ? 1u : 0u) << (2 * q + 1);
                word[2 * q] = l0 ? __ldg(&a.inv[v.x >> 5]) : 0u; // the bitmap is fixed during the pass
                word[2 * q + 1] = l1 ? __ldg(&a.inv[v.z >> 5]) : 0u;
            }
            uint32_t hit = 0; // bit k: pair k's destination is invalidated
#pragma unroll
            for (int k = 0; k < 16; ++k)
                hit |= ((word[k] >> (key[k] & 31u)) & 1u) << k;
            hit &= live;
            edges += __popc(live);
            targets += __popc(hit);
            while (hit) {
                const int k = __ffs(hit) - 1;
                hit &= hit - 1;
                // pair k sits in part (k/2 + lane) % 8, word 2 * (k & 1), weight next to it
                const uint32_t at = (((uint32_t)(k >> 1) + lane) & 7u) * 4 + 2 * (k & 1);
                const unsigned long long nd = (unsigned long long)dx + (a.unit ? 1u : mine[at + 1]);
                if (nd < kInf32)
                    atomicMin(&a.D[mine[at]], (nd << 32) | own);
            }
        });
    if (!ok)
        set_status(g.st, kErrTimeout);
    count_add(g.st, kCtrScanOwners, __reduce_add_sync(kFull, owners));
    count_add(g.st, kCtrScanSlabs, __reduce_add_sync(kFull, slabs));
    count_add(g.st, kCtrScanEdges, __reduce_add_sync(kFull, edges));
    count_add(g.st, kCtrScanTargets, __reduce_add_sync(kFull, targets));
}

// Enqueues the lists of every vertex invalidated by this call that the pass
// above gave a finite distance (one warp per 32-vertex word of the bitmap),
// stamped with the prologue's round so that the incremental prologue does
// not enqueue it again.  The frontier slots of vertices with few lists are
// reserved with one atomicAdd per block (a warp-level reservation would put
// one atomic per 32 vertices on the single frontier counter); a vertex with
// many lists is written by its whole warp.
__global__ void __launch_bounds__(256) k_enqueue_invalid(RoundArgs a)
{
    constexpr uint32_t kSmall = 8;
    __shared__ uint32_t s_total, s_base;
    const uint32_t lane = lane_id();
    const uint64_t word = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    if (threadIdx.x == 0)
        s_total = 0;
    __syncthreads();
    bool pred = false;
    uint2 vi = make_uint2(0, 0);
    const uint32_t y = (uint32_t)word * 32 + lane;
    if (word < ((uint64_t)a.g.V + 31) / 32 && __ldg(a.ctr + kInvTotal) != 0) {
        const uint32_t bits = __ldcg(&a.inv[word]);
        pred = (bits >> lane) & 1u;
        if (pred) {
            pred = __ldcg(&a.D[y]) != kInfNode;
            if (pred) {
                vi = a.g.vinfo[y];
                a.stamp[y] = __ldg(a.ctr + kRid) + 1;
            }
        }
    }
    count_add(a.g.st, kCtrScanImproved, __popc(__ballot_sync(kFull, pred)));
    // small vertices: warp scan of bucket counts, then a block reservation
    const bool small = pred && vi.y <= kSmall;
    const uint32_t c = small ? vi.y : 0;
    uint32_t incl = c;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o)
            incl += t;
    }
    const uint32_t wtotal = __shfl_sync(kFull, incl, 31);
    uint32_t woff = 0;
    if (lane == 0 && wtotal)
        woff = atomicAdd(&s_total, wtotal);
    __syncthreads();
    if (threadIdx.x == 0 && s_total)
        s_base = atomicAdd(a.ctr + kCnt0, s_total);
    __syncthreads();
    int *overflow = (int *)(a.ctr + kOverflow);
    if (wtotal) {
        const uint32_t at = s_base + __shfl_sync(kFull, woff, 0) + incl - c;
        for (uint32_t k = 0; k < c; ++k) {
            if (at + k < a.cap)
                a.front[0][at + k] = make_uint2(vi.x + k, y);
            else
                *overflow = 1;
        }
    }
    // large vertices: one at a time, written by the whole warp
    uint32_t big = __ballot_sync(kFull, pred && !small);
    while (big) {
        const uint32_t l = __ffs(big) - 1;
        big &= big - 1;
        const uint32_t first = __shfl_sync(kFull, vi.x, l), nb = __shfl_sync(kFull, vi.y, l);
        const uint32_t yl = __shfl_sync(kFull, y, l);
        uint32_t base = 0;
        if (lane == 0)
            base = atomicAdd(a.ctr + kCnt0, nb);
        base = __shfl_sync(kFull, base, 0);
        for (uint32_t k = lane; k < nb; k += 32) {
            if (base + k < a.cap)
                a.front[0][base + k] = make_uint2(first + k, yl);
            else
                *overflow = 1;
        }
    }
}


// Incremental seeds: relax the entries inserted since the last commit.
// Every list in the updated-list log is walked from its UpdateIterator start
// (the marker slab, skipping its lanes before the marker lane, or all of it
// when it is full).  Every 4-lane group of every warp takes one list at a
// time (group index + k * groups in the grid; eight lists per warp in
// flight); the next list's log entry, source and marker are loaded a step
// ahead.
__global__ void __launch_bounds__(256, 5) k_relax_updated(RoundArgs a)
{
    const GView &g = a.g;
    const uint32_t s4 = lane_id() & 3u, g4 = lane_id() >> 2;
    const uint32_t n = min(__ldg(&g.st->ulog_count), g.H);
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t gs = (((uint64_t)gridDim.x * blockDim.x) >> 5) * 8; // 4-lane groups in the grid
    __shared__ BlockFrontier bq;
    bq_init(bq);
    const uint32_t round = __ldg(a.ctr + kRid) + 1;
    int *overflow = (int *)(a.ctr + kOverflow);
    unsigned long long lists = 0, slabs = 0, edges = 0, improved = 0;
    uint64_t i = warp0 * 8 + g4;
    uint32_t L = i < n ? g.ulog[i] : kNil;
    uint32_t nL = i + gs < n ? g.ulog[i + gs] : kNil;
    uint32_t src = L != kNil ? g.list_src[L] : 0;
    unsigned long long mk = L != kNil ? g.lmark[L] : 0;
    for (uint64_t base = warp0 * 8; base < n; base += gs, i += gs) {
        const uint32_t nnL = i + 2 * gs < n ? g.ulog[i + 2 * gs] : kNil;
        const uint32_t nsrc = nL != kNil ? g.list_src[nL] : 0;
        const unsigned long long nmk = nL != kNil ? g.lmark[nL] : 0;
        const uint32_t dx = L != kNil ? node_dist(__ldcg(&a.D[src])) : kInf32;
        const uint32_t mlane = (uint32_t)(mk & 0xFF);
        const uint32_t first_lane = mlane == kInvalidLane ? 32u : mlane;
        const bool go = L != kNil && dx != kInf32;
        const uint32_t start = go ? (uint32_t)(mk >> 32) : kNil;
        uint4 lo, hi;
        group4_load(g, start, lo, hi);
        lists += __popc(__ballot_sync(kFull, go && s4 == 0));
        const uint32_t x = src;
        slabs += walk_lists_g4_from(g, start, true, lo, hi, first_lane, a.max_hops,
                                    [&](const uint32_t(&y)[4], const uint32_t(&w)[4], const bool(&live)[4]) {
                                        relax_edges4(a, x, dx, y, w, live, round, bq, a.front[0], a.ctr + kCnt0,
                                                     overflow, edges, improved);
                                    });
        L = nL;
        nL = nnL;
        src = nsrc;
        mk = nmk;
    }
    bq_flush(bq, a.front[0], a.ctr + kCnt0, a.cap, overflow);
    count_add(g.st, kCtrSeedLists, lists);
    count_add(g.st, kCtrSeedSlabs, slabs);
    count_add(g.st, kCtrSeedEdges, edges);
    count_add(g.st, kCtrSeedImproved, improved);
}

// Incremental seeds from the inserted-edge log (the paper's incremental
// frontier is the batch's inserted edges), used when the epoch holds no
// deletes, so every logged edge is still live with its stored weight: each
// lane takes four consecutive log entries <src, dst, w> and relaxes them
// together, as relax_edges4 does a slab's four pairs (the sources' tree
// nodes, the targets' tree nodes, the atomic minima of the candidates that
// beat them, then the improved targets' vertex index entries and round
// stamps), and enqueues the lists of each vertex it lowered first in this
// round.  Two dependent gathers per edge instead of the walk's five loads
// per updated list (log entry, list source, marker, source node, slab).
__global__ void __launch_bounds__(256) k_relax_inserted(RoundArgs a, const uint4 *__restrict__ ilog, uint32_t cap)
{
    __shared__ BlockFrontier bq;
    bq_init(bq);
    const uint32_t n = min(__ldg(&a.g.st->ilog_count), cap);
    const uint32_t round = __ldg(a.ctr + kRid) + 1;
    int *overflow = (int *)(a.ctr + kOverflow);
    unsigned long long entries = 0, edges = 0, improved = 0;
    const uint64_t lane4 = (uint64_t)lane_id() * 4;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x * 4;
    for (uint64_t wb = ((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) & ~31ull) * 4; wb < n; wb += stride) {
        uint32_t x[4], y[4], nd[4];
        bool up[4];
        unsigned long long cur[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const uint64_t i = wb + lane4 + k;
            const uint4 e = i < n ? __ldcs(&ilog[i]) : make_uint4(0, 0, 0, 0);
            x[k] = e.x;
            y[k] = e.y;
            nd[k] = e.z;
            up[k] = i < n;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            entries += __popc(__ballot_sync(kFull, up[k]));
            const uint32_t dx = up[k] ? node_dist(__ldcg(&a.D[x[k]])) : kInf32;
            const unsigned long long d = (unsigned long long)dx + (a.unit ? 1u : nd[k]);
            up[k] = up[k] && dx != kInf32 && d < kInf32;
            nd[k] = (uint32_t)d;
        }
        auto cand = [&](int k) { return ((unsigned long long)nd[k] << 32) | x[k]; };
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            edges += __popc(__ballot_sync(kFull, up[k]));
            cur[k] = up[k] ? __ldcg(&a.D[y[k]]) : 0ull;
        }
#pragma unroll
        for (int k = 0; k < 4; ++k)
            if (up[k] && cand(k) < cur[k])
                cur[k] = atomicMin(&a.D[y[k]], cand(k));
            else
                up[k] = false;
        uint2 vi[4];
        uint32_t st[4];
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            up[k] = up[k] && cand(k) < cur[k];
            vi[k] = make_uint2(0, 0);
            st[k] = round;
            if (up[k]) {
                vi[k] = a.g.vinfo[y[k]];
                st[k] = atomicExch(&a.stamp[y[k]], round);
            }
        }
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            up[k] = up[k] && st[k] != round;
            improved += __popc(__ballot_sync(kFull, up[k]));
            enqueue_lists_block(bq, y[k], up[k], vi[k], a.front[0], a.ctr + kCnt0, a.cap, overflow);
        }
    }
    bq_flush(bq, a.front[0], a.ctr + kCnt0, a.cap, overflow);
    count_add(a.g.st, kCtrSeedLog, entries);
    count_add(a.g.st, kCtrSeedEdges, edges);
    count_add(a.g.st, kCtrSeedImproved, improved);
}

// Ends a call of the host-driven fallback (the round kernel does this
// itself): advances the round stamp past every id used (`rounds` rounds),
// reports an overflowed frontier.
__global__ void k_sssp_finish(uint32_t *ctr, DevState *st, uint32_t rounds)
{
    ctr[kRoundsDone] = rounds;
    ctr[kRid] += rounds + 2;
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

// ------------------------------------------------- several states, one pass
//
// mk_incr_multi advances up to kMaxMulti BFS/SSSP states of one graph
// together: the passes that read the graph's change log or its whole slab
// array (the incremental prologue over the updated lists, the decremental
// relax-into-invalid scan) and the round loop run once for all of them, each
// slab or list read once and relaxed into every state, the rounds of all
// states sharing one grid barrier per round.

constexpr uint32_t kMaxMulti = 4;

struct MultiArgs {
    RoundArgs c[kMaxMulti];
    uint32_t k; // states in use
};

// The incremental prologue (k_relax_updated) for every state at once: each
// logged list is walked once from its UpdateIterator start and every slab's
// new edges are relaxed into each state whose copy of the list's source has
// a finite distance.  Dynamic shared memory: one BlockFrontier per state.
__global__ void __launch_bounds__(256, 5) k_relax_updated_multi(MultiArgs m)
{
    extern __shared__ unsigned char multi_smem[];
    BlockFrontier *bqs = reinterpret_cast<BlockFrontier *>(multi_smem);
    const GView &g = m.c[0].g;
    const uint32_t s4 = lane_id() & 3u, g4 = lane_id() >> 2;
    const uint32_t n = min(__ldg(&g.st->ulog_count), g.H);
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t gs = (((uint64_t)gridDim.x * blockDim.x) >> 5) * 8;
    for (uint32_t j = 0; j < m.k; ++j)
        if (threadIdx.x == 0)
            bqs[j].count = 0;
    __syncthreads();
    uint32_t round[kMaxMulti];
#pragma unroll
    for (uint32_t j = 0; j < kMaxMulti; ++j)
        round[j] = j < m.k ? __ldg(m.c[j].ctr + kRid) + 1 : 0u;
    unsigned long long lists = 0, slabs = 0, edges = 0, improved = 0;
    uint64_t i = warp0 * 8 + g4;
    uint32_t L = i < n ? g.ulog[i] : kNil;
    uint32_t nL = i + gs < n ? g.ulog[i + gs] : kNil;
    uint32_t src = L != kNil ? g.list_src[L] : 0;
    unsigned long long mk = L != kNil ? g.lmark[L] : 0;
    for (uint64_t base = warp0 * 8; base < n; base += gs, i += gs) {
        const uint32_t nnL = i + 2 * gs < n ? g.ulog[i + 2 * gs] : kNil;
        const uint32_t nsrc = nL != kNil ? g.list_src[nL] : 0;
        const unsigned long long nmk = nL != kNil ? g.lmark[nL] : 0;
        uint32_t dx[kMaxMulti];
        bool any = false;
#pragma unroll
        for (uint32_t j = 0; j < kMaxMulti; ++j) {
            dx[j] = (j < m.k && L != kNil) ? node_dist(__ldcg(&m.c[j].D[src])) : kInf32;
            any |= dx[j] != kInf32;
        }
        const uint32_t mlane = (uint32_t)(mk & 0xFF);
        const uint32_t first_lane = mlane == kInvalidLane ? 32u : mlane;
        const bool go = L != kNil && any;
        const uint32_t start = go ? (uint32_t)(mk >> 32) : kNil;
        uint4 lo, hi;
        group4_load(g, start, lo, hi);
        lists += __popc(__ballot_sync(kFull, go && s4 == 0));
        const uint32_t x = src;
        slabs += walk_lists_g4_from(g, start, true, lo, hi, first_lane, m.c[0].max_hops,
                                    [&](const uint32_t(&y)[4], const uint32_t(&w)[4], const bool(&live)[4]) {
                                        for (uint32_t j = 0; j < m.k; ++j) {
                                            const RoundArgs &a = m.c[j];
                                            relax_edges4(a, x, dx[j], y, w, live, round[j], bqs[j], a.front[0],
                                                         a.ctr + kCnt0, (int *)(a.ctr + kOverflow), edges,
                                                         improved);
                                        }
                                    });
        L = nL;
        nL = nnL;
        src = nsrc;
        mk = nmk;
    }
    for (uint32_t j = 0; j < m.k; ++j)
        bq_flush(bqs[j], m.c[j].front[0], m.c[j].ctr + kCnt0, m.c[j].cap, (int *)(m.c[j].ctr + kOverflow));
    count_add(g.st, kCtrSeedLists, lists);
    count_add(g.st, kCtrSeedSlabs, slabs);
    count_add(g.st, kCtrSeedEdges, edges);
    count_add(g.st, kCtrSeedImproved, improved);
}

// The decremental relax-into-invalid scan (k_relax_into_invalid_slabs) for
// every state at once: a slab is staged when its source has a finite
// distance in any state that invalidated something, and its live pairs are
// then tested against each such state's invalidation bitmap.
__global__ void __launch_bounds__(kScanWarps * 32) k_relax_into_invalid_multi(MultiArgs m)
{
    __shared__ ScanSmem sm;
    const GView &g = m.c[0].g;
    bool act[kMaxMulti];
    bool any_act = false;
#pragma unroll
    for (uint32_t j = 0; j < kMaxMulti; ++j) {
        act[j] = j < m.k && __ldg(m.c[j].ctr + kInvTotal) != 0;
        any_act |= act[j];
    }
    if (!any_act)
        return;
    const uint32_t lane = lane_id();
    uint32_t slabs = 0, edges = 0, owners = 0, targets = 0;
    const bool ok = scan_slab_chunks(
        g, sm,
        [&](uint32_t own) {
            owners += own != kNil;
            uint4 dx = make_uint4(kInf32, kInf32, kInf32, kInf32);
            if (own != kNil) {
                dx.x = act[0] ? node_dist(__ldcg(&m.c[0].D[own])) : kInf32;
                dx.y = act[1] ? node_dist(__ldcg(&m.c[1].D[own])) : kInf32;
                dx.z = act[2] ? node_dist(__ldcg(&m.c[2].D[own])) : kInf32;
                dx.w = act[3] ? node_dist(__ldcg(&m.c[3].D[own])) : kInf32;
            }
            return dx;
        },
        [](const uint4 &dx) { return dx.x != kInf32 || dx.y != kInf32 || dx.z != kInf32 || dx.w != kInf32; },
        [&](const uint4 *buf, const uint8_t *comp, uint32_t n, uint32_t own_l, const uint4 &dx_l) {
            const bool active = lane < n;
            const uint32_t it = active ? comp[lane] : 0u;
            const uint32_t own = __shfl_sync(kFull, own_l, it);
            const uint32_t dxs[kMaxMulti] = {__shfl_sync(kFull, dx_l.x, it), __shfl_sync(kFull, dx_l.y, it),
                                             __shfl_sync(kFull, dx_l.z, it), __shfl_sync(kFull, dx_l.w, it)};
            slabs += active;
            if (!__any_sync(kFull, active))
                return;
            const uint32_t *mine = reinterpret_cast<const uint32_t *>(buf + (active ? lane : 0) * 8);
            uint32_t key[16];
            uint32_t live = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                const uint32_t qq = (q + lane) & 7u;
                const uint4 v = reinterpret_cast<const uint4 *>(mine)[qq];
                const bool l0 = active && v.x < kTombKey, l1 = active && qq != 7u && v.z < kTombKey;
                key[2 * q] = v.x;
                key[2 * q + 1] = v.z;
                live |= (l0 ? 1u : 0u) << (2 * q) | (l1 ? 1u : 0u) << (2 * q + 1);
            }
            edges += __popc(live);
            for (uint32_t j = 0; j < m.k; ++j) {
                const RoundArgs &a = m.c[j];
                const uint32_t dx = dxs[j];
                const uint32_t lj = dx != kInf32 ? live : 0u;
                if (!__any_sync(kFull, lj != 0))
                    continue;
                uint32_t word[16];
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    word[k] = ((lj >> k) & 1u) ? __ldg(&a.inv[key[k] >> 5]) : 0u;
                uint32_t hit = 0;
#pragma unroll
                for (int k = 0; k < 16; ++k)
                    hit |= ((word[k] >> (key[k] & 31u)) & 1u) << k;
                hit &= lj;
                targets += __popc(hit);
                while (hit) {
                    const int k = __ffs(hit) - 1;
                    hit &= hit - 1;
                    const uint32_t at = (((uint32_t)(k >> 1) + lane) & 7u) * 4 + 2 * (k & 1);
                    const unsigned long long nd = (unsigned long long)dx + (a.unit ? 1u : mine[at + 1]);
                    if (nd < kInf32)
                        atomicMin(&a.D[mine[at]], (nd << 32) | own);
                }
            }
        });
    if (!ok)
        set_status(g.st, kErrTimeout);
    count_add(g.st, kCtrScanOwners, __reduce_add_sync(kFull, owners));
    count_add(g.st, kCtrScanSlabs, __reduce_add_sync(kFull, slabs));
    count_add(g.st, kCtrScanEdges, __reduce_add_sync(kFull, edges));
    count_add(g.st, kCtrScanTargets, __reduce_add_sync(kFull, targets));
}

// The round loop of every state in one cooperative launch: in round r each
// state with a non-empty frontier is relaxed over the whole grid (one state
// after another), then one grid barrier ends the round for all of them; the
// loop ends when every frontier is empty.  Block 0 clears each state's
// counter for round r + 2 every round, so a state whose frontier emptied
// keeps reading zero.  No solo phase: rounds of a few lists cost a grid
// barrier each.  Then every state's epilogue (dist/parent, round stamp).
// Dynamic shared memory: one BlockFrontier per state.
__global__ void __launch_bounds__(kRoundsMaxThreads, 1) k_rounds_multi(MultiArgs m)
{
    extern __shared__ unsigned char multi_smem[];
    BlockFrontier *bqs = reinterpret_cast<BlockFrontier *>(multi_smem);
    __shared__ uint32_t s_n[kMaxMulti];
    for (uint32_t j = 0; j < m.k; ++j)
        if (threadIdx.x == 0)
            bqs[j].count = 0;
    __syncthreads();
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const RoundArgs &a0 = m.c[0];
    uint32_t r = 0, bars = 0, passed = 0;
    bool ok = true;
    while (r < a0.max_rounds) {
        if (threadIdx.x == 0)
            for (uint32_t j = 0; j < m.k; ++j)
                s_n[j] = min(ld_volatile(m.c[j].ctr + kCnt0 + r % 3), m.c[j].cap);
        __syncthreads();
        uint32_t total = 0;
        for (uint32_t j = 0; j < m.k; ++j)
            total += s_n[j];
        if (total == 0)
            break;
        if (blockIdx.x == 0 && threadIdx.x == 0)
            for (uint32_t j = 0; j < m.k; ++j)
                m.c[j].ctr[kCnt0 + (r + 2) % 3] = 0;
        for (uint32_t j = 0; j < m.k; ++j) {
            const uint32_t n = s_n[j];
            if (n == 0)
                continue;
            const RoundArgs &a = m.c[j];
            const uint32_t in = r & 1;
            uint32_t *cnt = a.ctr + kCnt0 + (r + 1) % 3;
            relax_body(a, a.front[in], n, a.front[in ^ 1], cnt, __ldg(a.ctr + kRid) + 2 + r, warp0, nwarps, bqs[j]);
            bq_flush(bqs[j], a.front[in ^ 1], cnt, a.cap, (int *)(a.ctr + kOverflow));
        }
        ++bars;
        if (!grid_barrier(a0.ctr + kBar, passed, a0.barrier_spins)) {
            ok = false;
            break;
        }
        ++r;
    }
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint32_t j = 0; j < m.k; ++j) {
        const RoundArgs &a = m.c[j];
        if (a.dist || a.parent)
            for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < a.g.V; v += stride) {
                const unsigned long long d = __ldcg(&a.D[v]);
                if (a.dist)
                    a.dist[v] = node_dist(d);
                if (a.parent)
                    a.parent[v] = node_parent(d);
            }
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        bool bad = !ok || r >= a0.max_rounds;
        for (uint32_t j = 0; j < m.k; ++j) {
            const RoundArgs &a = m.c[j];
            a.ctr[kRoundsDone] = r;
            a.ctr[kRid] += r + 2;
            if (a.dist || a.parent)
                atomicAdd(&a.g.st->ctr[kCtrUnpacked][0], (unsigned long long)a.g.V);
            bad |= ld_volatile(a.ctr + kOverflow) != 0;
        }
        atomicAdd(&a0.g.st->ctr[kCtrRounds][0], (unsigned long long)r);
        atomicAdd(&a0.g.st->ctr[kCtrGridBarriers][0], (unsigned long long)bars);
        if (bad)
            set_status(a0.g.st, kErrTimeout);
    }
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
    // frontier slots hold <kNil, ...> until written, so a slot read before
    // it is written names no list
    if (st == MK_OK && (cudaMemset(c->front[0], 0xFF, H * 8) != cudaSuccess ||
                        cudaMemset(c->front[1], 0xFF, H * 8) != cudaSuccess))
        st = MK_ERR_CUDA;
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
        device_free(g, c->front[0], H * 8);
        device_free(g, c->front[1], H * 8);
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

} // namespace

namespace mk {

// The persistent round kernel runs one block per SM; the tuned value
// (rounds_blocks_per_sm) is the block size in units of 256 threads, at most
// what fits an SM (the occupancy of 256-thread blocks).  One block per SM
// keeps the grid barrier to one arrival per SM and gives the solo rounds
// the whole SM.
int rounds_max_blocks_per_sm()
{
    static int per = 0;
    if (!per) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, k_rounds<false>, 256, 0);
        per = std::min(std::max(per, 1), (int)(kRoundsMaxThreads / 256));
    }
    return per;
}

int rounds_grid(int) { return num_sms(); }

int rounds_block(int units)
{
    const int max_units = rounds_max_blocks_per_sm();
    return 256 * (units > 0 ? std::min(units, max_units) : max_units);
}

} // namespace mk

namespace {

// Runs every round of one phase and the call's epilogue (round stamp,
// overflow check, a.dist / a.parent written from D).  Input: front[0], size
// in ctr[kCnt0], ctr[kCnt0 + 1] zero.
mk_status run_phase(mk_graph *g, RoundArgs a, const char *name, cudaStream_t s)
{
    const int grid = rounds_grid(g->tune.rounds_blocks_per_sm);
    const int block = rounds_block(g->tune.rounds_blocks_per_sm);
    void *args[] = {&a};
    if (!g->dbg_host_rounds) {
        const mk_status st = timed(g, name, s, 1, [&]() {
            const void *k = a.delta ? (const void *)k_rounds<true> : (const void *)k_rounds<false>;
            return cudaLaunchCooperativeKernel(k, dim3(grid), dim3(block), args, 0, s);
        });
        if (st == MK_OK)
            return MK_OK;
        cudaGetLastError();
    }
    // fallback: one launch per round, the host reads each size
    for (uint32_t r = 0;; ++r) {
        if (r > a.max_rounds)
            return MK_ERR_TIMEOUT;
        MK_CUDA(cudaMemcpyAsync(g->h_pinned, a.ctr + kCnt0 + r % 3, 4, cudaMemcpyDeviceToHost, s));
        MK_CUDA(cudaStreamSynchronize(s));
        const uint32_t n = std::min(g->h_pinned[0], a.cap);
        if (n == 0) {
            return timed(g, "sssp_finish", s, 2, [&]() {
                k_sssp_finish<<<1, 1, 0, s>>>(a.ctr, g->d_state, r);
                if (a.dist || a.parent)
                    k_unpack<<<grid_for(a.g.V, 256), 256, 0, s>>>(a.D, a.g.V, a.dist, a.parent);
                return cudaSuccess;
            });
        }
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
    a.cap = H;
    a.max_hops = g->v.P + 2;
    a.max_rounds = V + 2;
    a.barrier_spins = g->dbg_barrier_spins != ~0ull ? (uint32_t)g->dbg_barrier_spins : kBarrierSpins;
    a.source = source;
    a.unit = kind == kBfs ? 1 : 0;
    a.dist = d_dist;
    a.parent = d_parent;
    const bool incremental = c->epoch == g->epoch;
    // Near-Far ordering for SSSP when a bucket width is set for this kind of
    // call (the host-driven fallback runs plain rounds)
    a.delta = kind == kSssp && !g->dbg_host_rounds ? (incremental ? g->sssp_delta_incr : g->sssp_delta_static) : 0;
    if (a.delta && !c->fstamp) {
        mk_status st = device_alloc(g, (void **)&c->far[0], (size_t)V * 4);
        if (st == MK_OK)
            st = device_alloc(g, (void **)&c->far[1], (size_t)V * 4);
        if (st == MK_OK)
            st = device_alloc(g, (void **)&c->fstamp, (size_t)V * 4);
        if (st == MK_OK && cudaMemsetAsync(c->fstamp, 0, (size_t)V * 4, s) != cudaSuccess)
            st = MK_ERR_CUDA;
        if (st != MK_OK) {
            device_free(g, c->far[0], (size_t)V * 4);
            device_free(g, c->far[1], (size_t)V * 4);
            device_free(g, c->fstamp, (size_t)V * 4);
            c->far[0] = c->far[1] = c->fstamp = nullptr;
            return st;
        }
    }
    a.far[0] = c->far[0];
    a.far[1] = c->far[1];
    a.fstamp = c->fstamp;
    MK_CUDA(cudaMemsetAsync(c->counters, 0, kClearWords * 4, s));
    MK_CUDA(cudaMemsetAsync(c->counters + kBar, 0, 4, s));
    if (a.delta) {
        // empty far piles, their minima and the first frontier's minimum at INF
        MK_CUDA(cudaMemsetAsync(c->counters + kFarCnt0, 0, 8, s));
        MK_CUDA(cudaMemsetAsync(c->counters + kFarMin0, 0xFF, 12, s));
    }
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
            MK_TRY(timed(g, "sssp_invalidate_walk", s, 1, [&]() {
                k_inv_walk<<<grid_for(V, 256), 256, 0, s>>>(a);
                return cudaSuccess;
            }));
            MK_TRY(timed(g, "sssp_relax_into_invalid", s, 1, [&]() {
                static const uint32_t grid = resident_grid(k_relax_into_invalid_slabs, kScanWarps * 32);
                k_relax_into_invalid_slabs<<<grid, kScanWarps * 32, 0, s>>>(a);
                return cudaSuccess;
            }));
            MK_TRY(timed(g, "sssp_enqueue_invalid", s, 1, [&]() {
                k_enqueue_invalid<<<grid_for(((uint64_t)V + 31) / 32 * 32, 256), 256, 0, s>>>(a);
                return cudaSuccess;
            }));
        }
        // incremental prologue: edges inserted since the last commit, from
        // the inserted-edge log when the epoch holds no deletes (every
        // logged edge still live), else by walking the updated lists from
        // their UpdateIterator markers
        if (g->ulog_bound && !g->epoch_has_deletes && g->ilog_ok && g->d_ilog) {
            MK_TRY(timed(g, "sssp_relax_updated", s, 1, [&]() {
                const uint64_t threads = (g->ilog_bound + 3) / 4;
                k_relax_inserted<<<std::min<uint32_t>(grid_for(threads, 256), num_sms() * 8), 256, 0, s>>>(
                    a, g->d_ilog, (uint32_t)g->ilog_cap);
                return cudaSuccess;
            }));
        } else if (g->ulog_bound) {
            MK_TRY(timed(g, "sssp_relax_updated", s, 1, [&]() {
                // one 4-lane group per logged list
                const uint64_t threads = g->ulog_bound * 4;
                k_relax_updated<<<std::min<uint32_t>(grid_for(threads, 256), num_sms() * 10), 256, 0, s>>>(a);
                return cudaSuccess;
            }));
        }
    }
    // common epilogue: rounds until no distance improves, then the outputs
    MK_TRY(run_phase(g, a, "sssp_rounds", s));
    c->epoch = g->epoch;
    c->seq = g->change_seq;
    return MK_OK;
}


// Several BFS/SSSP states of one graph in one call (see k_rounds_multi).
mk_status run_multi(mk_graph *g, const mk_algo_req *reqs, uint32_t n, cudaStream_t s)
{
    MultiArgs m{};
    m.k = n;
    Consumer *cs[kMaxMulti] = {};
    bool incr[kMaxMulti] = {};
    const uint32_t V = g->v.V, H = g->v.H;
    for (uint32_t j = 0; j < n; ++j) {
        const int kind = reqs[j].kind == MK_REQ_BFS ? kBfs : kSssp;
        MK_TRY(get_consumer(g, kind, reqs[j].source, &cs[j]));
        Consumer *c = cs[j];
        RoundArgs &a = m.c[j];
        a.g = g->v;
        a.D = c->D;
        a.front[0] = c->front[0];
        a.front[1] = c->front[1];
        a.ctr = c->counters;
        a.stamp = c->stamp;
        a.inv = c->inv;
        a.cap = H;
        a.max_hops = g->v.P + 2;
        a.max_rounds = V + 2;
        a.barrier_spins = g->dbg_barrier_spins != ~0ull ? (uint32_t)g->dbg_barrier_spins : kBarrierSpins;
        a.source = reqs[j].source;
        a.unit = kind == kBfs ? 1 : 0;
        a.dist = reqs[j].d_dist;
        a.parent = reqs[j].d_parent;
        incr[j] = c->epoch == g->epoch;
        MK_CUDA(cudaMemsetAsync(c->counters, 0, kClearWords * 4, s));
        MK_CUDA(cudaMemsetAsync(c->counters + kBar, 0, 4, s));
    }
    // the states that recompute statically start from their sources
    for (uint32_t j = 0; j < n; ++j)
        if (!incr[j])
            MK_TRY(timed(g, "sssp_init", s, 1, [&]() {
                k_sssp_init<<<grid_for(V, 256), 256, 0, s>>>(cs[j]->D, V, m.c[j].source, cs[j]->front[0],
                                                             cs[j]->counters + kCnt0, g->v.vinfo);
                return cudaSuccess;
            }));
    // decremental prologue: invalidation per state, one scan for all
    MultiArgs dec{};
    MultiArgs inc{};
    for (uint32_t j = 0; j < n; ++j)
        if (incr[j]) {
            if (g->epoch_has_deletes)
                dec.c[dec.k++] = m.c[j];
            if (g->ulog_bound)
                inc.c[inc.k++] = m.c[j];
        }
    for (uint32_t j = 0; j < dec.k; ++j) {
        const RoundArgs &a = dec.c[j];
        MK_CUDA(cudaMemsetAsync(a.inv, 0, (size_t)(V + 31) / 32 * 4, s));
        MK_TRY(timed(g, "sssp_invalidate", s, 1, [&]() {
            k_invalidate<<<grid_for(std::max<uint64_t>(g->dlog_bound, 1), 256), 256, 0, s>>>(g->d_dlog, g->d_state,
                                                                                             a);
            return cudaSuccess;
        }));
        MK_TRY(timed(g, "sssp_invalidate_walk", s, 1, [&]() {
            k_inv_walk<<<grid_for(V, 256), 256, 0, s>>>(a);
            return cudaSuccess;
        }));
    }
    if (dec.k) {
        MK_TRY(timed(g, "sssp_relax_into_invalid", s, 1, [&]() {
            static const uint32_t grid = resident_grid(k_relax_into_invalid_multi, kScanWarps * 32);
            k_relax_into_invalid_multi<<<grid, kScanWarps * 32, 0, s>>>(dec);
            return cudaSuccess;
        }));
        for (uint32_t j = 0; j < dec.k; ++j)
            MK_TRY(timed(g, "sssp_enqueue_invalid", s, 1, [&]() {
                k_enqueue_invalid<<<grid_for(((uint64_t)V + 31) / 32 * 32, 256), 256, 0, s>>>(dec.c[j]);
                return cudaSuccess;
            }));
    }
    // incremental prologue: one walk over the updated lists for all states
    if (inc.k) {
        const size_t smem = inc.k * sizeof(BlockFrontier);
        // (a function attribute of the current device: set on every call)
        MK_CUDA(cudaFuncSetAttribute(k_relax_updated_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)(kMaxMulti * sizeof(BlockFrontier))));
        MK_TRY(timed(g, "sssp_relax_updated", s, 1, [&]() {
            const uint64_t threads = g->ulog_bound * 4;
            k_relax_updated_multi<<<std::min<uint32_t>(grid_for(threads, 256), num_sms() * 10), 256, smem, s>>>(inc);
            return cudaSuccess;
        }));
    }
    // rounds of every state together
    const int grid = rounds_grid(g->tune.rounds_blocks_per_sm);
    const int block = rounds_block(g->tune.rounds_blocks_per_sm);
    const size_t smem = n * sizeof(BlockFrontier);
    MK_CUDA(cudaFuncSetAttribute(k_rounds_multi, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)(kMaxMulti * sizeof(BlockFrontier))));
    void *args[] = {&m};
    mk_status st = MK_ERR_CUDA;
    if (!g->dbg_host_rounds)
        st = timed(g, "sssp_rounds", s, 1, [&]() {
            return cudaLaunchCooperativeKernel((const void *)k_rounds_multi, dim3(grid), dim3(block), args, smem, s);
        });
    if (st != MK_OK) {
        cudaGetLastError();
        // one state at a time (the host-driven loop when the cooperative
        // launch is refused)
        for (uint32_t j = 0; j < n; ++j)
            MK_TRY(run_phase(g, m.c[j], "sssp_rounds", s));
    }
    for (uint32_t j = 0; j < n; ++j) {
        cs[j]->epoch = g->epoch;
        cs[j]->seq = g->change_seq;
    }
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

mk_status mk_incr_multi(mk_graph *g, const mk_algo_req *h_reqs, uint32_t n, void *stream)
{
    if (!g || !h_reqs || n == 0 || n > kMaxMulti)
        return MK_ERR_INVALID_ARG;
    for (uint32_t j = 0; j < n; ++j) {
        if ((h_reqs[j].kind != MK_REQ_SSSP && h_reqs[j].kind != MK_REQ_BFS) || h_reqs[j].source >= g->v.V)
            return MK_ERR_INVALID_ARG;
        for (uint32_t i = 0; i < j; ++i)
            if (h_reqs[i].kind == h_reqs[j].kind && h_reqs[i].source == h_reqs[j].source)
                return MK_ERR_INVALID_ARG; // one state cannot be advanced twice at once
    }
    cudaStream_t s = (cudaStream_t)stream;
    if (n == 1)
        return run_sssp(g, h_reqs[0].kind == MK_REQ_BFS ? kBfs : kSssp, h_reqs[0].source, h_reqs[0].d_dist,
                        h_reqs[0].d_parent, s);
    return run_multi(g, h_reqs, n, s);
}

} // extern "C"
