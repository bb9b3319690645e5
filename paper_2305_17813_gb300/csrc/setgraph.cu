// ConcurrentSet layout (paper, Sec. "Motivation": SlabHash's ConcurrentSet
// beside the ConcurrentMap that the weighted store uses; the paper stores the
// unweighted graphs of BFS and WCC this way).  An unweighted graph whose
// slabs hold 31 destination keys (lanes 0..30) and the next-slab index
// (lane 31): about twice the keys of a map slab's 15 pairs, so the slab
// array, and every traversal that streams it, is about half as large.
//
// The store keeps the map store's conventions: one head slab per bucket of a
// vertex in one allocation located by an exclusive scan of the bucket
// counts, overflow slabs claimed from a bitmap pool, EMPTY and TOMBSTONE
// keys, deleted keys never reused (so free keys exist only in a chain's last
// slab), set semantics with the first occurrence of a repeated pair applied
// (the batch is deduplicated by the map store's staging kernel).  Inserts,
// deletes and queries walk eight chains per warp in 4-lane groups, each
// lane reading 32 bytes of a slab (the whole group one 128-byte slab).  BFS
// (hop counts, with the smallest-id tight parent) and WCC (smallest-id
// labels) run statically: BFS level by level over a frontier of lists, WCC
// as one union-find pass over the slab array.
#include "mk_host.h"
#include "uf.cuh"

#include <algorithm>
#include <cstring>

using namespace mk;

// Kernels of other translation units, launched here unchanged.
__global__ void k_degree(const uint32_t *src, uint64_t n, uint32_t V, uint32_t *deg, int *bad);
__global__ void k_rule(uint32_t *deg, uint32_t V, float per_bucket);
__global__ void k_init_bitmap(uint32_t *bitmap, uint32_t words, uint32_t P);
__global__ void k_fill_buckets(uint32_t *b, uint32_t V, uint32_t nb, const uint32_t *user, int *bad);
__global__ void k_dedup(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                        const uint32_t *__restrict__ w, uint64_t n, uint32_t V, uint32_t *tpos, uint32_t mask,
                        uint32_t *__restrict__ slot, DevState *st);

namespace {

constexpr uint32_t kSetKeys = 31; // key lanes 0..30, lane 31 = next

__device__ __forceinline__ bool is_set_key_lane(uint32_t lane) { return lane < kSetKeys; }

} // namespace

struct mk_set_graph {
    GView v{};                 // V, H, P, pool_words, vinfo, slabs, bitmap, owner, st (the rest unused)
    uint64_t bytes = 0;
    uint64_t cap = 0, table = 0; // staging: batch hash set (table entries) and per-edge slots (cap)
    uint32_t *d_tpos = nullptr, *d_slot = nullptr;
    uint32_t *h_pinned = nullptr;
};

// -------------------------------------------------------------- kernels

__global__ void k_set_init_slabs(uint32_t *slabs, uint64_t count)
{
    const uint64_t words = count * 32;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x)
        slabs[i] = (i & 31) == kNextLane ? kNil : kEmptyKey;
}

// vinfo[v] = {first list, bucket count}; owner[list] = v; owner of every
// pool slab = kNil.
__global__ void k_set_init_lists(const uint64_t *off, const uint32_t *buckets, uint32_t V, uint2 *vinfo,
                                 uint32_t *owner, uint64_t H, uint64_t total)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t v = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; v < V; v += stride) {
        const uint32_t first = (uint32_t)off[v], nb = buckets[v];
        vinfo[v] = make_uint2(first, nb);
        for (uint32_t b = 0; b < nb; ++b)
            owner[first + b] = (uint32_t)v;
    }
    for (uint64_t s = H + blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < total; s += stride)
        owner[s] = kNil;
}

namespace {

// The list that holds (s, d).
__device__ __forceinline__ uint32_t set_list(const GView &g, uint32_t s, uint32_t d)
{
    const uint2 vi = __ldg(&g.vinfo[s]);
    return vi.x + bucket_of(d, vi.y);
}

// Lanes of the calling lane's 4-lane group in a warp-wide ballot.
__device__ __forceinline__ uint32_t set_group_bits(uint32_t ballot) { return (ballot >> (lane_id() & ~3u)) & 0xFu; }

// Lane s4 of a 4-lane group holds words 8*s4 .. 8*s4+7 of a slab as two
// 16-byte vectors; word 31 (the last of lane 3) is the next index.
__device__ __forceinline__ void set_group_load(const GView &g, uint32_t slab, uint4 &lo, uint4 &hi)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(slab_ptr(g, slab) + (lane_id() & 3u) * 8);
    lo = __ldcg(p);
    hi = __ldcg(p + 1);
}

// Index (0..7) of the lane's first key word equal to k, 8 if none.
__device__ __forceinline__ uint32_t set_first_with(const uint4 &lo, const uint4 &hi, uint32_t k)
{
    const bool last = (lane_id() & 3u) == 3u;
    return lo.x == k   ? 0u
           : lo.y == k ? 1u
           : lo.z == k ? 2u
           : lo.w == k ? 3u
           : hi.x == k ? 4u
           : hi.y == k ? 5u
           : hi.z == k ? 6u
           : (!last && hi.w == k) ? 7u
                                  : 8u;
}

// Inserts d into the list of s with one 4-lane group (go == false: the
// group has nothing to do; every group of the warp calls it in lockstep).
// Walks the whole chain (a present key ends the walk), claims the lowest
// free key of the tail with a CAS (a lost CAS re-reads the slab), or links a
// pool slab holding d with a CAS on the tail's next word (the loser frees
// its slab and follows the winner's).  Returns 1 if d was stored, 0 if it
// was present, or a negative device error code, on the group's lanes.
__device__ __forceinline__ int group_set_insert(const GView &g, bool go, uint32_t s, uint32_t d, uint32_t max_hops,
                                                unsigned long long &loads, unsigned long long &linked)
{
    const uint32_t s4 = lane_id() & 3u, gbase = lane_id() & ~3u;
    bool active = go;
    int res = 0;
    uint32_t slab = go ? set_list(g, s, d) : kNil;
    uint4 lo = make_uint4(kFull, kFull, kFull, kFull), hi = lo;
    if (active)
        set_group_load(g, slab, lo, hi);
    const uint32_t guard_max = 4 * max_hops + 64;
    for (uint32_t guard = 0; __any_sync(kFull, active); ++guard) {
        loads += __popc(__ballot_sync(kFull, active && s4 == 0));
        const uint32_t hits = set_group_bits(__ballot_sync(kFull, active && set_first_with(lo, hi, d) < 8u));
        const uint32_t fk = set_first_with(lo, hi, kEmptyKey);
        const uint32_t frees = set_group_bits(__ballot_sync(kFull, active && fk < 8u));
        const uint32_t nxt = __shfl_sync(kFull, hi.w, gbase + 3);
        // the lowest free key of the group's slab
        bool ok = false;
        if (active && !hits && frees && s4 == (uint32_t)(__ffs(frees) - 1))
            ok = atomicCAS(slab_ptr(g, slab) + 8 * s4 + fk, kEmptyKey, d) == kEmptyKey;
        const bool claimed = set_group_bits(__ballot_sync(kFull, ok)) != 0;
        // a full tail with nothing after it: a pool slab holding d
        const bool grow = active && !hits && !frees && nxt == kNil;
        uint32_t ns = kNil;
        if (grow && s4 == 0)
            ns = alloc_slab_one(g, s * 0x9E3779B9u ^ d ^ (guard << 26));
        ns = __shfl_sync(kFull, ns, gbase);
        uint32_t old = kNil;
        if (grow && ns != kNil) {
            const uint4 e = make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kEmptyKey);
            const uint4 wlo = s4 == 0 ? make_uint4(d, kEmptyKey, kEmptyKey, kEmptyKey) : e;
            const uint4 whi = s4 == 3u ? make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kNil) : e;
            uint4 *q = reinterpret_cast<uint4 *>(slab_ptr(g, ns) + s4 * 8);
            __stcg(q, wlo);
            __stcg(q + 1, whi);
            if (s4 == 0)
                g.owner[ns] = s;
            __threadfence();
            if (s4 == 0)
                old = atomicCAS(slab_ptr(g, slab) + kNextLane, kNil, ns);
        }
        old = __shfl_sync(kFull, old, gbase);
        const bool won = grow && ns != kNil && old == kNil;
        linked += __popc(__ballot_sync(kFull, won && s4 == 0));
        if (active) {
            if (hits) {
                active = false; // present already
            } else if (frees) {
                if (claimed) {
                    res = 1;
                    active = false;
                } // else another group took the key: read the slab again
            } else if (nxt != kNil) {
                slab = nxt;
            } else if (ns == kNil) {
                res = kErrPool;
                active = false;
            } else if (won) {
                res = 1;
                active = false;
            } else { // lost the link: give the slab back, follow the winner's
                if (s4 == 0)
                    g.owner[ns] = kNil;
                __threadfence();
                if (s4 == 0)
                    free_slab(g, ns);
                slab = old;
            }
            if (active && guard >= guard_max) {
                res = kErrTimeout;
                active = false;
            }
        }
        if (active)
            set_group_load(g, slab, lo, hi);
    }
    return res;
}

// Deletes d from the list of s with one 4-lane group (layout and lockstep
// as above): the key becomes TOMBSTONE (never reused); the walk stops at the
// key, at the chain's first free key or at its end.  Returns 1 if d was
// removed.
__device__ __forceinline__ int group_set_delete(const GView &g, bool go, uint32_t s, uint32_t d, uint32_t max_hops,
                                                unsigned long long &loads)
{
    const uint32_t s4 = lane_id() & 3u, gbase = lane_id() & ~3u;
    bool active = go;
    int res = 0;
    uint32_t slab = go ? set_list(g, s, d) : kNil;
    uint4 lo = make_uint4(kFull, kFull, kFull, kFull), hi = lo;
    for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
        if (active)
            set_group_load(g, slab, lo, hi);
        loads += __popc(__ballot_sync(kFull, active && s4 == 0));
        const uint32_t hk = set_first_with(lo, hi, d);
        const uint32_t hits = set_group_bits(__ballot_sync(kFull, active && hk < 8u));
        const uint32_t frees = set_group_bits(__ballot_sync(kFull, active && set_first_with(lo, hi, kEmptyKey) < 8u));
        const uint32_t nxt = __shfl_sync(kFull, hi.w, gbase + 3);
        bool ok = false;
        if (active && hits && s4 == (uint32_t)(__ffs(hits) - 1))
            ok = atomicCAS(slab_ptr(g, slab) + 8 * s4 + hk, d, kTombKey) == d;
        const bool removed = set_group_bits(__ballot_sync(kFull, ok)) != 0;
        if (active) {
            if (hits) {
                res = removed ? 1 : 0;
                active = false;
            } else if (frees || nxt == kNil || hop + 1 >= max_hops) {
                active = false;
            } else {
                slab = nxt;
            }
        }
    }
    return res;
}

} // namespace

// One warp per chunk of 32 edges: eight 4-lane groups take the chunk's first
// occurrences eight at a time (edge it * 8 + group in step it), so eight
// chains are walked at once.
__global__ void __launch_bounds__(256) k_set_insert(GView g, const uint32_t *__restrict__ src,
                                                    const uint32_t *__restrict__ dst, uint64_t n,
                                                    const uint32_t *__restrict__ tpos,
                                                    const uint32_t *__restrict__ slot, uint8_t *__restrict__ flags,
                                                    uint32_t max_hops)
{
    const uint32_t lane = lane_id(), gi = lane >> 2;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long loads = 0, linked = 0;
    for (uint64_t q0 = ((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5) * 32; q0 < n; q0 += warps * 32) {
        if (__any_sync(kFull, status_hint(g.st) != 0))
            break;
        const uint64_t i = q0 + lane;
        bool first = false;
        uint32_t s = 0, d = 0;
        if (i < n) {
            const uint32_t sl = slot[i];
            first = sl != kNil && __ldcg(&tpos[sl]) == (uint32_t)i;
            s = src[i];
            d = dst[i];
        }
        uint8_t mine = 0;
#pragma unroll 1
        for (uint32_t it = 0; it < 4; ++it) {
            const uint32_t who = it * 8 + gi;
            const bool go = __shfl_sync(kFull, first, who);
            const int r = group_set_insert(g, go, __shfl_sync(kFull, s, who), __shfl_sync(kFull, d, who), max_hops,
                                           loads, linked);
            if (r < 0 && (lane & 3u) == 0)
                set_status(g.st, r);
            // lane L's edge was taken by group L % 8 in step L / 8
            const int rl = __shfl_sync(kFull, r, (lane & 7u) * 4);
            if (lane / 8 == it)
                mine = rl > 0 ? 1 : 0;
        }
        if (flags && i < n)
            flags[i] = mine;
    }
    count_add(g.st, kCtrInsertSlabs, loads);
    count_add(g.st, kCtrInsertNewSlabs, linked);
}

// Deletes, in the same chunks and groups.
__global__ void __launch_bounds__(256) k_set_delete(GView g, const uint32_t *__restrict__ src,
                                                    const uint32_t *__restrict__ dst, uint64_t n,
                                                    const uint32_t *__restrict__ tpos,
                                                    const uint32_t *__restrict__ slot, uint8_t *__restrict__ flags,
                                                    uint32_t max_hops)
{
    const uint32_t lane = lane_id(), gi = lane >> 2;
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long loads = 0;
    for (uint64_t q0 = ((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5) * 32; q0 < n; q0 += warps * 32) {
        if (__any_sync(kFull, status_hint(g.st) != 0))
            break;
        const uint64_t i = q0 + lane;
        bool first = false;
        uint32_t s = 0, d = 0;
        if (i < n) {
            const uint32_t sl = slot[i];
            first = sl != kNil && __ldcg(&tpos[sl]) == (uint32_t)i;
            s = src[i];
            d = dst[i];
        }
        uint8_t mine = 0;
#pragma unroll 1
        for (uint32_t it = 0; it < 4; ++it) {
            const uint32_t who = it * 8 + gi;
            const bool go = __shfl_sync(kFull, first, who);
            const int r = group_set_delete(g, go, __shfl_sync(kFull, s, who), __shfl_sync(kFull, d, who), max_hops,
                                           loads);
            const int rl = __shfl_sync(kFull, r, (lane & 7u) * 4);
            if (lane / 8 == it)
                mine = rl > 0 ? 1 : 0;
        }
        if (flags && i < n)
            flags[i] = mine;
    }
    count_add(g.st, kCtrDeleteSlabs, loads);
}

// Queries: bit i % 32 of word i / 32 is set when edge i is present.  One
// warp answers 32 consecutive queries: every lane first finds its own
// query's list (32 gathers in flight), then the warp walks eight chains at
// a time, one per 4-lane group, each lane loading 8 consecutive words of
// the slab as two 16-byte vectors (the group's last lane holds the next
// index in its last word).
__global__ void __launch_bounds__(256) k_set_query(GView g, const uint32_t *__restrict__ src,
                                                   const uint32_t *__restrict__ dst, uint64_t n,
                                                   uint32_t *__restrict__ bitmap, uint32_t max_hops)
{
    constexpr uint32_t G = 4, W = 8, kGroups = 8;
    const uint32_t lane = lane_id(), gi = lane / G, sub = lane % G;
    const uint32_t gmask = 0xFu << (gi * G);
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long loads = 0;
    for (uint64_t q0 = ((blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5) * 32; q0 < n; q0 += warps * 32) {
        const uint64_t q = q0 + lane;
        uint32_t my_d = kNil, my_head = kNil;
        bool bad = false;
        if (q < n) {
            const uint32_t s = __ldg(src + q);
            my_d = __ldg(dst + q);
            if (s < g.V && my_d < g.V)
                my_head = set_list(g, s, my_d);
            else
                bad = true;
        }
        if (__ballot_sync(kFull, bad) && lane == 0)
            set_status(g.st, kErrInvalid);
        uint32_t word_bits = 0;
#pragma unroll 1
        for (uint32_t it = 0; it < 32 / kGroups; ++it) {
            const uint32_t who = it * kGroups + gi;
            const uint32_t d = __shfl_sync(kFull, my_d, who);
            uint32_t slab = __shfl_sync(kFull, my_head, who);
            bool active = slab != kNil, found = false;
            for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
                loads += __popc(__ballot_sync(kFull, active && sub == 0));
                uint4 a = make_uint4(kFull, kFull, kFull, kFull), b = a;
                if (active) {
                    const uint4 *v = reinterpret_cast<const uint4 *>(slab_ptr(g, slab) + sub * W);
                    a = __ldg(v);
                    b = __ldg(v + 1);
                }
                const uint32_t w[W] = {a.x, a.y, a.z, a.w, b.x, b.y, b.z, b.w};
                bool hit = false, emp = false;
#pragma unroll
                for (uint32_t k = 0; k < W; ++k)
                    if (sub * W + k < kSetKeys) {
                        hit |= active && w[k] == d;
                        emp |= active && w[k] == kEmptyKey;
                    }
                const uint32_t hm = __ballot_sync(kFull, hit) & gmask;
                const uint32_t em = __ballot_sync(kFull, emp) & gmask;
                const uint32_t nxt = __shfl_sync(kFull, b.w, gi * G + G - 1);
                if (hm)
                    found = true;
                if (active && (hm || em || nxt == kNil || hop >= max_hops))
                    active = false;
                else if (active)
                    slab = nxt;
            }
            const uint32_t fb = __ballot_sync(kFull, sub == 0 && found);
#pragma unroll
            for (uint32_t k = 0; k < kGroups; ++k)
                if (fb & (1u << (k * G)))
                    word_bits |= 1u << (it * kGroups + k);
        }
        if (lane == 0 && q0 < n)
            bitmap[q0 / 32] = word_bits;
    }
    count_add(g.st, kCtrQuerySlabs, loads);
}

// One BFS level over a frontier of lists, one list per 4-lane group (eight
// lists per warp in flight, so a hub's buckets spread over many groups);
// each lane tests the eight keys of its 32 bytes of a slab at once.  A
// destination still unreached gets level + 1 with a CAS and its lists join
// the next frontier: one atomicAdd a warp per slab step for all the new
// vertices of its eight slabs.  The parents come out of the same pass: an
// edge read into a vertex of the next level is tight, so an atomicMin of
// the list's source (its head slab's owner) leaves the smallest one.  The frontier sizes live on the device in
// three rotating counters (this level reads cnt[L % 3], appends to
// cnt[(L + 1) % 3] and clears cnt[(L + 2) % 3], the input of the level
// before), so several levels go out without the host.
__global__ void __launch_bounds__(256) k_set_bfs_level(GView g, const uint32_t *__restrict__ front, uint32_t *next,
                                                       uint32_t *cnt, uint32_t *dist, uint32_t *parent,
                                                       uint32_t level, uint32_t max_hops)
{
    const uint32_t lane = lane_id(), s4 = lane & 3u, gbase = lane & ~3u;
    const uint32_t n = __ldcg(&cnt[level % 3]);
    uint32_t *next_count = &cnt[(level + 1) % 3];
    if (blockIdx.x == 0 && threadIdx.x == 0)
        cnt[(level + 2) % 3] = 0;
    const uint64_t groups = ((uint64_t)gridDim.x * blockDim.x) >> 2;
    const uint64_t g0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 2;
    unsigned long long loads = 0;
    // the warp's eight groups move together: `wb` is its first group's index
    for (uint64_t wb = g0 & ~7ull; wb < n; wb += groups) {
        const uint64_t k = wb + (g0 & 7u);
        uint32_t slab = k < n ? __ldcg(&front[k]) : kNil;
        bool active = slab != kNil;
        const uint32_t u = active ? __ldg(&g.owner[slab]) : 0u; // the list's source, at this level
        for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
            uint4 lo = make_uint4(kFull, kFull, kFull, kFull), hi = lo;
            if (active)
                set_group_load(g, slab, lo, hi);
            loads += __popc(__ballot_sync(kFull, active && s4 == 0));
            const uint32_t wv[8] = {lo.x, lo.y, lo.z, lo.w, hi.x, hi.y, hi.z, hi.w};
            uint32_t cur[8];
            bool key[8];
#pragma unroll
            for (int q = 0; q < 8; ++q) {
                key[q] = active && s4 * 8 + q < kSetKeys && wv[q] < kTombKey;
                cur[q] = key[q] ? __ldcg(&dist[wv[q]]) : 0u;
            }
            uint32_t grab = 0;
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (key[q] && cur[q] == kNil && atomicCAS(&dist[wv[q]], kNil, level + 1) == kNil)
                    grab |= 1u << q;
            // every edge into a vertex of the next level is tight: the
            // smallest such source is the parent (dist only moves from
            // unreached to level + 1 during this launch, so a destination
            // read as unreached is at level + 1 now, whoever took it)
#pragma unroll
            for (int q = 0; q < 8; ++q)
                if (key[q] && (cur[q] == kNil || cur[q] == level + 1))
                    atomicMin(&parent[wv[q]], u);
            const uint32_t nxt = __shfl_sync(kFull, hi.w, gbase + 3);
            if (__any_sync(kFull, grab != 0)) {
                uint2 vi[8];
                uint32_t c = 0;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    vi[q] = (grab >> q) & 1u ? __ldg(&g.vinfo[wv[q]]) : make_uint2(0, 0);
                    c += vi[q].y;
                }
                // exclusive scan of the lanes' list counts, one reservation
                uint32_t incl = c;
#pragma unroll
                for (uint32_t o = 1; o < 32; o <<= 1) {
                    const uint32_t t = __shfl_up_sync(kFull, incl, o);
                    if (lane >= o)
                        incl += t;
                }
                const uint32_t total = __shfl_sync(kFull, incl, 31);
                uint32_t wbase = 0;
                if (lane == 0)
                    wbase = atomicAdd(next_count, total);
                uint32_t off[8];
                uint32_t o = __shfl_sync(kFull, wbase, 0) + incl - c;
                bool big = false;
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    off[q] = o;
                    if (vi[q].y <= 8) {
                        for (uint32_t b = 0; b < vi[q].y; ++b)
                            next[o + b] = vi[q].x + b;
                    } else {
                        big = true;
                    }
                    o += vi[q].y;
                }
                // vertices with many lists: written by the whole warp
                uint32_t bigs = __ballot_sync(kFull, big);
                while (bigs) {
                    const uint32_t j = __ffs(bigs) - 1;
                    bigs &= bigs - 1;
#pragma unroll
                    for (int q = 0; q < 8; ++q) {
                        const uint32_t nj = __shfl_sync(kFull, vi[q].y, j);
                        const uint32_t fj = __shfl_sync(kFull, vi[q].x, j);
                        const uint32_t oj = __shfl_sync(kFull, off[q], j);
                        if (nj > 8)
                            for (uint32_t b = lane; b < nj; b += 32)
                                next[oj + b] = fj + b;
                    }
                }
            }
            if (active) {
                if (nxt == kNil || hop + 1 >= max_hops)
                    active = false;
                else
                    slab = nxt;
            }
        }
    }
    count_add(g.st, kCtrRelaxSlabs, loads);
}

// dist / parent start values; the first frontier is the source's lists.
__global__ void k_set_bfs_init(GView g, uint32_t *dist, uint32_t *parent, uint32_t source, uint32_t *front,
                               uint32_t *cnt)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    const uint2 vi = __ldg(&g.vinfo[source]);
    if (v < g.V) {
        dist[v] = v == source ? 0u : kNil;
        parent[v] = v == source ? source : kNil;
    }
    for (uint32_t i = v; i < vi.y; i += gridDim.x * blockDim.x)
        front[i] = vi.x + i;
    if (v == 0) {
        cnt[0] = vi.y;
        cnt[1] = cnt[2] = 0;
    }
}

namespace {

__device__ __forceinline__ uint32_t set_find(uint32_t *p, uint32_t x)
{
    for (;;) {
        const uint32_t px = __ldcg(&p[x]);
        if (px == x)
            return x;
        const uint32_t ppx = __ldcg(&p[px]);
        if (ppx == px)
            return px;
        p[x] = ppx; // path halving: ppx is an ancestor of x
        x = ppx;
    }
}

} // namespace

__global__ void k_set_uf_init(uint32_t *p, uint32_t V)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V)
        p[v] = v;
}

// Static WCC (Union-Async, the larger root hooked under the smaller, so each
// root is its set's smallest vertex): a warp takes 32 consecutive slabs,
// keeps those in use (owner set) and unites four slabs at a time, one per
// 8-lane group, each lane holding four keys of the slab (one 16-byte load);
// the group's last lane puts the slab's owner in place of the next index,
// so the owner and the slab's 31 destinations are hooked under the
// smallest of their roots in one group union.  The next step's slabs are
// loaded a step ahead.
__global__ void __launch_bounds__(256) k_set_wcc_hook(GView g, uint32_t *p, int *failed)
{
    __shared__ uint8_t comp[8][32];
    const uint32_t lane = lane_id(), g8 = lane >> 3, s8 = lane & 7u, w = threadIdx.x >> 5;
    const uint64_t total = (uint64_t)g.H + g.P;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) * 32;
    const uint4 none = make_uint4(kEmptyKey, kEmptyKey, kEmptyKey, kEmptyKey);
    auto part = [&](uint64_t s) {
        return __ldcg(reinterpret_cast<const uint4 *>(slab_ptr(g, (uint32_t)s)) + s8);
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
            comp[w][__popc(live & lanemask_lt())] = (uint8_t)lane;
        __syncwarp();
        uint32_t it = g8 < n ? comp[w][g8] : 32u;
        uint4 q = it < 32 ? part(c + it) : none;
        for (uint32_t j = g8; j - g8 < n; j += 4) {
            const uint32_t nit = j + 4 < n ? comp[w][j + 4] : 32u;
            const uint4 nq = nit < 32 ? part(c + nit) : none;
            const bool active = it < 32;
            const uint32_t own = __shfl_sync(kFull, own_l, it & 31);
            slabs += __popc(__ballot_sync(kFull, active && s8 == 0));
            const bool last = s8 == 7u;
            const uint32_t e[4] = {q.x, q.y, q.z, last ? own : q.w};
            const bool act[4] = {active && q.x < kTombKey, active && q.y < kTombKey, active && q.z < kTombKey,
                                 last ? active : (active && q.w < kTombKey)};
            edges += __popc(__ballot_sync(kFull, act[0])) + __popc(__ballot_sync(kFull, act[1])) +
                     __popc(__ballot_sync(kFull, act[2])) + __popc(__ballot_sync(kFull, act[3] && !last));
            if (!group_union<8, 4>(p, e, act, 1u << 20) && lane == 0)
                *failed = 1;
            q = nq;
            it = nit;
        }
        __syncwarp();
    }
    count_add(g.st, kCtrWccSlabs, slabs);
    count_add(g.st, kCtrWccEdges, edges);
}

__global__ void k_set_wcc_label(uint32_t *p, uint32_t V, uint32_t *label)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V)
        label[v] = set_find(p, v);
}

__global__ void k_set_flag_status(const int *failed, DevState *st)
{
    if (*failed)
        set_status(st, kErrTimeout);
}

__global__ void k_set_pool_used(const DevState *st, unsigned long long *out)
{
    long long t = 0;
    for (uint32_t i = 0; i < kSlots; ++i)
        t += st->pool_used[i];
    *out = (unsigned long long)t;
}

// ------------------------------------------------------------- host side

namespace {

mk_status set_alloc(mk_set_graph *g, void **p, size_t bytes)
{
    *p = nullptr;
    if (!bytes)
        return MK_OK;
    const cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? MK_ERR_NO_MEMORY : MK_ERR_CUDA;
    }
    g->bytes += bytes;
    return MK_OK;
}

void set_free(mk_set_graph *g, void *p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        g->bytes -= bytes;
    }
}

mk_status set_stage(mk_set_graph *g, const uint32_t *src, const uint32_t *dst, uint64_t n, cudaStream_t s)
{
    if (n > g->cap) {
        uint64_t cap = std::max<uint64_t>(n, std::max<uint64_t>(1024, g->cap + g->cap / 2)), table = 1;
        while (table < 2 * cap)
            table <<= 1;
        MK_CUDA(cudaStreamSynchronize(s));
        set_free(g, g->d_tpos, g->table * 4);
        set_free(g, g->d_slot, g->cap * 4);
        g->d_tpos = g->d_slot = nullptr;
        g->cap = g->table = 0;
        MK_TRY(set_alloc(g, (void **)&g->d_tpos, table * 4));
        MK_TRY(set_alloc(g, (void **)&g->d_slot, cap * 4));
        g->cap = cap;
        g->table = table;
    }
    MK_CUDA(cudaMemsetAsync(g->d_tpos, 0xFF, g->table * 4, s));
    k_dedup<<<grid_for(n, 256), 256, 0, s>>>(src, dst, nullptr, n, g->v.V, g->d_tpos, (uint32_t)(g->table - 1),
                                             g->d_slot, g->v.st);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

uint32_t set_grid(uint64_t items_per_warp32)
{
    return std::min<uint32_t>(grid_for(std::max<uint64_t>(items_per_warp32, 1) * 32, 256), num_sms() * 32);
}

} // namespace

extern "C" {

mk_status mk_set_bucket_rule(uint32_t V, const uint32_t *d_src, uint64_t n, float load_factor, uint32_t *d_buckets,
                             void *stream)
{
    if (V == 0 || !d_buckets || (n > 0 && !d_src) || !(load_factor > 0.f) || load_factor > 1.f)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    int *d_bad = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&d_bad, sizeof(int), s));
    MK_CUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
    MK_CUDA(cudaMemsetAsync(d_buckets, 0, (size_t)V * 4, s));
    if (n)
        k_degree<<<std::min<uint64_t>(grid_for(n, 256), 4096), 256, 0, s>>>(d_src, n, V, d_buckets, d_bad);
    k_rule<<<grid_for(V, 256), 256, 0, s>>>(d_buckets, V, load_factor * (float)kSetKeys);
    int bad = 0;
    MK_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaFreeAsync(d_bad, s));
    MK_CUDA(cudaStreamSynchronize(s));
    return bad ? MK_ERR_INVALID_ARG : MK_OK;
}

mk_status mk_set_destroy(mk_set_graph *g)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    cudaFree((void *)g->v.vinfo);
    cudaFree(g->v.slabs);
    cudaFree(g->v.bitmap);
    cudaFree(g->v.owner);
    cudaFree(g->v.st);
    cudaFree(g->d_tpos);
    cudaFree(g->d_slot);
    if (g->h_pinned)
        cudaFreeHost(g->h_pinned);
    delete g;
    return MK_OK;
}

mk_status mk_set_create(uint32_t V, uint64_t edge_capacity_hint, uint32_t buckets, const uint32_t *d_bucket_per_vertex,
                        void *stream, mk_set_graph **out)
{
    if (!out || V == 0 || V > 0xFFFFFFFDu)
        return MK_ERR_INVALID_ARG;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    mk_set_graph *g = new mk_set_graph;
    g->v.V = V;
    uint32_t *d_b = nullptr;
    uint64_t *d_off = nullptr;
    void *d_tmp = nullptr;
    int *d_bad = nullptr;
    mk_status st = MK_OK;
    auto fail = [&](mk_status code) {
        cudaFree(d_b);
        cudaFree(d_off);
        cudaFree(d_tmp);
        cudaFree(d_bad);
        mk_set_destroy(g);
        return code;
    };
    if (cudaMalloc((void **)&d_b, (size_t)V * 4) != cudaSuccess ||
        cudaMalloc((void **)&d_off, ((size_t)V + 1) * 8) != cudaSuccess ||
        cudaMalloc((void **)&d_bad, sizeof(int)) != cudaSuccess ||
        cudaMalloc(&d_tmp, exclusive_scan_scratch_bytes(V + 1)) != cudaSuccess)
        return fail(MK_ERR_NO_MEMORY);
    cudaMemsetAsync(d_bad, 0, sizeof(int), s);
    k_fill_buckets<<<grid_for(V, 256), 256, 0, s>>>(d_b, V, buckets ? buckets : 1, d_bucket_per_vertex, d_bad);
    if (exclusive_scan_u32_u64(d_b, d_off, V, d_tmp, s, nullptr) != cudaSuccess)
        return fail(MK_ERR_CUDA);
    // H = last offset + last bucket count
    uint64_t last_off = 0;
    uint32_t last_b = 0;
    int bad = 0;
    if (cudaMemcpyAsync(&last_off, d_off + V - 1, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&last_b, d_b + V - 1, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess)
        return fail(MK_ERR_CUDA);
    if (bad)
        return fail(MK_ERR_INVALID_ARG);
    const uint64_t H = last_off + last_b;
    uint64_t P = edge_capacity_hint / kSetKeys + H / 8 + 1024;
    P = (P + 31) / 32 * 32;
    if (H + P >= 0xFFFFFFF0ull)
        return fail(MK_ERR_INVALID_ARG);
    g->v.H = (uint32_t)H;
    g->v.P = (uint32_t)P;
    g->v.pool_words = (uint32_t)(P / 32);
    uint2 *vinfo = nullptr;
    if ((st = set_alloc(g, (void **)&vinfo, (size_t)V * 8)) != MK_OK ||
        (st = set_alloc(g, (void **)&g->v.slabs, (H + P) * 128)) != MK_OK ||
        (st = set_alloc(g, (void **)&g->v.bitmap, (size_t)g->v.pool_words * 4)) != MK_OK ||
        (st = set_alloc(g, (void **)&g->v.owner, (H + P) * 4)) != MK_OK ||
        (st = set_alloc(g, (void **)&g->v.st, sizeof(DevState))) != MK_OK)
        return fail(st);
    g->v.vinfo = vinfo;
    if (cudaMallocHost((void **)&g->h_pinned, 64) != cudaSuccess)
        return fail(MK_ERR_NO_MEMORY);
    cudaMemsetAsync(g->v.st, 0, sizeof(DevState), s);
    k_set_init_slabs<<<std::min<uint64_t>(grid_for((H + P) * 32, 256), 65535), 256, 0, s>>>(g->v.slabs, H + P);
    k_set_init_lists<<<std::min<uint64_t>(grid_for(std::max<uint64_t>(V, P), 256), 65535), 256, 0, s>>>(
        d_off, d_b, V, vinfo, g->v.owner, H, H + P);
    k_init_bitmap<<<grid_for(g->v.pool_words, 256), 256, 0, s>>>(g->v.bitmap, g->v.pool_words, (uint32_t)P);
    if (cudaGetLastError() != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return fail(MK_ERR_CUDA);
    cudaFree(d_b);
    cudaFree(d_off);
    cudaFree(d_tmp);
    cudaFree(d_bad);
    *out = g;
    return MK_OK;
}

mk_status mk_set_insert_batch(mk_set_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                              uint8_t *d_inserted, void *stream)
{
    if (!g || (n && (!d_src || !d_dst)) || n >= 0xFFFFFFFFull)
        return MK_ERR_INVALID_ARG;
    if (!n)
        return MK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_inserted)
        MK_CUDA(cudaMemsetAsync(d_inserted, 0, n, s));
    MK_TRY(set_stage(g, d_src, d_dst, n, s));
    k_set_insert<<<set_grid((n + 31) / 32), 256, 0, s>>>(g->v, d_src, d_dst, n, g->d_tpos, g->d_slot, d_inserted,
                                                        g->v.P + 2);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_set_delete_batch(mk_set_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                              uint8_t *d_deleted, void *stream)
{
    if (!g || (n && (!d_src || !d_dst)) || n >= 0xFFFFFFFFull)
        return MK_ERR_INVALID_ARG;
    if (!n)
        return MK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (d_deleted)
        MK_CUDA(cudaMemsetAsync(d_deleted, 0, n, s));
    MK_TRY(set_stage(g, d_src, d_dst, n, s));
    k_set_delete<<<set_grid((n + 31) / 32), 256, 0, s>>>(g->v, d_src, d_dst, n, g->d_tpos, g->d_slot, d_deleted,
                                                        g->v.P + 2);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_set_query_batch(mk_set_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                             uint32_t *d_bitmap, void *stream)
{
    if (!g || (n && (!d_src || !d_dst || !d_bitmap)))
        return MK_ERR_INVALID_ARG;
    if (!n)
        return MK_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_set_query<<<set_grid((n + 31) / 32), 256, 0, s>>>(g->v, d_src, d_dst, n, d_bitmap, g->v.P + 2);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_set_bfs(mk_set_graph *g, uint32_t source, uint32_t *d_dist, uint32_t *d_parent, void *stream)
{
    if (!g || source >= g->v.V || !d_dist || !d_parent)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t V = g->v.V;
    const uint64_t H = g->v.H;
    // levels go out in groups; the host reads the frontier size once a group
    constexpr uint32_t kGroup = 6;
    uint32_t *front[2] = {nullptr, nullptr}, *cnt = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&front[0], H * 4, s));
    MK_CUDA(cudaMallocAsync((void **)&front[1], H * 4, s));
    MK_CUDA(cudaMallocAsync((void **)&cnt, 16, s));
    k_set_bfs_init<<<grid_for(V, 256), 256, 0, s>>>(g->v, d_dist, d_parent, source, front[0], cnt);
    const uint32_t grid = (uint32_t)num_sms() * 8;
    mk_status st = MK_OK;
    for (uint32_t level = 0;;) {
        if (level > V + kGroup) {
            st = MK_ERR_TIMEOUT;
            break;
        }
        for (uint32_t i = 0; i < kGroup; ++i, ++level)
            k_set_bfs_level<<<grid, 256, 0, s>>>(g->v, front[level & 1], front[(level + 1) & 1], cnt, d_dist,
                                                 d_parent, level, g->v.P + 2);
        if (cudaMemcpyAsync(g->h_pinned, cnt + level % 3, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            st = MK_ERR_CUDA;
            break;
        }
        if (g->h_pinned[0] == 0)
            break;
    }
    cudaFreeAsync(front[0], s);
    cudaFreeAsync(front[1], s);
    cudaFreeAsync(cnt, s);
    return st;
}

mk_status mk_set_wcc(mk_set_graph *g, uint32_t *d_label, void *stream)
{
    if (!g || !d_label)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t V = g->v.V;
    uint32_t *p = nullptr;
    int *failed = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&p, (size_t)V * 4, s));
    MK_CUDA(cudaMallocAsync((void **)&failed, sizeof(int), s));
    MK_CUDA(cudaMemsetAsync(failed, 0, sizeof(int), s));
    k_set_uf_init<<<grid_for(V, 256), 256, 0, s>>>(p, V);
    k_set_wcc_hook<<<resident_grid(k_set_wcc_hook, 256), 256, 0, s>>>(g->v, p, failed);
    k_set_wcc_label<<<grid_for(V, 256), 256, 0, s>>>(p, V, d_label);
    k_set_flag_status<<<1, 1, 0, s>>>(failed, g->v.st);
    const cudaError_t e = cudaGetLastError();
    cudaFreeAsync(p, s);
    cudaFreeAsync(failed, s);
    return e == cudaSuccess ? MK_OK : MK_ERR_CUDA;
}

mk_status mk_set_stats(mk_set_graph *g, uint64_t *h_lists, uint64_t *h_slabs_in_use, uint64_t *h_device_bytes,
                       void *stream)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned long long *d = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&d, 8, s));
    k_set_pool_used<<<1, 1, 0, s>>>(g->v.st, d);
    unsigned long long used = 0;
    const cudaError_t e1 = cudaMemcpyAsync(&used, d, 8, cudaMemcpyDeviceToHost, s);
    cudaFreeAsync(d, s);
    if (e1 != cudaSuccess || cudaStreamSynchronize(s) != cudaSuccess)
        return MK_ERR_CUDA;
    if (h_lists)
        *h_lists = g->v.H;
    if (h_slabs_in_use)
        *h_slabs_in_use = g->v.H + used;
    if (h_device_bytes)
        *h_device_bytes = g->bytes;
    return MK_OK;
}

mk_status mk_set_last_error(mk_set_graph *g)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    if (cudaDeviceSynchronize() != cudaSuccess)
        return MK_ERR_CUDA;
    int st = 0;
    MK_CUDA(cudaMemcpy(&st, &g->v.st->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0)
        MK_CUDA(cudaMemset(&g->v.st->status, 0, sizeof(int)));
    return st;
}

} // extern "C"
