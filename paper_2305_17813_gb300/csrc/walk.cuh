// Slab-list traversal and frontier helpers shared by the algorithm kernels.
#pragma once

#include "mk_device.cuh"

namespace mk {

// A block's staging area for frontier entries.  Warps reserve slots with
// shared-memory atomics; the block copies the staged entries to the global
// frontier with one global atomicAdd (bq_flush), instead of one atomic per
// enqueuing warp on the single global frontier counter, where thousands of
// warps a round would serialise.
constexpr uint32_t kBlockBuf = 2048;
struct BlockFrontier {
    uint2 buf[kBlockBuf];
    uint32_t count; // slots reserved; those at or past kBlockBuf went to the global frontier
    uint32_t base;
};

// Appends the slab lists of vertex y (for every lane with pred; vi is y's
// vinfo entry, loaded by the caller) to the list frontier as <list, y>
// entries (the source travels with the list, so a consumer needs no list_src
// lookup).  Lanes with few buckets write their entries through the block's
// staging area: the warp's entries take slots [off, off + total) of the
// block buffer and those that do not fit go to the global frontier directly.
// A vertex with many buckets is written to the global frontier by the whole
// warp.  Must be called by the full warp; sets *overflow for an entry that
// would not fit in `cap`.
__device__ __forceinline__ void enqueue_lists_block(BlockFrontier &bq, uint32_t y, bool pred, uint2 vi, uint2 *out,
                                                    uint32_t *count, uint32_t cap, int *overflow)
{
    constexpr uint32_t kSmall = 8;
    const uint32_t lane = lane_id();
    if (!__any_sync(kFull, pred))
        return;
    const bool small = pred && vi.y <= kSmall;
    const uint32_t c = small ? vi.y : 0;
    uint32_t incl = c;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint32_t t = __shfl_up_sync(kFull, incl, o);
        if (lane >= o)
            incl += t;
    }
    const uint32_t total = __shfl_sync(kFull, incl, 31);
    if (total) {
        uint32_t off = 0;
        if (lane == 0)
            off = atomicAdd(&bq.count, total);
        off = __shfl_sync(kFull, off, 0);
        const uint32_t room = off < kBlockBuf ? min(kBlockBuf - off, total) : 0u;
        uint32_t gbase = 0;
        if (room < total && lane == 0)
            gbase = atomicAdd(count, total - room);
        gbase = __shfl_sync(kFull, gbase, 0);
        for (uint32_t k = 0; k < c; ++k) {
            const uint32_t t = incl - c + k; // the warp's t-th entry
            const uint2 ent = make_uint2(vi.x + k, y);
            if (t < room)
                bq.buf[off + t] = ent;
            else if (gbase + (t - room) < cap)
                out[gbase + (t - room)] = ent;
            else
                *overflow = 1;
        }
    }
    uint32_t big = __ballot_sync(kFull, pred && !small);
    while (big) {
        const uint32_t l = __ffs(big) - 1;
        big &= big - 1;
        const uint32_t first = __shfl_sync(kFull, vi.x, l);
        const uint32_t nb = __shfl_sync(kFull, vi.y, l);
        const uint32_t yl = __shfl_sync(kFull, y, l);
        uint32_t base = 0;
        if (lane == 0)
            base = atomicAdd(count, nb);
        base = __shfl_sync(kFull, base, 0);
        for (uint32_t k = lane; k < nb; k += 32) {
            if (base + k < cap)
                out[base + k] = make_uint2(first + k, yl);
            else
                *overflow = 1;
        }
    }
}

// Copies the block's staged entries to the global frontier and empties the
// staging area.  Called by every thread of the block (it synchronises the
// block).
__device__ __forceinline__ void bq_flush(BlockFrontier &bq, uint2 *out, uint32_t *count, uint32_t cap, int *overflow)
{
    __syncthreads();
    const uint32_t n = min(bq.count, kBlockBuf);
    if (threadIdx.x == 0)
        bq.base = n ? atomicAdd(count, n) : 0u;
    __syncthreads();
    for (uint32_t t = threadIdx.x; t < n; t += blockDim.x) {
        if (bq.base + t < cap)
            out[bq.base + t] = bq.buf[t];
        else
            *overflow = 1;
    }
    __syncthreads();
    if (threadIdx.x == 0)
        bq.count = 0;
    __syncthreads();
}

__device__ __forceinline__ void bq_init(BlockFrontier &bq)
{
    if (threadIdx.x == 0)
        bq.count = 0;
    __syncthreads();
}


} // namespace mk

namespace mk {

// Tiled walk: each 4-lane group of the warp walks its own slab list (eight
// lists per warp, so a warp has eight slab loads in flight instead of one);
// lane s4 of a group holds words 8*s4 .. 8*s4+7 of the slab as two 16-byte
// vectors, i.e. pairs 4*s4 .. 4*s4+3 (lane 3: pairs 12-14, then the unused
// lane and the next lane).  `slab` and `first_lane` are per group (kNil =
// the group has no list).  Per slab, f(key, weight, live) is called once by
// every lane of the warp (convergent) with the lane's four pairs as arrays
// (key[k], weight[k], live[k], k = 0..3), so that the callee can put the
// memory accesses of all four in flight together; `live` is false for free /
// deleted keys, for key words below first_lane on the first slab, and for
// groups without a list.  With have_first, (lo0, hi0) already hold the
// lane's part of `slab` (group4_load), loaded ahead by the caller.  Stops
// after the slab whose next lane is null or after max_hops slabs; returns
// the number of slabs loaded by the warp.
template <typename F>
__device__ __forceinline__ uint32_t walk_lists_g4_from(const GView &g, uint32_t slab, bool have_first, uint4 lo0,
                                                       uint4 hi0, uint32_t first_lane, uint32_t max_hops, F &&f)
{
    const uint32_t lane = lane_id(), s4 = lane & 3u, gbase = lane & ~3u;
    bool active = slab != kNil;
    uint32_t loads = 0;
    for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
        uint4 lo = make_uint4(kEmptyKey, kFull, kFull, kFull), hi = lo;
        if (hop == 0 && have_first) {
            lo = lo0;
            hi = hi0;
        } else if (active) {
            const uint4 *p = reinterpret_cast<const uint4 *>(slab_ptr(g, slab) + s4 * 8);
            lo = __ldcg(p);
            hi = __ldcg(p + 1);
        }
        loads += __popc(__ballot_sync(kFull, active && s4 == 0));
        const uint32_t w0 = 8 * s4;
        const uint32_t key[4] = {lo.x, lo.z, hi.x, hi.z}, wt[4] = {lo.y, lo.w, hi.y, hi.w};
        const bool live[4] = {active && lo.x < kTombKey && w0 >= first_lane,
                              active && lo.z < kTombKey && w0 + 2 >= first_lane,
                              active && hi.x < kTombKey && w0 + 4 >= first_lane,
                              active && s4 != 3u && hi.z < kTombKey && w0 + 6 >= first_lane};
        f(key, wt, live);
        const uint32_t nxt = __shfl_sync(kFull, hi.w, gbase + 3);
        if (active) {
            if (nxt == kNil || hop + 1 >= max_hops)
                active = false;
            else
                slab = nxt;
        }
        first_lane = 0;
    }
    return loads;
}

// The lane's 32-byte part of slab s for a 4-lane group (words 8*s4 ..
// 8*s4+7); empty parts for s == kNil.
__device__ __forceinline__ void group4_load(const GView &g, uint32_t s, uint4 &lo, uint4 &hi)
{
    lo = make_uint4(kEmptyKey, kFull, kFull, kFull);
    hi = lo;
    if (s != kNil) {
        const uint4 *p = reinterpret_cast<const uint4 *>(slab_ptr(g, s) + (lane_id() & 3u) * 8);
        lo = __ldcg(p);
        hi = __ldcg(p + 1);
    }
}

// The k-th set bit of q handed to 4-lane group `gi` in pass `pass` (eight
// groups per pass): returns the lane index holding that group's item, or
// 32 when the pass has fewer items than groups.
__device__ __forceinline__ uint32_t group_item(uint32_t q, uint32_t pass, uint32_t gi)
{
    const uint32_t k = pass * 8 + gi;
    if (k >= (uint32_t)__popc(q))
        return 32;
    return nth_set_bit(q, k);
}

} // namespace mk
