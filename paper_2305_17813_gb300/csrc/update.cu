// Batched edge insert and delete.
//
// Staging: in-batch duplicates are found with a hash set of the batch's
// (src, dst) pairs that keeps, per pair, the smallest batch position
// (k_dedup); only that first occurrence is applied.  The insert and delete
// kernels then take the batch in tiles of 256 edges: each tile is sorted by
// slab list (source and bucket) in shared memory, so the edges of one list
// sit side by side, and one warp owns 32 consecutive sorted edges.  An edge
// whose list has no other edge in the warp (nearly every edge of a random
// batch) is handled by one 4-lane group, eight at a time per warp, with
// 16-byte slab loads; the lists with several edges in the warp are walked
// once each by the whole warp, which matches all of the list's destinations
// against every 128-byte slab (paper, Sec. "Experimental Evaluation",
// insertion and deletion; the warp-cooperative work strategy of Sec.
// "Motivation").  A list with edges in several warps is appended to by all
// of them; free pairs are claimed with 64-bit atomicCAS and new slabs are
// linked with a CAS on the next lane.
#include "mk_host.h"
#include "walk.cuh"

#include <algorithm>
#include <cstring>
#include <vector>

using namespace mk;

// 64-bit finaliser of splitmix64 (Steele, Lea and Flood, "Fast splittable
// pseudorandom number generators", 2014), as the hash of a (src, dst) pair.
__device__ __forceinline__ unsigned long long mix64(unsigned long long x)
{
    x ^= x >> 30;
    x *= 0xbf58476d1ce4e5b9ull;
    x ^= x >> 27;
    x *= 0x94d049bb133111ebull;
    x ^= x >> 31;
    return x;
}

// Validates edge i and enters its (src, dst) pair in the batch's hash set
// (open addressing with linear probing, at most half full).  An entry holds
// a batch position of its pair rather than the pair: an edge claims an empty
// entry with one CAS, and an edge that meets a taken entry compares its pair
// with the batch's pair at the stored position; on a match it lowers the
// entry to its own position if that is smaller (atomicMin), so every entry
// ends with the smallest position of its pair.  slot[i] names the entry.
// Invalid edges get slot kNil and set the invalid-argument status.
__global__ void k_dedup(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                        const uint32_t *__restrict__ w, uint64_t n, uint32_t V, uint32_t *tpos, uint32_t mask,
                        uint32_t *__restrict__ slot, DevState *st)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    bool bad = false;
    if (i < n) {
        const uint32_t s = src[i], d = dst[i];
        bad = s >= V || d >= V || (w && w[i] == 0);
        uint32_t at = kNil;
        if (!bad) {
            const unsigned long long key = ((unsigned long long)s << 32) | d;
            uint32_t h = (uint32_t)mix64(key) & mask;
            for (uint32_t probe = 0; probe <= mask; ++probe) {
                const uint32_t j = atomicCAS(&tpos[h], kNil, (uint32_t)i);
                if (j == kNil || (src[j] == s && dst[j] == d)) {
                    if (j != kNil && j > (uint32_t)i)
                        atomicMin(&tpos[h], (uint32_t)i);
                    at = h;
                    break;
                }
                h = (h + 1) & mask;
            }
        }
        slot[i] = at;
    }
    if (__ballot_sync(kFull, bad) && lane_id() == 0)
        set_status(st, kErrInvalid);
}

// One lane's edge after staging: its batch position, whether it is the
// first occurrence of its pair (only those are applied), and its list.
struct LaneEdge {
    bool first;
    uint32_t idx, src, dst, list;
};

// Sorts the 256 keys held one per thread of the block, ascending (bitonic
// network; thread t ends with the t-th smallest).  Compare-exchanges whose
// partner is in the same warp use shuffles; the six steps with partners 32
// or more threads away go through `xchg` (256 words of shared memory) with
// a block barrier around them.
__device__ __forceinline__ unsigned long long bitonic_sort_256(unsigned long long x, unsigned long long *xchg)
{
    const uint32_t t = threadIdx.x;
    for (uint32_t k = 2; k <= 256; k <<= 1) {
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            unsigned long long y;
            if (j >= 32) {
                xchg[t] = x;
                __syncthreads();
                y = xchg[t ^ j];
                __syncthreads();
            } else {
                y = __shfl_xor_sync(kFull, x, j);
            }
            const bool lower = (t & j) == 0, up = (t & k) == 0;
            x = (lower == up) ? min(x, y) : max(x, y);
        }
    }
    return x;
}

// Staging of the block's tile of 256 edges (called by the whole block, 256
// threads): each thread tests its edge for first occurrence, finds its list
// and forms key <list, position in tile> (or all-ones for an edge that is
// not applied); the tile is sorted by that key (`keys`: 256 words of shared
// memory for the sort) and thread t returns the t-th edge of the sorted
// tile.  Edges that are not applied get flag 0 here.
__device__ __forceinline__ LaneEdge stage_tile(const GView &g, const uint32_t *__restrict__ src,
                                               const uint32_t *__restrict__ dst, uint64_t n,
                                               const uint32_t *__restrict__ tpos, const uint32_t *__restrict__ slot,
                                               uint8_t *__restrict__ flags, unsigned long long *keys)
{
    const uint64_t tile0 = blockIdx.x * 256ull;
    const uint64_t i = tile0 + threadIdx.x;
    unsigned long long key = ~0ull;
    if (i < n) {
        const uint32_t sl = slot[i];
        if (sl != kNil && __ldcg(&tpos[sl]) == (uint32_t)i) {
            const uint32_t s = src[i], d = dst[i];
            const uint2 vi = g.vinfo[s];
            key = ((unsigned long long)(vi.x + bucket_of(d, vi.y)) << 32) | threadIdx.x;
        } else if (flags) {
            flags[i] = 0;
        }
    }
    const unsigned long long k = bitonic_sort_256(key, keys);
    LaneEdge e;
    e.first = k != ~0ull;
    e.list = (uint32_t)(k >> 32);
    e.idx = (uint32_t)(tile0 + (uint32_t)(k & 0xFFu));
    e.src = e.first ? src[e.idx] : 0;
    e.dst = e.first ? dst[e.idx] : 0;
    return e;
}

// Marks lanes of `members` whose destination occurs among the keys of the
// slab word v (held one word per lane).  Returns the per-lane match and, in
// *pair_of, the pair index where it matched.
__device__ __forceinline__ bool match_slab(uint32_t v, uint32_t members, bool mine, uint32_t dst, uint32_t *pair_of)
{
    const uint32_t lane = lane_id();
    if (__popc(members) == 1) {
        const uint32_t m = __ffs(members) - 1;
        const uint32_t d = __shfl_sync(kFull, dst, m);
        const uint32_t hit = __ballot_sync(kFull, is_key_lane(lane) && v == d);
        if (mine && hit) {
            *pair_of = (__ffs(hit) - 1) >> 1;
            return true;
        }
        return false;
    }
    bool found = false;
#pragma unroll
    for (uint32_t p = 0; p < kPairs; ++p) {
        const uint32_t k = __shfl_sync(kFull, v, 2 * p);
        if (mine && !found && k == dst) {
            found = true;
            *pair_of = p;
        }
    }
    return found;
}

// Lanes of the calling lane's 4-lane group in a warp-wide ballot.
__device__ __forceinline__ uint32_t group_bits(uint32_t ballot) { return (ballot >> (lane_id() & ~3u)) & 0xFu; }

// Index (0..3) of the lane's first pair whose key is k, 4 if none.  Lane s4
// of a 4-lane group holds words 8*s4 .. 8*s4+7 of a slab as two 16-byte
// vectors (lo, hi): pairs 4*s4 .. 4*s4+3; lane 3's last slot is the unused
// lane and the next lane, not a pair.
__device__ __forceinline__ uint32_t first_pair_with(const uint4 &lo, const uint4 &hi, uint32_t k)
{
    const bool last = (lane_id() & 3u) == 3u;
    return lo.x == k ? 0u : lo.z == k ? 1u : hi.x == k ? 2u : (!last && hi.z == k) ? 3u : 4u;
}

__device__ __forceinline__ void group_load(const GView &g, uint32_t s, uint4 &lo, uint4 &hi)
{
    const uint4 *p = reinterpret_cast<const uint4 *>(slab_ptr(g, s) + (lane_id() & 3u) * 8);
    lo = __ldcg(p);
    hi = __ldcg(p + 1);
}

// Finds key d in list L with one 4-lane group (layout of first_pair_with).
// Every group of the warp calls it in lockstep (L == kNil: the group has
// nothing to do).  On return *slab is the slab where the walk stopped -- the
// one holding d (*pair = its pair index) or the chain's tail -- and (lo, hi)
// hold the lane's part of it.  Returns 1 if d was found, 0 if not, 2 if the
// hop bound was hit.
__device__ __forceinline__ uint32_t group_find(const GView &g, uint32_t L, uint32_t d, uint32_t max_hops,
                                               uint32_t *slab, uint32_t *pair, uint4 &lo, uint4 &hi,
                                               unsigned long long &loads)
{
    const uint32_t s4 = lane_id() & 3u, gbase = lane_id() & ~3u;
    bool active = L != kNil;
    uint32_t res = 0, s = L;
    lo = make_uint4(kEmptyKey, kFull, kEmptyKey, kFull);
    hi = lo;
    for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
        if (active)
            group_load(g, s, lo, hi);
        loads += __popc(__ballot_sync(kFull, active && s4 == 0));
        const uint32_t hk = first_pair_with(lo, hi, d);
        const uint32_t hits = group_bits(__ballot_sync(kFull, active && hk < 4u));
        const uint32_t frees = group_bits(__ballot_sync(kFull, active && first_pair_with(lo, hi, kEmptyKey) < 4u));
        const uint32_t nxt = __shfl_sync(kFull, hi.w, gbase + 3);
        const uint32_t hp = __shfl_sync(kFull, 4 * s4 + hk, gbase + (hits ? __ffs(hits) - 1 : 0));
        if (active) {
            if (hits) {
                *pair = hp;
                res = 1;
                active = false;
            } else if (frees || nxt == kNil) {
                active = false; // the tail: free pairs exist only in the last slab
            } else if (hop + 1 >= max_hops) {
                res = 2;
                active = false;
            } else {
                s = nxt;
            }
        }
    }
    *slab = s;
    return res;
}

// Appends <d, wt> to a list whose tail is `tail` ((lo, hi) = the lane's part
// of it) with one 4-lane group: the tail's lowest free pair is claimed with
// a 64-bit CAS (a lost CAS re-reads the tail), so the pairs of a slab fill
// in order; a full tail with nothing after it gets a pool slab holding the
// pair, published with a CAS on the tail's next lane (the loser frees its
// slab and moves on to the winner's).  Every group calls it in lockstep
// (go == false: nothing to do).  Returns true on the group's lanes if the
// pair was stored; sets *err (kErrPool or kErrTimeout) when it gives up.
__device__ __forceinline__ bool group_append(const GView &g, bool go, uint32_t tail, uint4 lo, uint4 hi, uint32_t d,
                                             uint32_t wt, uint32_t owner_src, uint32_t salt, uint64_t guard_max,
                                             unsigned long long &loads, unsigned long long &linked, int *err)
{
    const uint32_t s4 = lane_id() & 3u, gbase = lane_id() & ~3u;
    bool active = go, stored = false;
    for (uint64_t guard = 0; __any_sync(kFull, active); ++guard) {
        const uint32_t fk = first_pair_with(lo, hi, kEmptyKey);
        const uint32_t frees = group_bits(__ballot_sync(kFull, active && fk < 4u));
        const uint32_t nxt = __shfl_sync(kFull, hi.w, gbase + 3);
        if (active && guard > guard_max) {
            *err = kErrTimeout;
            active = false;
        }
        // claim the group's lowest free pair
        bool ok = false;
        if (active && frees && s4 == (uint32_t)(__ffs(frees) - 1)) {
            const uint32_t p = 4 * s4 + fk;
            ok = atomicCAS(reinterpret_cast<unsigned long long *>(slab_ptr(g, tail) + 2 * p), kEmptyPair,
                           pack_pair(d, wt)) == kEmptyPair;
        }
        const bool claimed = group_bits(__ballot_sync(kFull, ok)) != 0;
        // a full tail with nothing after it: a new slab holding the pair
        const bool grow = active && !frees && nxt == kNil;
        uint32_t ns = kNil;
        if (grow && s4 == 0)
            ns = alloc_slab_one(g, salt ^ (uint32_t)(guard << 24));
        ns = __shfl_sync(kFull, ns, gbase);
        uint32_t old = kNil;
        if (grow && ns != kNil) {
            uint4 wlo = make_uint4(kEmptyKey, kFull, kEmptyKey, kFull), whi = wlo;
            if (s4 == 0)
                wlo = make_uint4(d, wt, kEmptyKey, kFull);
            else if (s4 == 3u)
                whi = make_uint4(kEmptyKey, kFull, kFull, kNil);
            uint4 *q = reinterpret_cast<uint4 *>(slab_ptr(g, ns) + s4 * 8);
            __stcg(q, wlo);
            __stcg(q + 1, whi);
            if (s4 == 0)
                g.owner[ns] = owner_src;
            __threadfence();
            if (s4 == 0)
                old = atomicCAS(slab_ptr(g, tail) + kNextLane, kNil, ns);
        }
        old = __shfl_sync(kFull, old, gbase);
        const bool won = grow && ns != kNil && old == kNil;
        linked += __popc(__ballot_sync(kFull, won && s4 == 0));
        if (active) {
            if (frees) {
                if (claimed) {
                    stored = true;
                    active = false;
                }
            } else if (nxt != kNil) {
                tail = nxt;
            } else if (ns == kNil) {
                *err = kErrPool;
                active = false;
            } else if (won) {
                stored = true;
                active = false;
            } else { // lost the link: free the slab, follow the winner's
                if (s4 == 0)
                    g.owner[ns] = kNil;
                __threadfence();
                if (s4 == 0)
                    free_slab(g, ns);
                tail = old;
            }
        }
        if (active)
            group_load(g, tail, lo, hi);
        loads += __popc(__ballot_sync(kFull, active && s4 == 0));
    }
    return stored;
}

// One block per tile of 256 edges, one warp per 32 sorted edges; see the
// file comment.
__global__ void __launch_bounds__(256, 6) k_insert(GView g, const uint32_t *__restrict__ src,
                                                   const uint32_t *__restrict__ dst, const uint32_t *__restrict__ w_in,
                                                   uint64_t n, const uint32_t *__restrict__ tpos,
                                                   const uint32_t *__restrict__ slot, uint8_t *__restrict__ flags,
                                                   uint32_t max_hops, uint32_t *__restrict__ cand)
{
    __shared__ unsigned long long keys[256];
    const uint32_t lane = lane_id();
    const uint64_t i = blockIdx.x * 256ull + threadIdx.x;
    const unsigned long long warp = i >> 5; // salt of this warp's pool probes
    if (i < n)
        cand[i] = kNil;
    const LaneEdge e = stage_tile(g, src, dst, n, tpos, slot, flags, keys);
    if (status_hint(g.st) != 0)
        return;
    const uint32_t w = (e.first && w_in) ? w_in[e.idx] : 1u;
    const uint32_t gi = lane >> 2, s4 = lane & 3u;
    uint8_t done = 0;
    unsigned long long loads = 0, linked = 0;
    // edges whose list no other lane of the warp has (nearly all of a random
    // batch): one per 4-lane group, eight per warp at a time
    const uint32_t peers = __match_any_sync(kFull, e.first ? (unsigned long long)e.list : (1ull << 32) | lane);
    const bool single = e.first && __popc(peers) == 1;
    const uint32_t sq = __ballot_sync(kFull, single);
    const uint32_t rank = __popc(sq & lanemask_lt());
    const uint64_t guard_max = n + 64 + 4ull * max_hops;
    int err = 0;
    for (uint32_t pass = 0; pass * 8 < (uint32_t)__popc(sq); ++pass) {
        const uint32_t own = group_item(sq, pass, gi);
        const uint32_t o = own & 31u;
        const uint32_t Lo = __shfl_sync(kFull, e.list, o), d = __shfl_sync(kFull, e.dst, o);
        const uint32_t wo = __shfl_sync(kFull, w, o), so = __shfl_sync(kFull, e.src, o);
        const uint32_t io = __shfl_sync(kFull, e.idx, o);
        const uint32_t L = own < 32 ? Lo : kNil;
        uint32_t tail = kNil, pair = 0;
        uint4 lo, hi;
        const uint32_t f = group_find(g, L, d, max_hops, &tail, &pair, lo, hi, loads);
        if (f == 2)
            err = kErrTimeout;
        const bool st = group_append(g, L != kNil && f == 0, tail, lo, hi, d, wo, so,
                                     (uint32_t)(warp * 8 + gi) * 0x9E3779B9u ^ tail, guard_max, loads, linked, &err);
        // the first insert into L in this epoch nominates L for the
        // updated-list log (k_log_updated compacts the nominations)
        if (st && s4 == 0 && flag_updated(g, L))
            cand[io] = L;
        // the edge of rank r went to group r % 8 in pass r / 8
        const uint32_t res = __shfl_sync(kFull, st ? 1u : 0u, (rank & 7u) * 4);
        if (single && (rank >> 3) == pass)
            done = (uint8_t)res;
    }
    if (err && s4 == 0)
        set_status(g.st, err);
    // lists with several edges in the warp: the whole warp per list
    uint32_t todo = __ballot_sync(kFull, e.first && !single);
    while (todo) {
        const uint32_t leader = __ffs(todo) - 1;
        const uint32_t L = __shfl_sync(kFull, e.list, leader);
        const uint32_t members = __ballot_sync(kFull, e.first && e.list == L) & todo;
        todo &= ~members;
        const bool mine = (members >> lane) & 1u;
        const uint32_t src_of_list = __shfl_sync(kFull, e.src, leader);
        bool absent = mine;
        // walk the whole chain: a present destination is a duplicate
        uint32_t slab = L, v = 0, em = 0, nxt = kNil, hop = 0;
        for (;; ++hop) {
            v = __ldcg(slab_ptr(g, slab) + lane);
            ++loads;
            uint32_t pf;
            if (match_slab(v, members, mine, e.dst, &pf))
                absent = false;
            em = __ballot_sync(kFull, is_key_lane(lane) && v == kEmptyKey);
            nxt = __shfl_sync(kFull, v, kNextLane);
            if (!__any_sync(kFull, absent) || em || nxt == kNil || hop >= max_hops)
                break;
            slab = nxt;
        }
        if (!__any_sync(kFull, absent))
            continue;
        if (hop >= max_hops) {
            if (lane == 0)
                set_status(g.st, kErrTimeout);
            break;
        }
        // the first insert into L in this epoch nominates L for the
        // updated-list log (k_log_updated compacts the nominations)
        if (lane == leader && flag_updated(g, L))
            cand[e.idx] = L;
        // append at the tail
        uint32_t tail = slab;
        for (uint64_t guard = 0;; ++guard) {
            const uint32_t need = __ballot_sync(kFull, absent);
            if (need == 0)
                break;
            if (guard > n + 64 + 4ull * max_hops) {
                if (lane == 0)
                    set_status(g.st, kErrTimeout);
                break;
            }
            if (em) {
                // r-th absent lane claims the r-th free pair of the tail
                const uint32_t r = __popc(need & lanemask_lt());
                if (absent && r < (uint32_t)__popc(em)) {
                    const uint32_t kl = nth_set_bit(em, r);
                    unsigned long long *pp = (unsigned long long *)(slab_ptr(g, tail) + kl);
                    if (atomicCAS(pp, kEmptyPair, pack_pair(e.dst, w)) == kEmptyPair) {
                        absent = false;
                        done = 1;
                    }
                }
                if (!__any_sync(kFull, absent))
                    break;
                v = __ldcg(slab_ptr(g, tail) + lane);
                ++loads;
                em = __ballot_sync(kFull, is_key_lane(lane) && v == kEmptyKey);
                nxt = __shfl_sync(kFull, v, kNextLane);
                continue;
            }
            if (nxt != kNil) { // someone linked a slab after our tail
                tail = nxt;
                v = __ldcg(slab_ptr(g, tail) + lane);
                ++loads;
                em = __ballot_sync(kFull, is_key_lane(lane) && v == kEmptyKey);
                nxt = __shfl_sync(kFull, v, kNextLane);
                continue;
            }
            // the tail is full: take a pool slab, fill it privately with up
            // to 15 absent edges, then publish it with a CAS on the next lane
            const uint32_t ns = alloc_slab(g, (uint32_t)warp * 0x9E3779B9u ^ tail ^ (uint32_t)(guard << 24));
            if (ns == kNil) {
                if (lane == 0)
                    set_status(g.st, kErrPool);
                break;
            }
            const uint32_t cnt = min((uint32_t)__popc(need), kPairs);
            const uint32_t p = lane >> 1;
            const uint32_t from = (lane < 30 && p < cnt) ? nth_set_bit(need, p) : 0;
            const uint32_t vd = __shfl_sync(kFull, e.dst, from);
            const uint32_t vw = __shfl_sync(kFull, w, from);
            uint32_t word;
            if (lane >= 30)
                word = kNil;
            else if (p < cnt)
                word = (lane & 1) ? vw : vd;
            else
                word = (lane & 1) ? kFull : kEmptyKey;
            __stcg(slab_ptr(g, ns) + lane, word);
            if (lane == 0)
                g.owner[ns] = src_of_list;
            __threadfence();
            uint32_t old = kNil;
            if (lane == 0)
                old = atomicCAS(slab_ptr(g, tail) + kNextLane, kNil, ns);
            old = __shfl_sync(kFull, old, 0);
            if (old == kNil) {
                ++linked;
                const uint32_t r = __popc(need & lanemask_lt());
                if (absent && r < cnt) {
                    absent = false;
                    done = 1;
                }
                tail = ns;
                v = word;
                em = __ballot_sync(kFull, is_key_lane(lane) && v == kEmptyKey);
                nxt = kNil;
            } else {
                if (lane == 0)
                    g.owner[ns] = kNil;
                __threadfence();
                if (lane == 0)
                    free_slab(g, ns);
                tail = old;
                v = __ldcg(slab_ptr(g, tail) + lane);
                ++loads;
                em = __ballot_sync(kFull, is_key_lane(lane) && v == kEmptyKey);
                nxt = __shfl_sync(kFull, v, kNextLane);
            }
        }
    }
    if (e.first && flags)
        flags[e.idx] = done;
    count_add(g.st, kCtrInsertSlabs, loads);
    count_add(g.st, kCtrInsertNewSlabs, linked);
}

// Appends the lists nominated by k_insert (cand[i] != kNil) to the
// updated-list log, with one global atomicAdd per block.
__global__ void __launch_bounds__(256) k_log_updated(GView g, const uint32_t *__restrict__ cand, uint64_t n,
                                                     const uint8_t *__restrict__ stored, const uint32_t *__restrict__ src,
                                                     const uint32_t *__restrict__ dst, const uint32_t *__restrict__ w,
                                                     uint4 *ilog, uint32_t ilog_cap)
{
    __shared__ uint32_t s2[2];
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint32_t L = i < n ? cand[i] : kNil;
    block_enqueue(g.ulog, &g.st->ulog_count, g.H, L, L != kNil, s2); // a list is logged once per epoch: fits
    // the inserted-edge log: <src, dst, stored weight> of each edge stored
    // by this batch (the host sized the log for every insert of the epoch)
    if (stored) {
        const bool ins = i < n && stored[i] != 0;
        const uint4 rec = ins ? make_uint4(src[i], dst[i], w ? w[i] : 1u, 0u) : make_uint4(0, 0, 0, 0);
        if (!block_enqueue(ilog, &g.st->ilog_count, ilog_cap, rec, ins, s2))
            set_status(g.st, kErrInternal);
    }
}

// One block per tile of 256 edges, one warp per 32 sorted edges: find each
// destination in its list's chain,
// overwrite the pair with TOMBSTONE, stop as soon as every destination of
// the group is found or the chain ends; removed edges go to the change log
// with a block-aggregated enqueue.
__global__ void __launch_bounds__(256, 8) k_delete(GView g, const uint32_t *__restrict__ src,
                                                   const uint32_t *__restrict__ dst, uint64_t n,
                                                   const uint32_t *__restrict__ tpos, const uint32_t *__restrict__ slot,
                                                   uint8_t *__restrict__ flags, unsigned long long *dlog,
                                                   uint32_t dlog_cap, uint32_t max_hops)
{
    __shared__ unsigned long long keys[256];
    __shared__ uint32_t s2[2];
    const uint32_t lane = lane_id();
    LaneEdge e = stage_tile(g, src, dst, n, tpos, slot, flags, keys);
    // no early exit: the whole block meets in block_enqueue
    if (status_hint(g.st) != 0)
        e.first = false;
    const uint32_t gi = lane >> 2, s4 = lane & 3u;
    bool removed = false;
    unsigned long long loads = 0;
    // edges whose list no other lane of the warp has: one per 4-lane group
    const uint32_t peers = __match_any_sync(kFull, e.first ? (unsigned long long)e.list : (1ull << 32) | lane);
    const bool single = e.first && __popc(peers) == 1;
    const uint32_t sq = __ballot_sync(kFull, single);
    const uint32_t rank = __popc(sq & lanemask_lt());
    for (uint32_t pass = 0; pass * 8 < (uint32_t)__popc(sq); ++pass) {
        const uint32_t own = group_item(sq, pass, gi);
        const uint32_t o = own & 31u;
        const uint32_t Lo = __shfl_sync(kFull, e.list, o), d = __shfl_sync(kFull, e.dst, o);
        const uint32_t L = own < 32 ? Lo : kNil;
        uint32_t at = kNil, pair = 0;
        uint4 lo, hi;
        const uint32_t f = group_find(g, L, d, max_hops, &at, &pair, lo, hi, loads);
        if (f == 2 && s4 == 0)
            set_status(g.st, kErrTimeout);
        if (f == 1 && s4 == 0)
            *reinterpret_cast<unsigned long long *>(slab_ptr(g, at) + 2 * pair) = kTombPair;
        const uint32_t res = __shfl_sync(kFull, f == 1 ? 1u : 0u, (rank & 7u) * 4);
        if (single && (rank >> 3) == pass)
            removed = res != 0;
    }
    // lists with several edges in the warp: the whole warp per list
    uint32_t todo = __ballot_sync(kFull, e.first && !single);
    while (todo) {
        const uint32_t leader = __ffs(todo) - 1;
        const uint32_t L = __shfl_sync(kFull, e.list, leader);
        const uint32_t members = __ballot_sync(kFull, e.first && e.list == L) & todo;
        todo &= ~members;
        const bool mine = (members >> lane) & 1u;
        bool open = mine;
        uint32_t slab = L;
        for (uint32_t hop = 0; hop < max_hops; ++hop) {
            uint32_t *sp = slab_ptr(g, slab);
            const uint32_t v = sp[lane];
            ++loads;
            uint32_t pf = 0;
            if (match_slab(v, members, mine, e.dst, &pf) && open) {
                *(unsigned long long *)(sp + 2 * pf) = kTombPair;
                removed = true;
                open = false;
            }
            const uint32_t em = __ballot_sync(kFull, is_key_lane(lane) && v == kEmptyKey);
            const uint32_t nxt = __shfl_sync(kFull, v, kNextLane);
            if (!__any_sync(kFull, open) || em || nxt == kNil)
                break;
            slab = nxt;
        }
    }
    const unsigned long long rec = ((unsigned long long)e.src << 32) | e.dst;
    if (!block_enqueue(dlog, &g.st->dlog_count, dlog_cap, rec, removed, s2))
        set_status(g.st, kErrTimeout);
    if (e.first && flags)
        flags[e.idx] = removed ? 1 : 0;
    count_add(g.st, kCtrDeleteSlabs, loads);
}

// ---------------------------------------------------------------- host side

namespace {

mk_status stage(mk_graph *g, const uint32_t *src, const uint32_t *dst, const uint32_t *w, uint64_t n,
                cudaStream_t s)
{
    MK_TRY(ensure_scratch(g, n, s));
    // the hash set must start empty (all-ones positions)
    MK_CUDA(cudaMemsetAsync(g->d_tpos, 0xFF, g->table_size * 4, s));
    return timed(g, "stage_dedup", s, 1, [&]() {
        k_dedup<<<grid_for(n, 256), 256, 0, s>>>(src, dst, w, n, g->v.V, g->d_tpos, (uint32_t)(g->table_size - 1),
                                                 g->d_slot, g->d_state);
        return cudaSuccess;
    });
}

} // namespace

// Gathers the edges of the update requests [0, nreq) into contiguous
// arrays: position i of the merged batch is edge i - prefix[r] of the
// request r with prefix[r] <= i < prefix[r + 1] (binary search; a request
// with no edges has prefix[r] == prefix[r + 1] and is never chosen).  A
// null weight array stands for weight 1.
__global__ void k_gather_updates(const mk_update_req *__restrict__ reqs, const uint64_t *__restrict__ prefix,
                                 uint32_t nreq, uint64_t total, uint32_t *__restrict__ src, uint32_t *__restrict__ dst,
                                 uint32_t *__restrict__ w)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += stride) {
        uint32_t lo = 0, hi = nreq;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (prefix[mid] <= i)
                lo = mid;
            else
                hi = mid;
        }
        const mk_update_req &r = reqs[lo];
        const uint64_t j = i - prefix[lo];
        src[i] = r.d_src[j];
        dst[i] = r.d_dst[j];
        if (w)
            w[i] = r.d_w ? r.d_w[j] : 1u;
    }
}

// Writes the merged batch's flags back to the requests that asked for them.
__global__ void k_scatter_flags(const mk_update_req *__restrict__ reqs, const uint64_t *__restrict__ prefix,
                                uint32_t nreq, uint64_t total, const uint8_t *__restrict__ flags)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < total; i += stride) {
        uint32_t lo = 0, hi = nreq;
        while (hi - lo > 1) {
            const uint32_t mid = (lo + hi) >> 1;
            if (prefix[mid] <= i)
                lo = mid;
            else
                hi = mid;
        }
        uint8_t *out = reqs[lo].d_flags;
        if (out)
            out[i - prefix[lo]] = flags[i];
    }
}

namespace {

mk_status insert_impl(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, const uint32_t *d_w, uint64_t n,
                      uint8_t *d_inserted, cudaStream_t s)
{
    g->change_seq++;
    if (n == 0)
        return MK_OK;
    // the inserted-edge log must hold every insert of the epoch
    const uint64_t need = g->ilog_bound + n;
    if (g->ilog_ok && need > g->ilog_cap) {
        uint64_t cap = std::max<uint64_t>(need, g->ilog_cap * 2);
        cap = std::min<uint64_t>(cap, 0xFFFFFFFFull);
        uint4 *nl = nullptr;
        if (need > cap || device_alloc(g, (void **)&nl, cap * 16) != MK_OK) {
            g->ilog_ok = false; // the prologues walk the updated lists instead
        } else {
            if (g->d_ilog) {
                MK_CUDA(cudaMemcpyAsync(nl, g->d_ilog, g->ilog_bound * 16, cudaMemcpyDeviceToDevice, s));
                MK_CUDA(cudaStreamSynchronize(s));
                device_free(g, g->d_ilog, g->ilog_cap * 16);
            }
            g->d_ilog = nl;
            g->ilog_cap = cap;
        }
    }
    MK_TRY(stage(g, d_src, d_dst, d_w, n, s));
    // the stored flags feed the log: the caller's array or the staging one
    uint8_t *fl = d_inserted ? d_inserted : g->d_iflags;
    MK_CUDA(cudaMemsetAsync(fl, 0, n, s));
    g->ulog_bound = std::min<uint64_t>(g->v.H, g->ulog_bound + n);
    const bool log = g->ilog_ok;
    if (log)
        g->ilog_bound = need;
    const uint32_t max_hops = g->v.P + 2;
    return timed(g, "insert", s, 2, [&]() {
        k_insert<<<grid_for(n, 256), 256, 0, s>>>(g->v, d_src, d_dst, d_w, n, g->d_tpos, g->d_slot, fl, max_hops,
                                                  g->d_cand);
        k_log_updated<<<grid_for(n, 256), 256, 0, s>>>(g->v, g->d_cand, n, log ? fl : nullptr, d_src, d_dst, d_w,
                                                       g->d_ilog, (uint32_t)g->ilog_cap);
        return cudaSuccess;
    });
}

mk_status delete_impl(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n, uint8_t *d_deleted,
                      cudaStream_t s)
{
    g->change_seq++;
    if (n == 0)
        return MK_OK;
    // the change log must hold every delete of the epoch
    const uint64_t need = g->dlog_bound + n;
    if (need > g->dlog_cap) {
        uint64_t cap = std::max<uint64_t>(need, g->dlog_cap * 2);
        cap = std::min<uint64_t>(cap, 0xFFFFFFFFull);
        unsigned long long *nl = nullptr;
        MK_TRY(device_alloc(g, (void **)&nl, cap * 8));
        if (g->d_dlog) {
            MK_CUDA(cudaMemcpyAsync(nl, g->d_dlog, g->dlog_bound * 8, cudaMemcpyDeviceToDevice, s));
            MK_CUDA(cudaStreamSynchronize(s));
            device_free(g, g->d_dlog, g->dlog_cap * 8);
        }
        g->d_dlog = nl;
        g->dlog_cap = cap;
    }
    g->dlog_bound = need;
    g->epoch_has_deletes = true;
    if (d_deleted)
        MK_CUDA(cudaMemsetAsync(d_deleted, 0, n, s));
    MK_TRY(stage(g, d_src, d_dst, nullptr, n, s));
    const uint32_t max_hops = g->v.P + 2;
    return timed(g, "delete", s, 1, [&]() {
        k_delete<<<grid_for(n, 256), 256, 0, s>>>(g->v, d_src, d_dst, n, g->d_tpos, g->d_slot, d_deleted, g->d_dlog,
                                                  (uint32_t)g->dlog_cap, max_hops);
        return cudaSuccess;
    });
}

} // namespace

extern "C" {

mk_status mk_insert_batch(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, const uint32_t *d_w,
                          uint64_t n, uint8_t *d_inserted, void *stream)
{
    if (!g || (n > 0 && (!d_src || !d_dst)) || n >= 0xFFFFFFFFull)
        return MK_ERR_INVALID_ARG;
    return insert_impl(g, d_src, d_dst, d_w, n, d_inserted, (cudaStream_t)stream);
}

mk_status mk_delete_batch(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                          uint8_t *d_deleted, void *stream)
{
    if (!g || (n > 0 && (!d_src || !d_dst)) || n >= 0xFFFFFFFFull)
        return MK_ERR_INVALID_ARG;
    return delete_impl(g, d_src, d_dst, n, d_deleted, (cudaStream_t)stream);
}

mk_status mk_update_multi(mk_graph *g, const mk_update_req *h_reqs, uint32_t nreq, void *stream)
{
    if (!g || (nreq && !h_reqs))
        return MK_ERR_INVALID_ARG;
    for (uint32_t i = 0; i < nreq; ++i) {
        const mk_update_req &r = h_reqs[i];
        if ((r.kind != MK_REQ_INSERT && r.kind != MK_REQ_DELETE) || (r.n && (!r.d_src || !r.d_dst)))
            return MK_ERR_INVALID_ARG;
    }
    cudaStream_t s = (cudaStream_t)stream;
    // runs of consecutive requests of one kind, and each run's prefix of
    // edge counts (nreq + runs entries in all)
    std::vector<std::pair<uint32_t, uint32_t>> runs;
    for (uint32_t i = 0; i < nreq;) {
        uint32_t j = i + 1;
        while (j < nreq && h_reqs[j].kind == h_reqs[i].kind)
            ++j;
        runs.push_back({i, j});
        i = j;
    }
    std::vector<uint64_t> prefix;
    uint64_t max_total = 0;
    for (auto &r : runs) {
        uint64_t acc = 0;
        for (uint32_t i = r.first; i < r.second; ++i) {
            prefix.push_back(acc);
            acc += h_reqs[i].n;
        }
        prefix.push_back(acc);
        if (acc >= 0xFFFFFFFFull)
            return MK_ERR_INVALID_ARG;
        if (r.second - r.first > 1)
            max_total = std::max(max_total, acc);
    }
    // descriptors and prefixes in one device block; staging for the largest
    // merged run
    const size_t desc_bytes = (size_t)nreq * sizeof(mk_update_req);
    const size_t block_bytes = desc_bytes + prefix.size() * 8;
    std::vector<unsigned char> img(block_bytes);
    std::memcpy(img.data(), h_reqs, desc_bytes);
    std::memcpy(img.data() + desc_bytes, prefix.data(), prefix.size() * 8);
    unsigned char *d_blk = nullptr;
    uint32_t *d_m = nullptr;
    uint8_t *d_mf = nullptr;
    if (max_total) {
        MK_CUDA(cudaMallocAsync((void **)&d_blk, block_bytes, s));
        MK_CUDA(cudaMemcpyAsync(d_blk, img.data(), block_bytes, cudaMemcpyHostToDevice, s));
        MK_CUDA(cudaMallocAsync((void **)&d_m, max_total * 12, s));
        MK_CUDA(cudaMallocAsync((void **)&d_mf, max_total, s));
    }
    mk_status st = MK_OK;
    size_t pre = 0;
    for (auto &r : runs) {
        const uint32_t k = r.second - r.first;
        const bool ins = h_reqs[r.first].kind == MK_REQ_INSERT;
        const uint64_t total = prefix[pre + k];
        if (k == 1) {
            const mk_update_req &q = h_reqs[r.first];
            st = ins ? insert_impl(g, q.d_src, q.d_dst, q.d_w, q.n, q.d_flags, s)
                     : delete_impl(g, q.d_src, q.d_dst, q.n, q.d_flags, s);
        } else if (total) {
            const mk_update_req *dreq = reinterpret_cast<const mk_update_req *>(d_blk) + r.first;
            const uint64_t *dpre = reinterpret_cast<const uint64_t *>(d_blk + desc_bytes) + pre;
            bool want_flags = false;
            for (uint32_t i = r.first; i < r.second; ++i)
                want_flags |= h_reqs[i].d_flags != nullptr && h_reqs[i].n;
            uint32_t *ms = d_m, *md = d_m + total, *mw = d_m + 2 * total;
            const uint32_t grid = std::min<uint32_t>(grid_for(total, 256), num_sms() * 8);
            st = timed(g, "update_gather", s, 1, [&]() {
                k_gather_updates<<<grid, 256, 0, s>>>(dreq, dpre, k, total, ms, md, ins ? mw : nullptr);
                return cudaSuccess;
            });
            if (st == MK_OK)
                st = ins ? insert_impl(g, ms, md, mw, total, want_flags ? d_mf : nullptr, s)
                         : delete_impl(g, ms, md, total, want_flags ? d_mf : nullptr, s);
            if (st == MK_OK && want_flags)
                st = timed(g, "update_scatter", s, 1, [&]() {
                    k_scatter_flags<<<grid, 256, 0, s>>>(dreq, dpre, k, total, d_mf);
                    return cudaSuccess;
                });
        } else {
            g->change_seq++;
        }
        pre += k + 1;
        if (st != MK_OK)
            break;
    }
    if (d_blk)
        cudaFreeAsync(d_blk, s);
    if (d_m)
        cudaFreeAsync(d_m, s);
    if (d_mf)
        cudaFreeAsync(d_mf, s);
    return st;
}

} // extern "C"
