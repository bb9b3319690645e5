// Device-side layout and warp helpers of the slab-hash graph store.
//
// Slab (paper, Sec. "Motivation"): 128 bytes = 32 lanes of 4 bytes, read by
// one warp in one coalesced load.  Weighted (ConcurrentMap) layout: lane 2p
// holds the destination key and lane 2p+1 its weight for p = 0..14, lane 30
// is unused and lane 31 holds the index of the next slab (kNil at the tail).
// A free pair is <EMPTY_KEY, 0xFFFFFFFF> (the 64-bit value UINT64_MAX - 1), a
// deleted pair <TOMBSTONE_KEY, TOMBSTONE_KEY> (footnotes on EMPTY_KEY and
// TOMBSTONE_KEY).  Deleted pairs are never reused, so free pairs only exist
// in the last slab of a chain and an insert always lands at the chain's end.
//
// Slab indices are 32-bit: the head slabs of all lists occupy [0, H) of one
// allocation and the overflow pool occupies [H, H + P) of the same one.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace mk {

constexpr uint32_t kFull = 0xFFFFFFFFu;
constexpr uint32_t kNil = 0xFFFFFFFFu;        // null slab / INF distance / INVALID vertex
constexpr uint32_t kEmptyKey = 0xFFFFFFFEu;
constexpr uint32_t kTombKey = 0xFFFFFFFDu;
constexpr unsigned long long kEmptyPair = 0xFFFFFFFFFFFFFFFEull;
constexpr unsigned long long kTombPair = 0xFFFFFFFDFFFFFFFDull;
constexpr unsigned long long kInfNode = 0xFFFFFFFFFFFFFFFFull; // <INF, INVALID>
constexpr uint32_t kPairs = 15;
constexpr uint32_t kNextLane = 31;
constexpr uint8_t kInvalidLane = 0xFF;

// Device status codes (mirror the public MK_ERR_* values).
constexpr int kErrInvalid = -1;
constexpr int kErrPool = -2;
constexpr int kErrTimeout = -3;
constexpr int kErrInternal = -6;

// Work counters (slabs loaded, edges examined, ...) accumulated by the
// kernels with one atomicAdd per warp; they give the algorithmic byte counts
// of the roofline figures.
enum Counter {
    kCtrQuerySlabs = 0,
    kCtrInsertSlabs = 1,
    kCtrInsertNewSlabs = 2,
    kCtrDeleteSlabs = 3,
    kCtrRelaxLists = 4,
    kCtrRelaxSlabs = 5,
    kCtrRelaxEdges = 6,
    kCtrRelaxImproved = 7,
    kCtrInvalidated = 8,   // vertices invalidated by deletions
    kCtrWccSlabs = 9,
    kCtrWccEdges = 10,
    kCtrCommitSlabs = 11,
    kCtrSeedLists = 12,    // prologue kernels (incremental / decremental seeds)
    kCtrSeedSlabs = 13,
    kCtrSeedEdges = 14,
    kCtrSeedImproved = 15,
    kCtrWccUpdSlabs = 16,  // incremental WCC pass (updated lists only)
    kCtrWccUpdEdges = 17,
    kCtrRounds = 18,       // BFS/SSSP rounds run by the persistent round kernel
    kCtrGridBarriers = 19, // grid barriers it crossed
    kCtrScanOwners = 20,   // relax-into-invalid scan: slabs in use (copied)
    kCtrScanSlabs = 21,    //   slabs read (source reached and valid)
    kCtrScanEdges = 22,    //   live edges examined
    kCtrScanTargets = 23,  //   edges into invalidated vertices (relaxed)
    kCtrScanImproved = 24, //   invalidated vertices given a finite distance
    kCtrWalkVertices = 25, // vertices visited by the invalidation pass
    kCtrUnpacked = 26,     // BFS/SSSP tree nodes written to the caller's dist/parent arrays
    kCtrSeedLog = 27,      // inserted-edge log entries read by the incremental prologue
    kCtrWccLog = 28,       // inserted-edge log entries read by the incremental WCC pass
    kNumCounters = 32
};

// Tallies that many warps bump (work counters, pool slabs in use) are kept
// in kSlots copies, the copy picked by block index, and summed when read:
// one shared word bumped by every warp of a large launch serialises tens of
// thousands of atomics on one L2 line.
constexpr uint32_t kSlots = 64;

// Mutable device-side state of one graph (one allocation).
struct DevState {
    int status;                    // sticky error word
    uint32_t dlog_count;           // entries in the delete log
    uint32_t ulog_count;           // entries in the updated-list log
    uint32_t ilog_count;           // entries in the inserted-edge log
    long long pool_used[kSlots];   // pool slabs allocated minus freed (kept with the bitmap), per slot
    unsigned long long ctr[kNumCounters][kSlots];
};

__device__ __forceinline__ uint32_t slot_of_block() { return blockIdx.x & (kSlots - 1); }

// Read-only view of one graph passed to kernels by value.
struct GView {
    uint32_t V;
    uint32_t H;            // slab lists (= head slabs)
    uint32_t P;            // pool slabs
    uint32_t pool_words;   // ceil(P / 32)
    const uint2 *vinfo;    // per vertex: {first list, bucket count}
    uint32_t *slabs;       // (H + P) * 32 words
    uint32_t *bitmap;      // pool occupancy, 1 bit per pool slab
    const uint32_t *list_src; // source vertex of each list
    uint32_t *owner;       // per slab (heads and pool): source vertex of its list, kNil if unused
    unsigned long long *lmark; // per list: marker slab << 32 | marker lane
    uint8_t *lupd;         // per list: updated since the last commit (H bytes, rounded up to whole words)
    uint32_t *ulog;        // the lists updated since the last commit, in order of their first update
    DevState *st;
};

__device__ __forceinline__ uint32_t lane_id() { return threadIdx.x & 31; }
__device__ __forceinline__ uint32_t lanemask_lt() { return (1u << lane_id()) - 1u; }
__device__ __forceinline__ bool is_key_lane(uint32_t lane) { return lane < 30 && (lane & 1) == 0; }
constexpr uint32_t kKeyLanes = 0x15555555u; // even lanes 0..28

__device__ __forceinline__ uint32_t *slab_ptr(const GView &g, uint32_t s)
{
    return g.slabs + (size_t)s * 32;
}

// Position of the (r+1)-th set bit of m (r < popc(m)).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t m, uint32_t r)
{
    for (uint32_t i = 0; i < r; ++i)
        m &= m - 1;
    return __ffs(m) - 1;
}

// 32-bit integer hash "lowbias32" (C. Wellons, hash-prospector, 2018).
__device__ __forceinline__ uint32_t hash32(uint32_t x)
{
    x ^= x >> 16;
    x *= 0x7feb352du;
    x ^= x >> 15;
    x *= 0x846ca68bu;
    x ^= x >> 16;
    return x;
}

// Bucket of destination d among nb buckets: multiply-shift range reduction
// of the hash (any hash works; it only changes the layout, never a result).
__device__ __forceinline__ uint32_t bucket_of(uint32_t d, uint32_t nb)
{
    return nb <= 1 ? 0u : (uint32_t)(((unsigned long long)hash32(d) * nb) >> 32);
}

__device__ __forceinline__ unsigned long long pack_pair(uint32_t key, uint32_t w)
{
    return ((unsigned long long)w << 32) | key;
}

__device__ __forceinline__ void set_status(DevState *st, int code)
{
    atomicCAS(&st->status, 0, code);
}

// Block-collective (every thread of the block calls it, converged):
// appends `value` for every thread with pred to arr (capacity cap) at slots
// reserved with one global atomicAdd per block.  This is the paper's
// warp-aggregated enqueue (Algorithm "Warp device APIs") lifted to the
// block: one atomic per warp on the single count word serialises when tens
// of thousands of warps append.
// `s2` is two words of shared memory.  Returns false for a thread whose slot
// was at or past cap.
template <typename T>
__device__ __forceinline__ bool block_enqueue(T *arr, uint32_t *count, uint32_t cap, T value, bool pred, uint32_t *s2)
{
    const uint32_t mask = __ballot_sync(0xFFFFFFFFu, pred);
    if (threadIdx.x == 0)
        s2[0] = 0;
    __syncthreads();
    uint32_t woff = 0;
    if (lane_id() == 0 && mask)
        woff = atomicAdd(&s2[0], (uint32_t)__popc(mask));
    __syncthreads();
    if (threadIdx.x == 0 && s2[0])
        s2[1] = atomicAdd(count, s2[0]);
    __syncthreads();
    woff = __shfl_sync(0xFFFFFFFFu, woff, 0);
    if (!pred)
        return true;
    const uint32_t at = s2[1] + woff + __popc(mask & ((1u << lane_id()) - 1));
    if (at >= cap)
        return false;
    arr[at] = value;
    return true;
}

// Flags list L as updated since the last commit (a 32-bit atomicOr on the
// word holding its byte); true if this call set the flag, i.e. L's first
// update in the epoch, which puts L in the updated-list log: later passes
// over the updated lists (UpdateIterator consumers, UpdateSlabPointers) read
// the log instead of testing every list's flag.
__device__ __forceinline__ bool flag_updated(const GView &g, uint32_t L)
{
    if (*(volatile const uint8_t *)&g.lupd[L])
        return false;
    uint32_t *word = reinterpret_cast<uint32_t *>(g.lupd + (L & ~3u));
    const uint32_t bit = 1u << ((L & 3u) * 8);
    return !(atomicOr(word, bit) & bit);
}

// Adds a per-warp count to a work counter (lane 0 only; v must be
// warp-uniform).
__device__ __forceinline__ void count_add(DevState *st, int which, unsigned long long v)
{
    if ((threadIdx.x & 31) == 0 && v)
        atomicAdd(&st->ctr[which][slot_of_block()], v);
}

__device__ __forceinline__ int read_status(const DevState *st)
{
    return *((volatile const int *)&st->status);
}

// The status word through the read-only path: one cached copy per SM
// instead of one request per warp to a single L2 line.  A stale 0 only
// delays an early exit.
__device__ __forceinline__ int status_hint(const DevState *st) { return __ldg(&st->status); }


// Warp-cooperative claim of one pool slab from the occupancy bitmap.  The
// warp probes 32 consecutive words at once, starting at a word chosen by
// hashing `salt` uniformly over the whole pool (so concurrent claims land on
// different words and a probe finds a free bit at once unless the pool is
// nearly full), and the lowest lane that sees a free bit claims it with
// atomicOr.  All 32 lanes must call; all receive the slab index (H + bit),
// or kNil when a sweep over the whole bitmap found nothing.
__device__ __forceinline__ uint32_t alloc_slab(const GView &g, uint32_t salt)
{
    const uint32_t W = g.pool_words;
    if (W == 0)
        return kNil;
    const uint32_t lane = lane_id();
    const uint64_t start = (uint64_t)hash32(salt) % W;
    const uint32_t sweeps = W / 32 + 2;
    for (uint32_t it = 0; it < sweeps; ++it) {
        const uint32_t wi = (uint32_t)((start + (uint64_t)it * 32 + lane) % W);
        uint32_t word = __ldcg(&g.bitmap[wi]);
        uint32_t cand = __ballot_sync(kFull, word != kFull);
        while (cand) {
            const uint32_t l = __ffs(cand) - 1;
            uint32_t got = kNil;
            if (lane == l) {
                const uint32_t b = __ffs(~word) - 1;
                const uint32_t old = atomicOr(&g.bitmap[wi], 1u << b);
                if (!(old & (1u << b)))
                    got = g.H + wi * 32 + b;
                else
                    word = old | (1u << b);
            }
            if (got != kNil)
                atomicAdd((unsigned long long *)&g.st->pool_used[slot_of_block()], 1ull);
            got = __shfl_sync(kFull, got, l);
            if (got != kNil)
                return got;
            cand = __ballot_sync(kFull, word != kFull);
        }
    }
    return kNil;
}

// One thread's slab allocation: probes the bitmap word by word from a start
// hashed from `salt` and claims the lowest free bit of the first word that
// has one with atomicOr.  Returns the slab index (H + bit), or kNil after a
// sweep over the whole bitmap found nothing.
__device__ __forceinline__ uint32_t alloc_slab_one(const GView &g, uint32_t salt)
{
    const uint32_t W = g.pool_words;
    if (W == 0)
        return kNil;
    uint32_t wi = (uint32_t)((uint64_t)hash32(salt) % W);
    for (uint32_t it = 0; it < W; ++it) {
        uint32_t word = __ldcg(&g.bitmap[wi]);
        while (word != kFull) {
            const uint32_t b = __ffs(~word) - 1;
            const uint32_t old = atomicOr(&g.bitmap[wi], 1u << b);
            if (!(old & (1u << b))) {
                atomicAdd((unsigned long long *)&g.st->pool_used[slot_of_block()], 1ull);
                return g.H + wi * 32 + b;
            }
            word = old | (1u << b);
        }
        wi = wi + 1 == W ? 0 : wi + 1;
    }
    return kNil;
}

__device__ __forceinline__ void free_slab(const GView &g, uint32_t s)
{
    const uint32_t i = s - g.H;
    atomicAnd(&g.bitmap[i >> 5], ~(1u << (i & 31)));
    atomicAdd((unsigned long long *)&g.st->pool_used[slot_of_block()], ~0ull);
}

} // namespace mk
