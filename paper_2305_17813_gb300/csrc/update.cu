// Batched edge insert and delete.
//
// Staging: each batch is keyed by (src << b | dst) and radix sorted, so the
// edges of one source are contiguous and repeated (src, dst) pairs are
// adjacent with the first occurrence first (the sort is stable).  One warp
// then owns 32 consecutive sorted edges; it groups its lanes by slab list
// (src and bucket), walks each list's chain once with coalesced 128-byte
// slab loads and matches all of the group's destinations against every
// slab (paper, Sec. "Experimental Evaluation", insertion and deletion; the
// warp-cooperative work strategy of Sec. "Motivation").  A list whose edges
// straddle two warps is appended to by both; free pairs are claimed with
// 64-bit atomicCAS and new slabs are linked with a CAS on the next lane.
#include "mk_host.h"

#include <algorithm>

using namespace mk;

// Validates the batch and writes sort keys and original positions.
__global__ void k_build_keys(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                             const uint32_t *__restrict__ w, uint64_t n, uint32_t V, uint32_t vbits,
                             uint64_t *__restrict__ keys, uint32_t *__restrict__ idx, DevState *st)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    bool bad = false;
    if (i < n) {
        const uint32_t s = src[i], d = dst[i];
        bad = s >= V || d >= V || (w && w[i] == 0);
        keys[i] = ((uint64_t)s << vbits) | d;
        idx[i] = (uint32_t)i;
    }
    if (__ballot_sync(kFull, bad) && lane_id() == 0)
        set_status(st, kErrInvalid);
}

// Sorted-batch prologue shared by insert and delete: decodes this lane's
// edge, flags the first occurrence of each (src, dst) and finds its list.
struct LaneEdge {
    bool inb, first;
    uint32_t idx, src, dst, list;
};

__device__ __forceinline__ LaneEdge load_sorted(const GView &g, const uint64_t *skey, const uint32_t *sidx,
                                                uint64_t n, uint32_t vbits, uint64_t pos)
{
    LaneEdge e;
    e.inb = pos < n;
    const uint64_t key = e.inb ? skey[pos] : ~0ull;
    uint64_t prev = __shfl_up_sync(kFull, key, 1);
    if (lane_id() == 0)
        prev = (e.inb && pos > 0) ? skey[pos - 1] : ~0ull;
    e.first = e.inb && (pos == 0 || prev != key);
    e.idx = e.inb ? sidx[pos] : 0;
    e.src = (uint32_t)(key >> vbits);
    e.dst = (uint32_t)(key & ((1ull << vbits) - 1));
    e.list = 0;
    if (e.first) {
        const uint2 vi = g.vinfo[e.src];
        e.list = vi.x + bucket_of(e.dst, vi.y);
    }
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

// One warp per 32 sorted edges; see the file comment.
__global__ void __launch_bounds__(256, 8) k_insert(GView g, const uint64_t *__restrict__ skey,
                                                const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ w_in,
                                                uint64_t n, uint32_t vbits, uint8_t *__restrict__ flags,
                                                uint32_t max_hops, uint32_t *__restrict__ cand)
{
    const uint32_t lane = lane_id();
    const unsigned long long warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t pos = warp * 32 + lane;
    if (warp * 32 >= n)
        return;
    if (pos < n)
        cand[pos] = kNil;
    if (status_hint(g.st) != 0)
        return;
    const LaneEdge e = load_sorted(g, skey, sidx, n, vbits, pos);
    const uint32_t w = (e.first && w_in) ? w_in[e.idx] : 1u;
    uint8_t done = 0;
    unsigned long long loads = 0, linked = 0;
    uint32_t todo = __ballot_sync(kFull, e.first);
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
            cand[pos] = L;
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
    if (e.inb && flags)
        flags[e.idx] = done;
    count_add(g.st, kCtrInsertSlabs, loads);
    count_add(g.st, kCtrInsertNewSlabs, linked);
}

// Appends the lists nominated by k_insert (cand[i] != kNil) to the
// updated-list log, with one global atomicAdd per block.
__global__ void __launch_bounds__(256) k_log_updated(GView g, const uint32_t *__restrict__ cand, uint64_t n)
{
    __shared__ uint32_t s2[2];
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    const uint32_t L = i < n ? cand[i] : kNil;
    block_enqueue(g.ulog, &g.st->ulog_count, g.H, L, L != kNil, s2); // a list is logged once per epoch: fits
}

// One warp per 32 sorted edges: find each destination in its list's chain,
// overwrite the pair with TOMBSTONE, stop as soon as every destination of
// the group is found or the chain ends; removed edges go to the change log
// with a block-aggregated enqueue.
__global__ void __launch_bounds__(256, 8) k_delete(GView g, const uint64_t *__restrict__ skey,
                                                const uint32_t *__restrict__ sidx, uint64_t n, uint32_t vbits,
                                                uint8_t *__restrict__ flags, unsigned long long *dlog,
                                                uint32_t dlog_cap, uint32_t max_hops)
{
    __shared__ uint32_t s2[2];
    const uint32_t lane = lane_id();
    const unsigned long long warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t pos = warp * 32 + lane;
    // no early exit: the whole block meets in block_enqueue
    const bool run = warp * 32 < n && status_hint(g.st) == 0;
    LaneEdge e{};
    if (run)
        e = load_sorted(g, skey, sidx, n, vbits, pos);
    bool removed = false;
    unsigned long long loads = 0;
    uint32_t todo = run ? __ballot_sync(kFull, e.first) : 0u;
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
    if (run && e.inb && flags)
        flags[e.idx] = removed ? 1 : 0;
    count_add(g.st, kCtrDeleteSlabs, loads);
}

// ---------------------------------------------------------------- host side

namespace {

mk_status stage(mk_graph *g, const uint32_t *src, const uint32_t *dst, const uint32_t *w, uint64_t n,
                cudaStream_t s)
{
    MK_TRY(ensure_scratch(g, n, s));
    const int bits = 2 * (int)g->vbits;
    MK_TRY(timed(g, "stage_keys", s, 1, [&]() {
        k_build_keys<<<grid_for(n, 256), 256, 0, s>>>(src, dst, w, n, g->v.V, g->vbits, g->d_kin, g->d_iin,
                                                      g->d_state);
        return cudaSuccess;
    }));
    return timed(g, "stage_sort", s, sort_pairs_launches(n, bits), [&]() {
        size_t tb = g->tmp_bytes;
        return sort_pairs_u64_u32(g->d_tmp, tb, g->d_kin, g->d_kout, g->d_iin, g->d_iout, n, bits, s);
    });
}

} // namespace

extern "C" {

mk_status mk_insert_batch(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, const uint32_t *d_w,
                          uint64_t n, uint8_t *d_inserted, void *stream)
{
    if (!g || (n > 0 && (!d_src || !d_dst)) || n >= 0xFFFFFFFFull)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->change_seq++;
    if (n == 0)
        return MK_OK;
    if (d_inserted)
        MK_CUDA(cudaMemsetAsync(d_inserted, 0, n, s));
    MK_TRY(stage(g, d_src, d_dst, d_w, n, s));
    g->ulog_bound = std::min<uint64_t>(g->v.H, g->ulog_bound + n);
    const uint32_t max_hops = g->v.P + 2;
    return timed(g, "insert", s, 2, [&]() {
        // the sort's input positions (d_iin) are free now: they hold the log nominations
        k_insert<<<grid_for(n, 256), 256, 0, s>>>(g->v, g->d_kout, g->d_iout, d_w, n, g->vbits, d_inserted, max_hops,
                                                  g->d_iin);
        k_log_updated<<<grid_for(n, 256), 256, 0, s>>>(g->v, g->d_iin, n);
        return cudaSuccess;
    });
}

mk_status mk_delete_batch(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                          uint8_t *d_deleted, void *stream)
{
    if (!g || (n > 0 && (!d_src || !d_dst)) || n >= 0xFFFFFFFFull)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
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
        k_delete<<<grid_for(n, 256), 256, 0, s>>>(g->v, g->d_kout, g->d_iout, n, g->vbits, d_deleted, g->d_dlog,
                                                  (uint32_t)g->dlog_cap, max_hops);
        return cudaSuccess;
    });
}

} // extern "C"
