// Batched edge query (paper, Sec. "Experimental Evaluation", query: the
// destination is hashed to one bucket of the source and only that chain is
// walked; the walk stops at the key, at the first free pair or at the end).
//
// Queries are independent, so the batch is not sorted.  One warp answers 32
// consecutive queries: each lane first fetches the source's bucket range for
// its own query (32 independent gathers in flight), then the warp walks four
// chains at a time, one per 8-lane group, each lane loading 16 bytes of the
// 128-byte slab (two pairs; the last lane of a group holds pair 14 and the
// next-slab lane).  The warp writes one bitmap word.
#include "mk_host.h"

using namespace mk;

template <int GROUP>
__global__ void __launch_bounds__(256) k_query(GView g, const uint32_t *__restrict__ src,
                                               const uint32_t *__restrict__ dst, uint64_t n,
                                               uint32_t *__restrict__ bitmap, uint32_t *__restrict__ w_out,
                                               uint32_t max_hops)
{
    static_assert(GROUP == 8, "8 lanes x 16 bytes per slab");
    constexpr uint32_t kGroups = 32 / GROUP;
    const uint32_t lane = lane_id();
    const unsigned long long warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t base = warp * 32;
    if (base >= n || read_status(g.st) != 0)
        return;
    // this lane's own query: source range -> head slab of its bucket
    const uint64_t q = base + lane;
    uint32_t my_d = kNil, my_head = kNil;
    bool bad = false;
    if (q < n) {
        const uint32_t s = __ldg(src + q);
        my_d = __ldg(dst + q);
        if (s < g.V && my_d < g.V) {
            const uint2 vi = __ldg(&g.vinfo[s]);
            my_head = vi.x + bucket_of(my_d, vi.y);
        } else {
            bad = true;
        }
    }
    if (__ballot_sync(kFull, bad) && lane == 0)
        set_status(g.st, kErrInvalid);
    const uint32_t gi = lane / GROUP, sub = lane % GROUP;
    const uint32_t gmask = ((1u << GROUP) - 1u) << (gi * GROUP);
    uint32_t word_bits = 0;
    unsigned long long loads = 0;
#pragma unroll 1
    for (uint32_t it = 0; it < 32 / kGroups; ++it) {
        const uint32_t who = it * kGroups + gi; // query handled by my group
        const uint32_t d = __shfl_sync(kFull, my_d, who);
        uint32_t slab = __shfl_sync(kFull, my_head, who);
        bool active = slab != kNil;
        bool found = false;
        for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
            loads += __popc(__ballot_sync(kFull, active && sub == 0));
            uint4 x = make_uint4(kNil, kNil, kNil, kNil);
            if (active)
                x = *reinterpret_cast<const uint4 *>(slab_ptr(g, slab) + sub * 4);
            const bool last = sub == GROUP - 1; // x.z is lane 30 (unused), x.w is the next lane
            const bool m0 = active && x.x == d;
            const bool m1 = active && !last && x.z == d;
            const uint32_t hit = __ballot_sync(kFull, m0 || m1) & gmask;
            const bool e0 = active && (x.x == kEmptyKey || (!last && x.z == kEmptyKey));
            const uint32_t emp = __ballot_sync(kFull, e0) & gmask;
            const uint32_t nxt = __shfl_sync(kFull, x.w, gi * GROUP + GROUP - 1);
            if (m0 || m1) {
                if (w_out)
                    w_out[base + who] = m0 ? x.y : x.w;
            }
            if (hit)
                found = true;
            if (active && (hit || emp || nxt == kNil || hop >= max_hops))
                active = false;
            else if (active)
                slab = nxt;
        }
        const uint32_t fb = __ballot_sync(kFull, sub == 0 && found);
        // bits at lanes 0, 8, 16, 24 -> query bits it*4 .. it*4+3
        uint32_t packed = 0;
#pragma unroll
        for (uint32_t k = 0; k < kGroups; ++k)
            packed |= ((fb >> (k * GROUP)) & 1u) << k;
        word_bits |= packed << (it * kGroups);
        if (w_out && sub == 0 && !found && base + who < n)
            w_out[base + who] = 0;
    }
    if (lane == 0)
        bitmap[warp] = word_bits;
    count_add(g.st, kCtrQuerySlabs, loads);
}

extern "C" mk_status mk_query_batch(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst, uint64_t n,
                                    uint32_t *d_bitmap, uint32_t *d_w, void *stream)
{
    if (!g || (n > 0 && (!d_src || !d_dst || !d_bitmap)) || n >= 0xFFFFFFFFull)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    g->last_stream = s;
    if (n == 0)
        return MK_OK;
    const uint32_t max_hops = g->v.P + 2;
    return timed(g, "query", s, 1, [&]() {
        k_query<8><<<grid_for(n, 256), 256, 0, s>>>(g->v, d_src, d_dst, n, d_bitmap, d_w, max_hops);
        return cudaSuccess;
    });
}
