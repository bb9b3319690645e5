// Bulk asynchronous copies (the TMA unit's untiled cp.async.bulk) from
// global into shared memory, completed through a shared-memory mbarrier, for
// the kernels that stream the whole slab array.  Inline PTX for sm_103a.
//
// Rules kept by the callers: source and destination 16-byte aligned, sizes a
// multiple of 16 bytes (whole 128-byte slabs); one thread arms a barrier with
// the byte count of the copy it issues (arrive.expect_tx, arrival count 1);
// a buffer is refilled only after every thread that read it has passed a
// __syncwarp, and the proxy fence orders those generic-proxy reads before the
// async-proxy write.  Every wait is bounded.
#pragma once

#include <cstdint>

#include "mk_device.cuh"

namespace mk {

__device__ __forceinline__ uint32_t smem_addr(const void *p)
{
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_addr(bar)), "r"(count) : "memory");
}

// Makes initialised barriers visible to the async proxy.
__device__ __forceinline__ void mbar_init_fence()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

// Orders this thread's earlier shared-memory accesses (generic proxy) before
// later bulk copies (async proxy) into the same buffer.
__device__ __forceinline__ void fence_proxy_async_smem()
{
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// The arming thread's arrival, announcing `bytes` of copies on this phase.
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_addr(bar)), "r"(bytes)
                 : "memory");
}

// Copies `bytes` from global `src` to shared `dst`; completion is counted on
// `bar`.  A CTA launched without clusters is its own cluster, so its shared
// addresses are valid shared::cluster addresses.
__device__ __forceinline__ void bulk_copy_g2s(void *dst, const void *src, uint32_t bytes, uint64_t *bar)
{
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                     smem_addr(dst)),
                 "l"(src), "r"(bytes), "r"(smem_addr(bar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t done;
    asm volatile("{\n\t.reg .pred p;\n\t"
                 "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
                 "selp.u32 %0, 1, 0, p;\n\t}"
                 : "=r"(done)
                 : "r"(smem_addr(bar)), "r"(parity)
                 : "memory");
    return done != 0;
}

// Waits until the phase with the given parity of `bar` has completed; gives
// up after `limit` polls (each try_wait may itself suspend the thread for a
// while) and returns false.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, uint32_t limit)
{
    for (uint32_t i = 0; i < limit; ++i)
        if (mbar_try_wait(bar, parity))
            return true;
    return false;
}

// Streaming scans over the whole slab array (static WCC, decremental
// relax-into-invalid).  Each warp walks chunks of 32 consecutive slabs
// (chunk k of warp w starts at slab (w + k * warps) * 32).  For every chunk
// the warp reads the 32 owners (per-slab source, kNil for an unused pool
// slab) and copies only the slabs the caller keeps, compacted, into one of
// two 4 KB shared-memory buffers: each such lane issues one 128-byte bulk
// copy, all completing on the buffer's mbarrier.  The copies of chunk k+1
// are issued before chunk k is processed, the caller's per-owner gather
// (aux, which decides what is kept) runs two chunks ahead and the owners
// three, so slab data, owners and gathers are in flight while the warp
// works.
constexpr uint32_t kScanWarps = 4;               // warps per block of a scan kernel
constexpr uint32_t kScanChunk = 32;              // slabs per chunk
constexpr uint32_t kScanWaitLimit = 1u << 20;    // polls of one chunk's barrier

struct ScanSmem {
    uint4 buf[kScanWarps][2][kScanChunk * 8];    // compacted slabs, 16 B per uint4
    uint64_t bar[kScanWarps][2];
    uint8_t comp[kScanWarps][2][kScanChunk];     // compacted position -> lane of its owner
};

// Scans every slab of the array.  aux_fn(owner) -> Aux (any register-sized
// value type) is evaluated per lane two chunks ahead (kNil owners
// included); a slab is copied and
// processed only if its owner is not kNil and keep_fn(aux) holds.
// chunk_fn(buf, comp, n, owner, aux) processes one chunk: buf holds its n
// kept slabs (slab j at buf[8j .. 8j+7]) and comp[j] the lane whose owner /
// aux belong to slab j.  Returns false if a wait timed out (the copies still
// in flight were then given a bounded time to land).  Must be called by
// full warps; the barriers are initialised here.
template <typename AuxFn, typename KeepFn, typename ChunkFn>
__device__ __forceinline__ bool scan_slab_chunks(const GView &g, ScanSmem &sm, AuxFn &&aux_fn, KeepFn &&keep_fn,
                                                 ChunkFn &&chunk_fn)
{
    const uint32_t lane = lane_id(), w = threadIdx.x >> 5;
    const uint64_t total = (uint64_t)g.H + g.P;
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t stride = (((uint64_t)gridDim.x * blockDim.x) >> 5) * kScanChunk;
    if (lane == 0) {
        mbar_init(&sm.bar[w][0], 1);
        mbar_init(&sm.bar[w][1], 1);
        mbar_init_fence();
    }
    __syncwarp();
    auto owner_of = [&](uint64_t c) -> uint32_t { return c + lane < total ? __ldcg(&g.owner[c + lane]) : kNil; };
    // copies chunk c's kept slabs into buffer b; returns how many
    using Aux = decltype(aux_fn(0u));
    auto issue = [&](uint64_t c, uint32_t own, const Aux &aux, uint32_t b) -> uint32_t {
        if (c >= total)
            return 0;
        const bool keep = own != kNil && keep_fn(aux);
        const uint32_t live = __ballot_sync(kFull, keep);
        if (lane == 0) {
            fence_proxy_async_smem(); // the warp's reads of this buffer (ordered by __syncwarp) first
            mbar_arrive_expect_tx(&sm.bar[w][b], __popc(live) * 128u);
        }
        __syncwarp();
        if (keep) {
            const uint32_t pos = __popc(live & ((1u << lane) - 1));
            sm.comp[w][b][pos] = (uint8_t)lane;
            bulk_copy_g2s(&sm.buf[w][b][pos * 8], slab_ptr(g, (uint32_t)(c + lane)), 128u, &sm.bar[w][b]);
        }
        return __popc(live);
    };
    uint64_t c = warp0 * kScanChunk;
    uint32_t own0 = owner_of(c), own1 = owner_of(c + stride), own2 = owner_of(c + 2 * stride);
    Aux aux0 = aux_fn(own0);
    uint32_t n0 = issue(c, own0, aux0, 0);
    Aux aux1 = aux_fn(own1);
    uint32_t k = 0;
    bool ok = true;
    for (; c < total; c += stride, ++k) {
        const uint32_t b = k & 1;
        const uint32_t n1 = issue(c + stride, own1, aux1, b ^ 1);
        const Aux aux2 = aux_fn(own2);
        const uint32_t own3 = owner_of(c + 3 * stride);
        ok = __all_sync(kFull, mbar_wait(&sm.bar[w][b], (k >> 1) & 1, kScanWaitLimit));
        if (!ok)
            break;
        __syncwarp();
        chunk_fn(sm.buf[w][b], sm.comp[w][b], n0, own0, aux0);
        __syncwarp();
        own0 = own1;
        n0 = n1;
        aux0 = aux1;
        own1 = own2;
        aux1 = aux2;
        own2 = own3;
    }
    if (!ok) {
        mbar_wait(&sm.bar[w][k & 1], (k >> 1) & 1, kScanWaitLimit);
        if (c + stride < total)
            mbar_wait(&sm.bar[w][(k + 1) & 1], ((k + 1) >> 1) & 1, kScanWaitLimit);
    }
    return ok;
}

} // namespace mk
