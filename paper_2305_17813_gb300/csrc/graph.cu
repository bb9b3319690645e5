// Graph object: creation with one head-slab allocation, the slab pool, the
// per-list update metadata, UpdateSlabPointers, export and statistics.
#include "mk_host.h"

#include <vector>

#include <algorithm>
#include <cstring>

using namespace mk;

namespace mk {

mk_status device_alloc(mk_graph *g, void **p, size_t bytes)
{
    *p = nullptr;
    if (bytes == 0)
        return MK_OK;
    cudaError_t e = cudaMalloc(p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return e == cudaErrorMemoryAllocation ? MK_ERR_NO_MEMORY : MK_ERR_CUDA;
    }
    if (g)
        g->bytes += bytes;
    return MK_OK;
}

void device_free(mk_graph *g, void *p, size_t bytes)
{
    if (p) {
        cudaFree(p);
        if (g)
            g->bytes -= bytes;
    }
}

// Grows the staging buffers to hold n batch entries (keys, indices and the
// radix-sort workspace for the widest key).
mk_status ensure_scratch(mk_graph *g, uint64_t n, cudaStream_t s)
{
    if (n <= g->scratch_cap)
        return MK_OK;
    uint64_t cap = std::max<uint64_t>(n, 1024);
    cap = std::max<uint64_t>(cap, g->scratch_cap + g->scratch_cap / 2);
    uint64_t table = 1;
    while (table < 2 * cap)
        table <<= 1;
    MK_CUDA(cudaStreamSynchronize(s));
    device_free(g, g->d_tpos, g->table_size * 4);
    device_free(g, g->d_slot, g->scratch_cap * 4);
    device_free(g, g->d_cand, g->scratch_cap * 4);
    device_free(g, g->d_iflags, g->scratch_cap);
    g->d_tpos = g->d_slot = g->d_cand = nullptr;
    g->d_iflags = nullptr;
    g->scratch_cap = g->table_size = 0;
    MK_TRY(device_alloc(g, (void **)&g->d_tpos, table * 4));
    MK_TRY(device_alloc(g, (void **)&g->d_slot, cap * 4));
    MK_TRY(device_alloc(g, (void **)&g->d_cand, cap * 4));
    MK_TRY(device_alloc(g, (void **)&g->d_iflags, cap));
    g->table_size = table;
    g->scratch_cap = cap;
    return MK_OK;
}

} // namespace mk

// ------------------------------------------------------------------ kernels

// Fills slabs [first, first + count) with the empty pattern: free pairs,
// unused lane 30 and a null next pointer.
__global__ void k_init_slabs(uint32_t *slabs, uint64_t first, uint64_t count)
{
    const uint64_t words = count * 32;
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < words;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t lane = (uint32_t)(i & 31);
        slabs[first * 32 + i] = is_key_lane(lane) ? kEmptyKey : kFull;
    }
}

__global__ void k_fill_buckets(uint32_t *b, uint32_t V, uint32_t nb, const uint32_t *user, int *bad)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V)
        return;
    uint32_t x = user ? user[v] : nb;
    if (x == 0) {
        *bad = 1;
        x = 1;
    }
    b[v] = x;
}

__global__ void k_set_vinfo(uint2 *vinfo, const uint32_t *b, const uint64_t *off, uint32_t V)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v < V)
        vinfo[v] = make_uint2((uint32_t)off[v], b[v]);
}

// Per list: its source vertex (also the owner of its head slab), marker at
// lane 0 of its head slab, not updated.
__global__ void k_init_lists(const uint2 *vinfo, uint32_t V, uint32_t *list_src, unsigned long long *lmark,
                             uint8_t *lupd, uint32_t *owner)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V)
        return;
    const uint2 vi = vinfo[v];
    for (uint32_t b = 0; b < vi.y; ++b) {
        const uint32_t l = vi.x + b;
        list_src[l] = v;
        owner[l] = v;
        lmark[l] = (unsigned long long)l << 32;
        lupd[l] = 0;
    }
}

__global__ void k_init_bitmap(uint32_t *bitmap, uint32_t words, uint32_t P)
{
    const uint32_t i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= words)
        return;
    uint32_t w = 0;
    const uint64_t lo = (uint64_t)i * 32;
    if (lo + 32 > P) {
        const uint32_t valid = (uint32_t)(P - lo);
        w = valid >= 32 ? 0u : ~((1u << valid) - 1u);
    }
    bitmap[i] = w;
}

__global__ void k_degree(const uint32_t *src, uint64_t n, uint32_t V, uint32_t *deg, int *bad)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n; i += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t s = src[i];
        if (s < V)
            atomicAdd(&deg[s], 1u);
        else
            *bad = 1;
    }
}

__global__ void k_rule(uint32_t *deg, uint32_t V, float per_bucket)
{
    const uint32_t v = blockIdx.x * blockDim.x + threadIdx.x;
    if (v >= V)
        return;
    const double want = (double)deg[v] / (double)per_bucket;
    uint32_t b = (uint32_t)ceil(want);
    deg[v] = b < 1 ? 1 : b;
}

// UpdateSlabPointers (paper, Sec. "Graph Primitives", Fig.
// "UpdateSlabPointers()"): for every updated list, walk from its marker slab
// to the last slab; the new marker is that slab and the first free key lane
// in it, or kInvalidLane when it is full; the updated flag is cleared.  The
// updated lists are read from the updated-list log; every 4-lane group of
// every warp takes one logged list at a time (eight per warp) and walks it
// with two 16-byte loads per lane (lane s4 holds words 8*s4 .. 8*s4+7).
__global__ void __launch_bounds__(256) k_update_slab_pointers(GView g, uint32_t max_hops)
{
    const uint32_t lane = lane_id(), s4 = lane & 3u, gi = lane >> 2, gbase = lane & ~3u;
    const uint32_t n = min(__ldg(&g.st->ulog_count), g.H);
    const uint64_t warp0 = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t gs = (((uint64_t)gridDim.x * blockDim.x) >> 5) * 8;
    unsigned long long loads = 0;
    for (uint64_t base = warp0 * 8; base < n; base += gs) {
        const uint64_t i = base + gi;
        const uint32_t list = i < n ? g.ulog[i] : kNil;
        uint32_t slab = list != kNil ? (uint32_t)(g.lmark[list] >> 32) : kNil;
        bool active = slab != kNil;
        uint4 lo = make_uint4(kEmptyKey, kFull, kFull, kFull), hi = lo;
        for (uint32_t hop = 0; __any_sync(kFull, active); ++hop) {
            if (active) {
                const uint4 *p = reinterpret_cast<const uint4 *>(slab_ptr(g, slab) + s4 * 8);
                lo = __ldcg(p);
                hi = __ldcg(p + 1);
            }
            loads += __popc(__ballot_sync(kFull, active && s4 == 0));
            const uint32_t nxt = __shfl_sync(kFull, hi.w, gbase + 3);
            if (active) {
                if (nxt == kNil || hop + 1 >= max_hops)
                    active = false; // (lo, hi) keep the last slab
                else
                    slab = nxt;
            }
        }
        // first free key lane of the last slab: key words 8*s4, +2, +4, +6
        // (word 30, lane 3's seventh word, is not a key lane)
        const uint32_t w0 = 8 * s4;
        uint32_t fl = lo.x == kEmptyKey   ? w0
                      : lo.z == kEmptyKey ? w0 + 2
                      : hi.x == kEmptyKey ? w0 + 4
                      : (s4 != 3u && hi.z == kEmptyKey) ? w0 + 6
                                                        : 32u;
        fl = min(fl, __shfl_xor_sync(kFull, fl, 2));
        fl = min(fl, __shfl_xor_sync(kFull, fl, 1));
        if (s4 == 0 && list != kNil) {
            g.lmark[list] = ((unsigned long long)slab << 32) | (fl < 32 ? fl : (uint32_t)kInvalidLane);
            g.lupd[list] = 0;
        }
    }
    count_add(g.st, kCtrCommitSlabs, loads);
}

// Per-list chain statistics (one warp per list).
struct ChainStats {
    unsigned long long chain_slabs, live, tomb, max_chain;
};

__global__ void k_chain_stats(GView g, ChainStats *out, uint32_t max_hops)
{
    const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = lane_id();
    if (w >= g.H)
        return;
    uint32_t slab = (uint32_t)w;
    unsigned long long nslab = 0, live = 0, tomb = 0;
    for (uint32_t hop = 0; hop < max_hops && slab != kNil; ++hop) {
        const uint32_t v = slab_ptr(g, slab)[lane];
        const bool key = is_key_lane(lane);
        live += __popc(__ballot_sync(kFull, key && v < kTombKey));
        tomb += __popc(__ballot_sync(kFull, key && v == kTombKey));
        ++nslab;
        slab = __shfl_sync(kFull, v, kNextLane);
    }
    if (lane == 0) {
        atomicAdd(&out->chain_slabs, nslab);
        atomicAdd(&out->live, live);
        atomicAdd(&out->tomb, tomb);
        atomicMax(&out->max_chain, nslab);
    }
}

__global__ void k_popcount(const uint32_t *bitmap, uint32_t words, uint32_t P, unsigned long long *out)
{
    unsigned long long c = 0;
    for (uint32_t i = blockIdx.x * blockDim.x + threadIdx.x; i < words; i += gridDim.x * blockDim.x) {
        uint32_t w = bitmap[i];
        const uint64_t lo = (uint64_t)i * 32;
        if (lo + 32 > P) {
            const uint32_t valid = (uint32_t)(P - lo);
            if (valid < 32)
                w &= (1u << valid) - 1u;
        }
        c += __popc(w);
    }
    atomicAdd(out, c);
}

// Export: live pairs per list, then (key, weight) at the list's offset.
__global__ void k_count_live(GView g, uint32_t *cnt, uint32_t max_hops)
{
    const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = lane_id();
    if (w >= g.H)
        return;
    uint32_t slab = (uint32_t)w, c = 0;
    for (uint32_t hop = 0; hop < max_hops && slab != kNil; ++hop) {
        const uint32_t v = slab_ptr(g, slab)[lane];
        c += __popc(__ballot_sync(kFull, is_key_lane(lane) && v < kTombKey));
        slab = __shfl_sync(kFull, v, kNextLane);
    }
    if (lane == 0)
        cnt[w] = c;
}

__global__ void k_write_live(GView g, const uint64_t *off, uint64_t *keys, uint32_t *wts, uint32_t vbits,
                             uint32_t max_hops)
{
    const uint64_t w = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint32_t lane = lane_id();
    if (w >= g.H)
        return;
    const uint32_t src = g.list_src[w];
    uint64_t at = off[w];
    uint32_t slab = (uint32_t)w;
    for (uint32_t hop = 0; hop < max_hops && slab != kNil; ++hop) {
        const uint32_t v = slab_ptr(g, slab)[lane];
        const uint32_t wt = __shfl_down_sync(kFull, v, 1);
        const bool live = is_key_lane(lane) && v < kTombKey;
        const uint32_t m = __ballot_sync(kFull, live);
        if (live) {
            const uint64_t i = at + __popc(m & lanemask_lt());
            keys[i] = ((uint64_t)src << vbits) | v;
            wts[i] = wt;
        }
        at += __popc(m);
        slab = __shfl_sync(kFull, v, kNextLane);
    }
}

__global__ void k_decode_export(const uint64_t *keys, const uint32_t *wts, uint64_t m, uint64_t cap, uint32_t vbits,
                                uint32_t *src, uint32_t *dst, uint32_t *w, uint64_t *count)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i == 0)
        *count = m;
    if (i >= m || i >= cap)
        return;
    const uint64_t k = keys[i];
    if (src)
        src[i] = (uint32_t)(k >> vbits);
    if (dst)
        dst[i] = (uint32_t)(k & ((1ull << vbits) - 1));
    if (w)
        w[i] = wts[i];
}

__global__ void k_clear_logs(DevState *st)
{
    st->dlog_count = 0;
    st->ulog_count = 0;
    st->ilog_count = 0;
}

// ---------------------------------------------------------------- host API

static uint32_t bits_for(uint32_t V)
{
    uint32_t b = 1;
    while (b < 32 && (1ull << b) < (uint64_t)V)
        ++b;
    return b;
}

static void destroy_consumer(mk_graph *g, Consumer *c)
{
    const size_t V = g->v.V, H = g->v.H;
    device_free(g, c->D, V * 8);
    device_free(g, c->front[0], H * 8);
    device_free(g, c->front[1], H * 8);
    device_free(g, c->stamp, V * 4);
    device_free(g, c->inv, (V + 31) / 32 * 4);
    device_free(g, c->uf, V * 4);
    device_free(g, c->far[0], V * 4);
    device_free(g, c->far[1], V * 4);
    device_free(g, c->fstamp, V * 4);
    device_free(g, c->counters, 64);
    delete c;
}

extern "C" {

const char *mk_version(void) { return "meerkat-gb300 0.1 (sm_103a)"; }

uint64_t mk_launch_count(mk_graph *g) { return g ? g->launches : 0; }

mk_status mk_bucket_rule(uint32_t V, const uint32_t *d_src, uint64_t n, float load_factor, uint32_t *d_buckets,
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
    k_rule<<<grid_for(V, 256), 256, 0, s>>>(d_buckets, V, load_factor * 15.f);
    int bad = 0;
    MK_CUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaFreeAsync(d_bad, s));
    MK_CUDA(cudaStreamSynchronize(s));
    return bad ? MK_ERR_INVALID_ARG : MK_OK;
}

mk_status mk_graph_create_ex(const mk_config *cfg, void *stream, mk_graph **out)
{
    if (!cfg || !out || cfg->V == 0 || cfg->V > 0xFFFFFFFDu)
        return MK_ERR_INVALID_ARG;
    *out = nullptr;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t V = cfg->V;
    mk_graph *g = new mk_graph;
    g->vbits = bits_for(V);
    auto fail = [&](mk_status st) {
        mk_graph_destroy(g);
        return st;
    };
    uint32_t *d_b = nullptr;
    uint64_t *d_off = nullptr;
    int *d_bad = nullptr;
    mk_status st = MK_OK;
    st = device_alloc(nullptr, (void **)&d_b, (size_t)V * 4);
    if (st == MK_OK)
        st = device_alloc(nullptr, (void **)&d_off, (size_t)V * 8);
    if (st == MK_OK)
        st = device_alloc(nullptr, (void **)&d_bad, sizeof(int));
    if (st != MK_OK) {
        device_free(nullptr, d_b, 0);
        device_free(nullptr, d_off, 0);
        device_free(nullptr, d_bad, 0);
        return fail(st);
    }
    auto cleanup_tmp = [&]() {
        device_free(nullptr, d_b, 0);
        device_free(nullptr, d_off, 0);
        device_free(nullptr, d_bad, 0);
        d_b = nullptr;
    };
    cudaMemsetAsync(d_bad, 0, sizeof(int), s);
    k_fill_buckets<<<grid_for(V, 256), 256, 0, s>>>(d_b, V, cfg->buckets ? cfg->buckets : 1,
                                                       cfg->d_bucket_per_vertex, d_bad);
    // exclusive scan of bucket counts -> head offsets (one allocation for
    // every head slab; paper, Sec. "Memory Management in Meerkat")
    void *d_tmp = nullptr;
    if (cudaMalloc(&d_tmp, exclusive_scan_scratch_bytes(V)) != cudaSuccess ||
        exclusive_scan_u32_u64(d_b, d_off, V, d_tmp, s, nullptr) != cudaSuccess) {
        cudaFree(d_tmp);
        cleanup_tmp();
        return fail(MK_ERR_CUDA);
    }
    uint64_t last_off = 0;
    uint32_t last_b = 0;
    int bad = 0;
    cudaMemcpyAsync(&last_off, d_off + (V - 1), 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&last_b, d_b + (V - 1), 4, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&bad, d_bad, 4, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaFree(d_tmp);
        cleanup_tmp();
        return fail(MK_ERR_CUDA);
    }
    cudaFree(d_tmp);
    const uint64_t H = last_off + last_b;
    uint64_t P = cfg->pool_slabs;
    if (P == 0)
        P = cfg->edge_capacity_hint / 15 + H / 8 + 1024;
    P = (P + 31) / 32 * 32;
    if (bad || H + P >= 0xFFFFFFFFull) {
        cleanup_tmp();
        return fail(MK_ERR_INVALID_ARG);
    }
    GView &v = g->v;
    v.V = V;
    v.H = (uint32_t)H;
    v.P = (uint32_t)P;
    v.pool_words = (uint32_t)(P / 32);
    st = device_alloc(g, (void **)&v.vinfo, (size_t)V * 8);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&v.slabs, (size_t)(H + P) * 128);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&v.bitmap, (size_t)v.pool_words * 4 + 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&v.list_src, (size_t)H * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&v.lmark, (size_t)H * 8);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&v.lupd, ((size_t)H + 3) & ~(size_t)3);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&v.ulog, (size_t)H * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&v.owner, (size_t)(H + P) * 4);
    if (st == MK_OK)
        st = device_alloc(g, (void **)&g->d_state, sizeof(DevState));
    if (st == MK_OK && cudaMallocHost((void **)&g->h_pinned, 64) != cudaSuccess)
        st = MK_ERR_NO_MEMORY;
    if (st != MK_OK) {
        cleanup_tmp();
        return fail(st);
    }
    v.st = g->d_state;
    k_set_vinfo<<<grid_for(V, 256), 256, 0, s>>>((uint2 *)v.vinfo, d_b, d_off, V);
    k_init_slabs<<<std::min<uint64_t>(grid_for(H * 32, 256), 152 * 64), 256, 0, s>>>(v.slabs, 0, H);
    cudaMemsetAsync(v.owner + H, 0xFF, (size_t)P * 4, s);
    cudaMemsetAsync(v.lupd, 0, ((size_t)H + 3) & ~(size_t)3, s);
    k_init_lists<<<grid_for(V, 256), 256, 0, s>>>(v.vinfo, V, (uint32_t *)v.list_src, v.lmark, v.lupd, v.owner);
    k_init_bitmap<<<grid_for(v.pool_words, 256), 256, 0, s>>>(v.bitmap, v.pool_words, v.P);
    cudaMemsetAsync(g->d_state, 0, sizeof(DevState), s);
    g->launches += 5;
    cudaError_t e = cudaStreamSynchronize(s);
    cleanup_tmp();
    if (e != cudaSuccess || cudaGetLastError() != cudaSuccess)
        return fail(MK_ERR_CUDA);
    *out = g;
    return MK_OK;
}

mk_status mk_graph_create(uint32_t V, uint64_t edge_capacity_hint, uint32_t buckets,
                          const uint32_t *d_bucket_per_vertex, void *stream, mk_graph **out)
{
    mk_config c{};
    c.V = V;
    c.edge_capacity_hint = edge_capacity_hint;
    c.buckets = buckets;
    c.d_bucket_per_vertex = d_bucket_per_vertex;
    return mk_graph_create_ex(&c, stream, out);
}

mk_status mk_graph_destroy(mk_graph *g)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    cudaDeviceSynchronize();
    for (auto &kv : g->consumers)
        destroy_consumer(g, kv.second);
    g->consumers.clear();
    GView &v = g->v;
    cudaFree((void *)v.vinfo);
    cudaFree(v.slabs);
    cudaFree(v.bitmap);
    cudaFree((void *)v.list_src);
    cudaFree(v.lmark);
    cudaFree(v.lupd);
    cudaFree(v.ulog);
    cudaFree(v.owner);
    cudaFree(g->d_state);
    cudaFree(g->d_tpos);
    cudaFree(g->d_slot);
    cudaFree(g->d_cand);
    cudaFree(g->d_iflags);
    cudaFree(g->d_dlog);
    cudaFree(g->d_ilog);
    if (g->h_pinned)
        cudaFreeHost(g->h_pinned);
    for (auto &t : g->timed) {
        cudaEventDestroy(t.a);
        cudaEventDestroy(t.b);
    }
    for (auto e : g->spare_events)
        cudaEventDestroy(e);
    delete g;
    return MK_OK;
}

mk_status mk_commit_batch(mk_graph *g, void *stream)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint32_t max_hops = g->v.P + 2;
    MK_TRY(timed(g, "update_slab_pointers", s, 2, [&]() {
        // one 4-lane group per logged list
        const uint32_t grid = std::min<uint32_t>(grid_for(std::max<uint64_t>(g->ulog_bound, 1) * 4, 256), num_sms() * 16);
        k_update_slab_pointers<<<grid, 256, 0, s>>>(g->v, max_hops);
        k_clear_logs<<<1, 1, 0, s>>>(g->d_state);
        return cudaSuccess;
    }));
    // states that have applied every batch of this epoch stay incremental
    for (auto &kv : g->consumers) {
        Consumer *c = kv.second;
        if (c->epoch == g->epoch && c->seq == g->change_seq)
            c->epoch = g->epoch + 1;
    }
    g->epoch++;
    g->dlog_bound = 0;
    g->ulog_bound = 0;
    g->ilog_bound = 0;
    g->ilog_ok = true;
    g->epoch_has_deletes = false;
    return MK_OK;
}

mk_status mk_graph_export(mk_graph *g, uint64_t cap, uint32_t *d_src, uint32_t *d_dst, uint32_t *d_w,
                          uint64_t *d_count, void *stream)
{
    if (!g || !d_count)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    const uint64_t H = g->v.H;
    const uint32_t max_hops = g->v.P + 2;
    uint32_t *d_cnt = nullptr;
    uint64_t *d_off = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&d_cnt, (H + 1) * 4, s));
    MK_CUDA(cudaMallocAsync((void **)&d_off, (H + 1) * 8, s));
    MK_CUDA(cudaMemsetAsync(d_cnt + H, 0, 4, s));
    k_count_live<<<grid_for(H * 32, 256), 256, 0, s>>>(g->v, d_cnt, max_hops);
    void *d_tmp = nullptr;
    int scan_launches = 0;
    MK_CUDA(cudaMallocAsync(&d_tmp, exclusive_scan_scratch_bytes(H + 1), s));
    MK_CUDA(exclusive_scan_u32_u64(d_cnt, d_off, H + 1, d_tmp, s, &scan_launches));
    uint64_t m = 0;
    MK_CUDA(cudaMemcpyAsync(&m, d_off + H, 8, cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    uint64_t *k0 = nullptr, *k1 = nullptr;
    uint32_t *w0 = nullptr, *w1 = nullptr;
    const uint64_t mm = std::max<uint64_t>(m, 1);
    MK_CUDA(cudaMallocAsync((void **)&k0, mm * 8, s));
    MK_CUDA(cudaMallocAsync((void **)&k1, mm * 8, s));
    MK_CUDA(cudaMallocAsync((void **)&w0, mm * 4, s));
    MK_CUDA(cudaMallocAsync((void **)&w1, mm * 4, s));
    k_write_live<<<grid_for(H * 32, 256), 256, 0, s>>>(g->v, d_off, k0, w0, g->vbits, max_hops);
    size_t tb2 = 0;
    MK_CUDA(sort_pairs_u64_u32(nullptr, tb2, k0, k1, w0, w1, m, 2 * g->vbits, s));
    void *d_tmp2 = nullptr;
    MK_CUDA(cudaMallocAsync(&d_tmp2, std::max<size_t>(tb2, 1), s));
    if (m)
        MK_CUDA(sort_pairs_u64_u32(d_tmp2, tb2, k0, k1, w0, w1, m, 2 * g->vbits, s));
    k_decode_export<<<grid_for(mm, 256), 256, 0, s>>>(k1, w1, m, cap, g->vbits, d_src, d_dst, d_w, d_count);
    g->launches += 4 + scan_launches + sort_pairs_launches(m, 2 * g->vbits);
    cudaFreeAsync(d_cnt, s);
    cudaFreeAsync(d_off, s);
    cudaFreeAsync(d_tmp, s);
    cudaFreeAsync(d_tmp2, s);
    cudaFreeAsync(k0, s);
    cudaFreeAsync(k1, s);
    cudaFreeAsync(w0, s);
    cudaFreeAsync(w1, s);
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}

mk_status mk_graph_stats(mk_graph *g, mk_stats *out, void *stream)
{
    if (!g || !out)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    ChainStats *d_cs = nullptr;
    unsigned long long *d_pop = nullptr;
    MK_CUDA(cudaMallocAsync((void **)&d_cs, sizeof(ChainStats), s));
    MK_CUDA(cudaMallocAsync((void **)&d_pop, 8, s));
    MK_CUDA(cudaMemsetAsync(d_cs, 0, sizeof(ChainStats), s));
    MK_CUDA(cudaMemsetAsync(d_pop, 0, 8, s));
    k_chain_stats<<<grid_for((uint64_t)g->v.H * 32, 256), 256, 0, s>>>(g->v, d_cs, g->v.P + 2);
    k_popcount<<<std::min<uint32_t>(grid_for(g->v.pool_words, 256), 1024), 256, 0, s>>>(g->v.bitmap, g->v.pool_words,
                                                                                         g->v.P, d_pop);
    g->launches += 2;
    ChainStats cs{};
    unsigned long long pop = 0;
    MK_CUDA(cudaMemcpyAsync(&cs, d_cs, sizeof cs, cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaMemcpyAsync(&pop, d_pop, 8, cudaMemcpyDeviceToHost, s));
    cudaFreeAsync(d_cs, s);
    cudaFreeAsync(d_pop, s);
    MK_CUDA(cudaStreamSynchronize(s));
    std::memset(out, 0, sizeof *out);
    out->V = g->v.V;
    out->lists = g->v.H;
    out->pool_slabs = g->v.P;
    out->pool_used = pop;
    out->chain_slabs = cs.chain_slabs;
    out->live_edges = cs.live;
    out->tombstones = cs.tomb;
    out->chain_max = (uint32_t)cs.max_chain;
    out->chain_mean = g->v.H ? (double)cs.chain_slabs / (double)g->v.H : 0.0;
    out->device_bytes = g->bytes;
    out->epoch = g->epoch;
    return MK_OK;
}

mk_status mk_last_error(mk_graph *g)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    // the whole device, not a remembered stream: a caller's stream may have
    // been destroyed since its last use
    if (cudaDeviceSynchronize() != cudaSuccess)
        return MK_ERR_CUDA;
    int st = 0;
    MK_CUDA(cudaMemcpy(&st, &g->d_state->status, sizeof(int), cudaMemcpyDeviceToHost));
    if (st != 0) {
        MK_CUDA(cudaMemset(&g->d_state->status, 0, sizeof(int)));
        // a call that failed on the device may have left its algorithm
        // state half updated: every state recomputes statically next time
        for (auto &kv : g->consumers)
            kv.second->epoch = ~0ull;
    }
    return st;
}

mk_status mk_debug_set(mk_graph *g, int knob, uint64_t value)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    switch (knob) {
    case MK_DEBUG_BARRIER_SPINS:
        g->dbg_barrier_spins = value ? std::min<uint64_t>(value - 1, 0xFFFFFFFFull) : ~0ull;
        return MK_OK;
    case MK_DEBUG_HOST_ROUNDS:
        g->dbg_host_rounds = value != 0;
        return MK_OK;
    default:
        return MK_ERR_INVALID_ARG;
    }
}

mk_status mk_set_sssp_delta(mk_graph *g, uint32_t delta_static, uint32_t delta_incremental)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    g->sssp_delta_static = delta_static;
    g->sssp_delta_incr = delta_incremental;
    return MK_OK;
}

mk_status mk_list_marker(mk_graph *g, uint32_t v, uint32_t bucket, uint32_t *slab, uint32_t *lane,
                         uint32_t *updated, void *stream)
{
    if (!g || v >= g->v.V || !slab || !lane || !updated)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    uint2 vi;
    MK_CUDA(cudaMemcpyAsync(&vi, g->v.vinfo + v, 8, cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    if (bucket >= vi.y)
        return MK_ERR_INVALID_ARG;
    unsigned long long m = 0;
    uint8_t u = 0;
    MK_CUDA(cudaMemcpyAsync(&m, g->v.lmark + vi.x + bucket, 8, cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaMemcpyAsync(&u, g->v.lupd + vi.x + bucket, 1, cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    *slab = (uint32_t)(m >> 32);
    *lane = (uint32_t)(m & 0xFF);
    *updated = u;
    return MK_OK;
}

mk_status mk_counters(mk_graph *g, uint64_t *out, int n, int reset, void *stream)
{
    if (!g || n < 0 || (n > 0 && !out))
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<unsigned long long> c((size_t)kNumCounters * kSlots);
    const size_t bytes = c.size() * sizeof(unsigned long long);
    MK_CUDA(cudaMemcpyAsync(c.data(), g->d_state->ctr, bytes, cudaMemcpyDeviceToHost, s));
    if (reset)
        MK_CUDA(cudaMemsetAsync(g->d_state->ctr, 0, bytes, s));
    MK_CUDA(cudaStreamSynchronize(s));
    for (int i = 0; i < n && i < (int)kNumCounters; ++i) {
        unsigned long long sum = 0;
        for (uint32_t k = 0; k < kSlots; ++k)
            sum += c[(size_t)i * kSlots + k];
        out[i] = sum;
    }
    return MK_OK;
}

mk_status mk_pool_free(mk_graph *g, uint64_t *out, void *stream)
{
    if (!g || !out)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    long long slots[kSlots];
    MK_CUDA(cudaMemcpyAsync(slots, g->d_state->pool_used, sizeof slots, cudaMemcpyDeviceToHost, s));
    MK_CUDA(cudaStreamSynchronize(s));
    long long used = 0;
    for (uint32_t k = 0; k < kSlots; ++k)
        used += slots[k];
    *out = used >= (long long)g->v.P ? 0 : g->v.P - (uint64_t)(used > 0 ? used : 0);
    return MK_OK;
}

mk_status mk_profile_enable(mk_graph *g, int on)
{
    if (!g)
        return MK_ERR_INVALID_ARG;
    g->prof = on != 0;
    return MK_OK;
}

mk_status mk_profile_read(mk_graph *g, mk_kernel_time *out, int cap, int *n_out)
{
    if (!g || !n_out || (cap > 0 && !out))
        return MK_ERR_INVALID_ARG;
    MK_CUDA(cudaDeviceSynchronize());
    std::vector<std::string> order;
    std::map<std::string, std::pair<uint64_t, double>> acc;
    for (auto &t : g->timed) {
        float ms = 0.f;
        cudaEventElapsedTime(&ms, t.a, t.b);
        if (!acc.count(t.name))
            order.push_back(t.name);
        acc[t.name].first++;
        acc[t.name].second += ms;
        g->spare_events.push_back(t.a);
        g->spare_events.push_back(t.b);
    }
    g->timed.clear();
    int n = 0;
    for (auto &name : order) {
        if (n < cap) {
            std::memset(&out[n], 0, sizeof(mk_kernel_time));
            std::strncpy(out[n].name, name.c_str(), sizeof(out[n].name) - 1);
            out[n].launches = acc[name].first;
            out[n].total_ms = acc[name].second;
        }
        ++n;
    }
    *n_out = std::min(n, cap);
    return MK_OK;
}

} // extern "C"
