// mk_insert_batch_noalloc: the batched insert of update.cu with its staging
// scratch (the batch's hash set of (src, dst) pairs, each edge's entry and
// the updated-list nominations) taken from one fixed device array declared
// in this file instead of buffers grown with cudaMalloc.  The graph itself
// must already exist; this call allocates nothing, on the device or on the
// host.
//
// Why: mk_insert_batch grows its staging buffers on demand, and growing them
// calls cudaStreamSynchronize, cudaFree and cudaMalloc, which stall the
// device and may fail.  Some callers cannot do that: a serving loop that must
// never synchronise the device between requests, and a process whose device
// memory is handed out by another allocator (a framework's caching allocator)
// or fixed at start-up, where an extra cudaMalloc can fail or break the
// budget.  They can use this entry point for batches of up to
// kNoAllocMaxBatch edges.
#include "mk_host.h"

#include <algorithm>
#include <mutex>

using namespace mk;

// Kernels of update.cu, launched here unchanged.
__global__ void k_dedup(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                        const uint32_t *__restrict__ w, uint64_t n, uint32_t V, uint32_t *tpos, uint32_t mask,
                        uint32_t *__restrict__ slot, DevState *st);
__global__ void __launch_bounds__(256, 6) k_insert(GView g, const uint32_t *__restrict__ src,
                                                   const uint32_t *__restrict__ dst, const uint32_t *__restrict__ w_in,
                                                   uint64_t n, const uint32_t *__restrict__ tpos,
                                                   const uint32_t *__restrict__ slot, uint8_t *__restrict__ flags,
                                                   uint32_t max_hops, uint32_t *__restrict__ cand);
__global__ void __launch_bounds__(256) k_log_updated(GView g, const uint32_t *__restrict__ cand, uint64_t n,
                                                     const uint8_t *__restrict__ stored, const uint32_t *__restrict__ src,
                                                     const uint32_t *__restrict__ dst, const uint32_t *__restrict__ w,
                                                     uint4 *ilog, uint32_t ilog_cap);

namespace {

constexpr uint64_t kNoAllocMaxBatch = MK_NOALLOC_MAX_BATCH;
static_assert(kNoAllocMaxBatch == (1ull << 16), "the scratch layout below is sized for 2^16 edges");
constexpr uint64_t kTable = 2 * kNoAllocMaxBatch;            // hash-set entries (a power of two)
constexpr size_t kTposBytes = kTable * 4;
constexpr size_t kEdgeBytes = kNoAllocMaxBatch * 4;
constexpr size_t kScratchBytes = kTposBytes + 2 * kEdgeBytes; // 1 MiB

} // namespace

// The scratch of every call on a device.  Device code could name it
// directly; host code must not pass `g_noalloc_scratch` itself to a kernel
// (on the host it is only a stand-in symbol), so its device address is looked
// up with cudaGetSymbolAddress at set-up, once per device (with that device
// current), and that address is passed to the kernels.  Every GPU that
// loads this library holds the array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

typedef int (*CtxGetCurrentFn)(void **ctx);

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
struct DeviceSetup {
    bool done = false;
    void *ctx = nullptr;          // context the address belongs to
    unsigned char *addr = nullptr;
};
DeviceSetup g_setup[kMaxDevices];

// The calling thread's current context, from the driver's cuCtxGetCurrent
// fetched through the runtime (so the library needs no link against the
// driver library); nullptr if it cannot be had.
void *current_context()
{
    static CtxGetCurrentFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q = cudaDriverEntryPointSymbolNotFound;
        if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (CtxGetCurrentFn)p;
        cudaGetLastError();
    }
    void *ctx = nullptr;
    if (fn && fn(&ctx) != 0)
        ctx = nullptr;
    return ctx;
}

// The array's device address on the current device.  The set-up (the
// lookup) runs on the first call on each device, and again if that
// device's context is no longer the one the address was taken in (after a
// cudaDeviceReset the module, and the array, may be loaded elsewhere).  The
// first lookup may make the runtime load this library's device code on the
// device, which is why the first call on a device belongs before any stream
// capture; nothing else here allocates.
mk_status scratch_base(unsigned char **base)
{
    int dev = 0;
    MK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return MK_ERR_INTERNAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    DeviceSetup &d = g_setup[dev];
    void *ctx = current_context();
    if (!d.done || ctx != d.ctx) {
        void *p = nullptr;
        const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return MK_ERR_CUDA;
        }
        d.addr = (unsigned char *)p;
        d.ctx = current_context(); // the lookup may have created the context
        d.done = true;
    }
    *base = d.addr;
    return MK_OK;
}

} // namespace

extern "C" mk_status mk_insert_batch_noalloc(mk_graph *g, const uint32_t *d_src, const uint32_t *d_dst,
                                             const uint32_t *d_w, uint64_t n, uint8_t *d_inserted, void *stream)
{
    if (!g || (n > 0 && (!d_src || !d_dst)))
        return MK_ERR_INVALID_ARG;
    if (n > kNoAllocMaxBatch)
        return MK_ERR_INVALID_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    unsigned char *base = nullptr;
    MK_TRY(scratch_base(&base));
    g->change_seq++;
    if (n == 0)
        return MK_OK;
    uint32_t *tpos = (uint32_t *)base;
    uint32_t *slot = (uint32_t *)(base + kTposBytes);
    uint32_t *cand = (uint32_t *)(base + kTposBytes + kEdgeBytes);
    // the hash set must start empty (all-ones positions); slots and
    // nominations are written in full before they are read; the caller's
    // flags are cleared
    MK_CUDA(cudaMemsetAsync(tpos, 0xFF, kTposBytes, s));
    if (d_inserted)
        MK_CUDA(cudaMemsetAsync(d_inserted, 0, n, s));
    // launched without the profiling hook (which creates events and grows
    // a host vector): with profiling on, these kernels are counted in the
    // launch total but missing from the per-kernel times
    k_dedup<<<grid_for(n, 256), 256, 0, s>>>(d_src, d_dst, d_w, n, g->v.V, tpos, (uint32_t)(kTable - 1), slot,
                                             g->d_state);
    g->ulog_bound = std::min<uint64_t>(g->v.H, g->ulog_bound + n);
    const uint32_t max_hops = g->v.P + 2;
    k_insert<<<grid_for(n, 256), 256, 0, s>>>(g->v, d_src, d_dst, d_w, n, tpos, slot, d_inserted, max_hops, cand);
    // no inserted-edge log (growing it could allocate): this epoch's
    // incremental prologues walk the updated lists instead
    g->ilog_ok = false;
    k_log_updated<<<grid_for(n, 256), 256, 0, s>>>(g->v, cand, n, nullptr, nullptr, nullptr, nullptr, nullptr, 0);
    g->launches += 3;
    MK_CUDA(cudaGetLastError());
    return MK_OK;
}
