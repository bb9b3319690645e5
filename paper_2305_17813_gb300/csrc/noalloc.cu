// mk_insert_batch_noalloc: the batched insert of update.cu with its staging
// scratch (sort keys, positions and the radix-sort workspace) taken from one
// fixed device array declared in this file instead of buffers grown with
// cudaMalloc.  The graph itself must already exist; this call allocates
// nothing, on the device or on the host.
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
__global__ void k_build_keys(const uint32_t *__restrict__ src, const uint32_t *__restrict__ dst,
                             const uint32_t *__restrict__ w, uint64_t n, uint32_t V, uint32_t vbits,
                             uint64_t *__restrict__ keys, uint32_t *__restrict__ idx, DevState *st);
__global__ void __launch_bounds__(256, 8) k_insert(GView g, const uint64_t *__restrict__ skey,
                                                const uint32_t *__restrict__ sidx, const uint32_t *__restrict__ w_in,
                                                uint64_t n, uint32_t vbits, uint8_t *__restrict__ flags,
                                                uint32_t max_hops, uint32_t *__restrict__ cand);
__global__ void __launch_bounds__(256) k_log_updated(GView g, const uint32_t *__restrict__ cand, uint64_t n);

namespace {

constexpr uint64_t kNoAllocMaxBatch = 1ull << 16;
constexpr size_t kKeyBytes = kNoAllocMaxBatch * 8;
constexpr size_t kIdxBytes = kNoAllocMaxBatch * 4;
constexpr size_t kSortWorkspace = 2u << 20;
constexpr size_t kScratchBytes = 2 * kKeyBytes + 2 * kIdxBytes + kSortWorkspace; // 3.5 MiB

} // namespace

// The scratch of every call on a device.  Device code could name it
// directly; host code must not pass `g_noalloc_scratch` itself to a kernel
// (on the host it is only a stand-in symbol), so its device address is looked
// up once per device with cudaGetSymbolAddress.  Every GPU that loads this
// library holds the array until the process exits.
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

namespace {

constexpr int kMaxDevices = 64;
std::mutex g_setup_mutex;
unsigned char *g_scratch_addr[kMaxDevices] = {};
bool g_setup_done[kMaxDevices] = {};

// Per-device set-up, done by the first call on each device (with that device
// current): the array's device address and a check that the radix sort's
// workspace for the largest batch fits the reserved part.  Neither step
// allocates.
mk_status setup_device(unsigned char **base)
{
    int dev = 0;
    MK_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= kMaxDevices)
        return MK_ERR_INTERNAL;
    std::lock_guard<std::mutex> lock(g_setup_mutex);
    if (!g_setup_done[dev]) {
        void *p = nullptr;
        cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
        if (e != cudaSuccess || p == nullptr) {
            cudaGetLastError();
            return MK_ERR_CUDA;
        }
        size_t need = 0;
        e = sort_pairs_u64_u32(nullptr, need, nullptr, nullptr, nullptr, nullptr, kNoAllocMaxBatch, 64, nullptr);
        if (e != cudaSuccess || need > kSortWorkspace)
            return MK_ERR_INTERNAL;
        g_scratch_addr[dev] = (unsigned char *)p;
        g_setup_done[dev] = true;
    }
    *base = g_scratch_addr[dev];
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
    MK_TRY(setup_device(&base));
    g->change_seq++;
    if (n == 0)
        return MK_OK;
    uint64_t *kin = (uint64_t *)base;
    uint64_t *kout = (uint64_t *)(base + kKeyBytes);
    uint32_t *iin = (uint32_t *)(base + 2 * kKeyBytes);
    uint32_t *iout = (uint32_t *)(base + 2 * kKeyBytes + kIdxBytes);
    void *work = base + 2 * kKeyBytes + 2 * kIdxBytes;
    // nothing in the scratch has to start at zero: keys and positions are
    // written in full before they are read, and the sort initialises its own
    // workspace; only the caller's flags are cleared
    if (d_inserted)
        MK_CUDA(cudaMemsetAsync(d_inserted, 0, n, s));
    const int bits = 2 * (int)g->vbits;
    MK_TRY(timed(g, "stage_keys", s, 1, [&]() {
        k_build_keys<<<grid_for(n, 256), 256, 0, s>>>(d_src, d_dst, d_w, n, g->v.V, g->vbits, kin, iin, g->d_state);
        return cudaSuccess;
    }));
    MK_TRY(timed(g, "stage_sort", s, sort_pairs_launches(n, bits), [&]() {
        size_t tb = kSortWorkspace;
        return sort_pairs_u64_u32(work, tb, kin, kout, iin, iout, n, bits, s);
    }));
    g->ulog_bound = std::min<uint64_t>(g->v.H, g->ulog_bound + n);
    const uint32_t max_hops = g->v.P + 2;
    return timed(g, "insert", s, 2, [&]() {
        // the sort's input positions (iin) are free now: they hold the log nominations
        k_insert<<<grid_for(n, 256), 256, 0, s>>>(g->v, kout, iout, d_w, n, g->vbits, d_inserted, max_hops, iin);
        k_log_updated<<<grid_for(n, 256), 256, 0, s>>>(g->v, iin, n);
        return cudaSuccess;
    });
}
