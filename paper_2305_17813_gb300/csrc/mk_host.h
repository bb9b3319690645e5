// Host-side state of one graph and launch helpers shared by the CUDA
// translation units of the library.
#pragma once

#include "meerkat.h"
#include "mk_device.cuh"

#include <cuda_runtime.h>

#include <map>
#include <string>
#include <utility>
#include <vector>

namespace mk {

enum ConsumerKind { kSssp = 0, kBfs = 1, kWcc = 2 };

// State of one incremental algorithm on one graph.
struct Consumer {
    int kind = 0;
    uint32_t source = 0;
    uint64_t epoch = ~0ull;     // graph epoch whose change log this state has applied
    uint64_t seq = ~0ull;       // graph change counter at the last update
    unsigned long long *D = nullptr; // BFS/SSSP: V packed <distance, parent>
    uint2 *front[2] = {nullptr, nullptr}; // BFS/SSSP list frontiers (H entries <list, source> each)
    uint32_t *stamp = nullptr;  // BFS/SSSP: round in which a vertex was last enqueued
    uint32_t *inv = nullptr;    // BFS/SSSP: bitmap of vertices invalidated by this call's deletes
    uint32_t round = 0;         // last stamp value used
    uint32_t *uf = nullptr;     // WCC: union-find parents (V)
    uint32_t *far[2] = {nullptr, nullptr}; // SSSP with Near-Far ordering: far piles (V each)
    uint32_t *fstamp = nullptr; // SSSP with Near-Far ordering: pile stamp per vertex (V)
    uint32_t *counters = nullptr; // device: frontier sizes etc. (16 words)
};

struct TimedLaunch {
    std::string name;
    cudaEvent_t a, b;
};

// Exclusive prefix sum of n counts into 64-bit offsets (sort.cu; the
// library's own kernels); `scratch` holds exclusive_scan_scratch_bytes(n).
// *launches (nullable) is increased by the kernels launched.
uint64_t exclusive_scan_scratch_bytes(uint64_t n);
cudaError_t exclusive_scan_u32_u64(const uint32_t *in, uint64_t *out, uint64_t n, void *scratch, cudaStream_t s,
                                   int *launches);
// Radix sort of (key, value) pairs for the canonical order of an export
// (CUB, compiled in-tree), and the kernel launches it makes.
cudaError_t sort_pairs_u64_u32(void *tmp, size_t &tmp_bytes, const uint64_t *kin, uint64_t *kout,
                               const uint32_t *vin, uint32_t *vout, uint64_t n, int end_bit,
                               cudaStream_t s);
int sort_pairs_launches(uint64_t n, int end_bit);

} // namespace mk

namespace mk {
// Kernel shapes picked by the autotuner (mk_autotune).
struct Tuning {
    int query_group = 8;          // lanes per query chain (4, 8, 16 or 32)
    int query_block = 256;        // threads per block of the query kernels
    int rounds_blocks_per_sm = 0; // size of the persistent round kernel's one block per SM, in units of
                                  // 256 threads (0 = as large as fits)
};
} // namespace mk

struct mk_graph {
    mk::GView v{};               // device pointers + sizes
    mk::Tuning tune{};
    uint32_t vbits = 1;          // bits of a vertex id in a sort key
    mk::DevState *d_state = nullptr;
    uint64_t bytes = 0;          // device bytes held
    // staging scratch, grown on demand: the batch's hash set of (src, dst)
    // pairs as batch positions (table_size entries, a power of two >= 2 *
    // scratch_cap), each edge's entry, and the updated-list nominations of
    // an insert
    uint64_t scratch_cap = 0;
    uint64_t table_size = 0;
    uint32_t *d_tpos = nullptr, *d_slot = nullptr, *d_cand = nullptr;
    uint8_t *d_iflags = nullptr;  // an insert's per-edge stored flags when the caller asks for none
    // change log of the current epoch: deleted (src << 32 | dst)
    unsigned long long *d_dlog = nullptr;
    uint64_t dlog_cap = 0, dlog_bound = 0;
    uint64_t ulog_bound = 0;      // upper bound on the updated-list log's entries (<= H)
    // inserted-edge log of the current epoch: <src, dst, stored weight, 0>
    // of every edge an insert stored (ilog_ok false once an insert of the
    // epoch could not log: the prologues then walk the updated lists)
    uint4 *d_ilog = nullptr;
    uint64_t ilog_cap = 0, ilog_bound = 0;
    bool ilog_ok = true;
    uint64_t epoch = 0, change_seq = 0;
    bool epoch_has_deletes = false;
    std::map<std::pair<int, uint32_t>, mk::Consumer *> consumers;
    uint32_t *h_pinned = nullptr; // 16 pinned words for small device->host reads
    // test hooks (mk_debug_set): grid-barrier poll limit of the round kernel
    // (~0 = the default), and the host-driven round loop instead of the
    // cooperative kernel
    uint64_t dbg_barrier_spins = ~0ull;
    bool dbg_host_rounds = false;
    // Near-Far bucket widths of the SSSP rounds, static and incremental
    // calls (mk_set_sssp_delta; 0 = off)
    uint32_t sssp_delta_static = 0, sssp_delta_incr = 0;
    // profiling
    bool prof = false;
    std::vector<mk::TimedLaunch> timed;
    std::vector<cudaEvent_t> spare_events;
    uint64_t launches = 0;
};

namespace mk {

#define MK_CUDA(call)                                                                                              \
    do {                                                                                                           \
        cudaError_t e_ = (call);                                                                                   \
        if (e_ != cudaSuccess)                                                                                     \
            return e_ == cudaErrorMemoryAllocation ? MK_ERR_NO_MEMORY : MK_ERR_CUDA;                               \
    } while (0)

#define MK_TRY(call)                                                                                               \
    do {                                                                                                           \
        mk_status s_ = (call);                                                                                     \
        if (s_ != MK_OK)                                                                                           \
            return s_;                                                                                             \
    } while (0)

inline cudaEvent_t take_event(mk_graph *g)
{
    if (!g->spare_events.empty()) {
        cudaEvent_t e = g->spare_events.back();
        g->spare_events.pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    cudaEventCreate(&e);
    return e;
}

// Runs `launch` (which enqueues `count` kernels on s), counts the launches
// and, when profiling is on, brackets them with events on s.
template <typename F>
inline mk_status timed(mk_graph *g, const char *name, cudaStream_t s, int count, F &&launch)
{
    cudaEvent_t a = nullptr, b = nullptr;
    if (g->prof) {
        a = take_event(g);
        cudaEventRecord(a, s);
    }
    cudaError_t e = launch();
    if (e == cudaSuccess)
        e = cudaGetLastError();
    g->launches += (uint64_t)count;
    if (g->prof) {
        b = take_event(g);
        cudaEventRecord(b, s);
        g->timed.push_back({name, a, b});
    }
    if (e != cudaSuccess)
        return e == cudaErrorMemoryAllocation ? MK_ERR_NO_MEMORY : MK_ERR_CUDA;
    return MK_OK;
}

// Streaming multiprocessors of the current device (queried once).
inline int num_sms()
{
    static int sms = 0;
    if (!sms) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        if (sms <= 0)
            sms = 1;
    }
    return sms;
}

// A persistent grid for `kernel` launched with `block` threads and no
// dynamic shared memory: every SM filled to its occupancy limit.
template <typename K>
inline uint32_t resident_grid(K kernel, int block)
{
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kernel, block, 0) != cudaSuccess || per < 1)
        per = 1;
    return (uint32_t)(num_sms() * per);
}

inline uint32_t grid_for(uint64_t threads, uint32_t block)
{
    uint64_t b = (threads + block - 1) / block;
    return (uint32_t)(b == 0 ? 1 : b);
}

mk_status ensure_scratch(mk_graph *g, uint64_t n, cudaStream_t s);
int rounds_grid(int units);
int rounds_block(int units);
int rounds_max_blocks_per_sm();
mk_status device_alloc(mk_graph *g, void **p, size_t bytes);
void device_free(mk_graph *g, void *p, size_t bytes);

} // namespace mk
