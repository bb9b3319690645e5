// Prefix sums (graph creation's head offsets, export's output offsets) and
// the radix sort that puts an export in canonical (src, dst) order.
//
// The scan is this library's own: tiles of 4,096 counts per 1,024-thread
// block (warp shuffles, then a scan of the warp totals in shared memory),
// the tile totals scanned the same way, recursively, and added back.  The
// export's sort is CUB's device radix sort, shipped as header source with
// the CUDA toolkit (CCCL) and compiled here for sm_103a; export is a
// checking utility, not part of the update or algorithm path.
#include "mk_host.h"

#include <cub/device/device_radix_sort.cuh>

#include <vector>

namespace mk {

namespace {

constexpr uint32_t kScanThreads = 1024;
constexpr uint32_t kScanItems = 4;
constexpr uint64_t kScanTile = kScanThreads * kScanItems;

// Exclusive scan of each tile of `in` into `out`; tile totals to `sums`.
template <typename T>
__global__ void __launch_bounds__(kScanThreads) k_scan_tiles(const T *__restrict__ in, uint64_t *__restrict__ out,
                                                              uint64_t n, uint64_t *__restrict__ sums)
{
    __shared__ uint64_t warp_tot[kScanThreads / 32];
    const uint32_t t = threadIdx.x, lane = t & 31, w = t >> 5;
    const uint64_t base = blockIdx.x * kScanTile + (uint64_t)t * kScanItems;
    uint64_t v[kScanItems], run = 0;
#pragma unroll
    for (uint32_t k = 0; k < kScanItems; ++k) {
        v[k] = base + k < n ? (uint64_t)in[base + k] : 0;
        run += v[k];
    }
    // inclusive scan of the thread totals within the warp
    uint64_t incl = run;
#pragma unroll
    for (uint32_t o = 1; o < 32; o <<= 1) {
        const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, incl, o);
        if (lane >= o)
            incl += y;
    }
    if (lane == 31)
        warp_tot[w] = incl;
    __syncthreads();
    if (w == 0) {
        uint64_t x = warp_tot[lane], xi = x;
#pragma unroll
        for (uint32_t o = 1; o < 32; o <<= 1) {
            const uint64_t y = __shfl_up_sync(0xFFFFFFFFu, xi, o);
            if (lane >= o)
                xi += y;
        }
        warp_tot[lane] = xi - x; // exclusive over warps
        if (lane == 31 && sums)
            sums[blockIdx.x] = xi;
    }
    __syncthreads();
    uint64_t acc = warp_tot[w] + incl - run;
#pragma unroll
    for (uint32_t k = 0; k < kScanItems; ++k) {
        if (base + k < n)
            out[base + k] = acc;
        acc += v[k];
    }
}

__global__ void k_add_tile_offsets(uint64_t *out, uint64_t n, const uint64_t *__restrict__ offs)
{
    const uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x;
    if (i < n)
        out[i] += offs[i / kScanTile];
}

uint64_t tiles_of(uint64_t n) { return (n + kScanTile - 1) / kScanTile; }

// Words of scratch for every level of the recursion.
uint64_t scan_scratch_words(uint64_t n)
{
    uint64_t words = 0;
    for (uint64_t t = tiles_of(n); t > 1; t = tiles_of(t))
        words += 2 * t;
    return words;
}

template <typename T>
cudaError_t scan_level(const T *in, uint64_t *out, uint64_t n, uint64_t *scratch, cudaStream_t s, int *launches)
{
    const uint64_t tiles = tiles_of(n);
    if (n == 0)
        return cudaSuccess;
    uint64_t *sums = tiles > 1 ? scratch : nullptr;
    k_scan_tiles<T><<<(uint32_t)tiles, kScanThreads, 0, s>>>(in, out, n, sums);
    ++*launches;
    if (tiles == 1)
        return cudaGetLastError();
    uint64_t *offs = scratch + tiles;
    cudaError_t e = scan_level<uint64_t>(sums, offs, tiles, scratch + 2 * tiles, s, launches);
    if (e != cudaSuccess)
        return e;
    k_add_tile_offsets<<<grid_for(n, 256), 256, 0, s>>>(out, n, offs);
    ++*launches;
    return cudaGetLastError();
}

} // namespace

uint64_t exclusive_scan_scratch_bytes(uint64_t n) { return std::max<uint64_t>(scan_scratch_words(n), 1) * 8; }

cudaError_t exclusive_scan_u32_u64(const uint32_t *in, uint64_t *out, uint64_t n, void *scratch, cudaStream_t s,
                                   int *launches)
{
    int dummy = 0;
    return scan_level<uint32_t>(in, out, n, (uint64_t *)scratch, s, launches ? launches : &dummy);
}

cudaError_t sort_pairs_u64_u32(void *tmp, size_t &tmp_bytes, const uint64_t *kin, uint64_t *kout,
                               const uint32_t *vin, uint32_t *vout, uint64_t n, int end_bit,
                               cudaStream_t s)
{
    return cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, kin, kout, vin, vout, (int64_t)n, 0, end_bit, s);
}

// CUB's onesweep radix sort launches a histogram kernel, a scan of the
// histograms and one onesweep kernel per 8-bit digit; inputs that fit one
// tile take a single-block kernel instead.
int sort_pairs_launches(uint64_t n, int end_bit)
{
    if (n <= 1)
        return 0;
    if (n <= 3072)
        return 1;
    return 2 + (end_bit + 7) / 8;
}

} // namespace mk
