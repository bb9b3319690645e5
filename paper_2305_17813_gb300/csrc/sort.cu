// Radix sort and prefix sum used by batch staging and export.
//
// These are the CUB device algorithms shipped as header source with the CUDA
// toolkit (CCCL), instantiated and compiled here for sm_103a; no closed
// library is called.
#include "mk_host.h"

#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

namespace mk {

cudaError_t sort_pairs_u64_u32(void *tmp, size_t &tmp_bytes, const uint64_t *kin, uint64_t *kout,
                               const uint32_t *vin, uint32_t *vout, uint64_t n, int end_bit,
                               cudaStream_t s)
{
    return cub::DeviceRadixSort::SortPairs(tmp, tmp_bytes, kin, kout, vin, vout, (int64_t)n, 0, end_bit, s);
}

cudaError_t exclusive_sum_u32_u64(void *tmp, size_t &tmp_bytes, const uint32_t *in, uint64_t *out, uint64_t n,
                                  cudaStream_t s)
{
    return cub::DeviceScan::ExclusiveSum(tmp, tmp_bytes, in, out, (int64_t)n, s);
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

// CUB's decoupled look-back scan: an initialisation kernel and the scan.
int exclusive_sum_launches(uint64_t n)
{
    return n == 0 ? 0 : 2;
}

} // namespace mk
