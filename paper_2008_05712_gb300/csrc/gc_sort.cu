// gc_sort.cu -- device-wide sort and scan primitives (CUB), kept in their own
// translation unit because their templates dominate compile time.
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>

#include "gc_common.cuh"

namespace {

template <class F>
int run_twice(DBuf &tmp, F &&f)
{
    size_t bytes = 0;
    if (f((void *)nullptr, bytes) != cudaSuccess) return GC_ERR_CUDA;
    if (tmp.reserve(bytes ? bytes : 16) != GC_OK) return GC_ERR_OOM;
    size_t have = tmp.cap;
    if (f(tmp.p, have) != cudaSuccess) return GC_ERR_CUDA;
    return GC_OK;
}

}  // namespace

int gc_sort_pairs_u64(DBuf &tmp, const uint64_t *kin, uint64_t *kout, const uint32_t *vin,
                      uint32_t *vout, uint64_t n, int end_bit, cudaStream_t s)
{
    if (n == 0) return GC_OK;
    return run_twice(tmp, [&](void *t, size_t &b) {
        return cub::DeviceRadixSort::SortPairs(t, b, kin, kout, vin, vout, (int64_t)n, 0,
                                               end_bit, s);
    });
}

int gc_sort_pairs_u32(DBuf &tmp, const uint32_t *kin, uint32_t *kout, const uint32_t *vin,
                      uint32_t *vout, uint64_t n, int end_bit, cudaStream_t s)
{
    if (n == 0) return GC_OK;
    return run_twice(tmp, [&](void *t, size_t &b) {
        return cub::DeviceRadixSort::SortPairs(t, b, kin, kout, vin, vout, (int64_t)n, 0,
                                               end_bit, s);
    });
}

int gc_sort_keys_u32(DBuf &tmp, const uint32_t *kin, uint32_t *kout, uint64_t n, int end_bit,
                     cudaStream_t s)
{
    if (n == 0) return GC_OK;
    return run_twice(tmp, [&](void *t, size_t &b) {
        return cub::DeviceRadixSort::SortKeys(t, b, kin, kout, (int64_t)n, 0, end_bit, s);
    });
}

int gc_sort_keys_u64(DBuf &tmp, const uint64_t *kin, uint64_t *kout, uint64_t n,
                     cudaStream_t s)
{
    if (n == 0) return GC_OK;
    return run_twice(tmp, [&](void *t, size_t &b) {
        return cub::DeviceRadixSort::SortKeys(t, b, kin, kout, (int64_t)n, 0, 64, s);
    });
}

int gc_exclusive_scan_u64(DBuf &tmp, const uint64_t *in, uint64_t *out, uint64_t n,
                          cudaStream_t s)
{
    if (n == 0) return GC_OK;
    return run_twice(tmp, [&](void *t, size_t &b) {
        return cub::DeviceScan::ExclusiveSum(t, b, in, out, (int64_t)n, s);
    });
}

int gc_exclusive_scan_u32(DBuf &tmp, const uint32_t *in, uint32_t *out, uint64_t n,
                          cudaStream_t s)
{
    if (n == 0) return GC_OK;
    return run_twice(tmp, [&](void *t, size_t &b) {
        return cub::DeviceScan::ExclusiveSum(t, b, in, out, (int64_t)n, s);
    });
}
