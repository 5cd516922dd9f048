// gc_probe.cu -- FP32 throughput probe (the denominator of the interaction
// kernel's roofline: independent paired-FP32 FMA chains on every lane of
// every SM, timed with CUDA events) and the check of the bounded-wait expiry
// path.  No counterpart in the paper (measurement and diagnostics, not part
// of the method).
#include "gc_common.cuh"
#include "gc_ptx.cuh"

namespace {

constexpr int PR_CHAINS = 8;     // independent float2 chains per thread
constexpr int PR_THREADS = 256;

__global__ void __launch_bounds__(PR_THREADS) k_ffma2_probe(float *sink, int iters, float seed)
{
    float2 v[PR_CHAINS];
    const float2 a = make_float2(0.999999f, 0.999998f);
    const float2 b = make_float2(1e-7f, 2e-7f);
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c)
        v[c] = make_float2(seed + (float)threadIdx.x + (float)c, seed - (float)c);
    for (int i = 0; i < iters; i += 4) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
#pragma unroll
            for (int c = 0; c < PR_CHAINS; ++c) v[c] = __ffma2_rn(v[c], a, b);
        }
    }
    float acc = 0.f;
#pragma unroll
    for (int c = 0; c < PR_CHAINS; ++c) acc += v[c].x + v[c].y;
    if (acc == 12345.678f) sink[blockIdx.x] = acc;   // keeps the chains live
}

// One warp waits on a barrier that nothing arrives at, with the warp-wide
// bounded wait of the interaction kernel; it gives up after `polls` polls and
// records the timeout status.
__global__ void k_wait_expiry(unsigned long long *flags, uint32_t polls)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x >= 32) return;
    if (threadIdx.x == 0) {
        gc_mbar_init(&bar, 1);
        gc_fence_mbar_init();
    }
    __syncwarp();
    const bool ok = gc_mbar_wait_bounded_warp(&bar, 0, polls);
    if (!ok && threadIdx.x == 0) atomicOr(flags, (unsigned long long)GC_FLAG_TIMEOUT);
}

}  // namespace

extern "C" int gc_check_wait_expiry(gc_pool_t *p, uint32_t polls)
{
    if (!p || polls == 0 || polls > (1u << 24)) return GC_ERR_ARG;
    k_wait_expiry<<<1, 32, 0, p->s>>>(p->d_ctr + CTR_FLAGS, polls);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

extern "C" int gc_fp32_peak(double *tflops_out, double *ms_out)
{
    if (!tflops_out) return GC_ERR_ARG;
    int dev = 0, sms = 0;
    GC_CUDA_TRY(cudaGetDevice(&dev));
    GC_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    int per_sm = 0;
    GC_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_ffma2_probe,
                                                              PR_THREADS, 0));
    const int blocks = sms * (per_sm > 0 ? per_sm : 1);
    const int iters = 1 << 14;
    float *sink = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    int rc = GC_OK;
    if (cudaMalloc((void **)&sink, sizeof(float) * blocks) != cudaSuccess ||
        cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        rc = GC_ERR_CUDA;
    } else {
        float best = 1e30f;
        for (int rep = 0; rep < 4; ++rep) {   // first launch warms up
            cudaEventRecord(e0, 0);
            k_ffma2_probe<<<blocks, PR_THREADS>>>(sink, iters, 1.0f);
            cudaEventRecord(e1, 0);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = GC_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (rep > 0 && ms < best) best = ms;
        }
        if (rc == GC_OK) {
            // per iteration and chain: one paired FMA = 2 FMAs = 4 flops
            const double flops = (double)blocks * PR_THREADS * iters * PR_CHAINS * 4.0;
            *tflops_out = flops / (best * 1e-3) / 1e12;
            if (ms_out) *ms_out = best;
        }
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (sink) cudaFree(sink);
    cudaGetLastError();
    return rc;
}
