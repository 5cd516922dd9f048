// gc_noalloc.cu -- softened-gravity evaluation of a batch of tasks whose
// target and source values already sit in the caller's device memory, with
// no allocation of any kind.
//
// Why it exists: some callers cannot allocate device memory at the moment
// they need the result -- code inside another framework whose caching
// allocator already holds the device memory budget (a cudaMalloc beside it
// can fail or fragment that budget), and latency-critical serving threads
// where the implicit device-wide synchronisation of cudaMalloc/cudaFree is
// not acceptable.  The regular path (gc_pool_*/gc_flush) grows its buffers with
// cudaMalloc; this entry point instead keeps all of its scratch (work-unit
// table, per-task counts and offsets, work-queue head) in one fixed-size
// file-scope device array.
//
// Scratch: NaScratch below, about 4.5 MiB, resident on every GPU that loads
// the library until the process exits.  Limits: at most GC_NOALLOC_MAX_TASKS
// tasks and GC_NOALLOC_MAX_TARGETS targets per call (source entries are
// read in place and are not limited by the scratch).  All calls share the
// array and it keeps the previous call's contents; each call rewrites what
// it uses and zeroes its queue head.  Two calls whose work overlaps on the
// GPU (different streams, or the same stream from different host threads
// without ordering) race on the array.
//
// Bad offsets (not starting at 0, decreasing, not ending at n_tgt_total, a
// task with 2^32 or more sources) are found on the device: such a call
// computes nothing and writes NaN into every one of its n_tgt_total output
// rows, so stale rows are never mistaken for results.
//
// Set-up: the first call on a device (with that device current) looks up
// the array's device address with cudaGetSymbolAddress -- the array's name
// in host code is only a host-side stand-in -- and the device's SM count;
// make that first call before any stream capture begins.
#include <mutex>

#include "gc_common.cuh"

namespace {

constexpr uint32_t NA_MAX_TASKS = GC_NOALLOC_MAX_TASKS;
constexpr uint32_t NA_MAX_TARGETS = GC_NOALLOC_MAX_TARGETS;
constexpr int NA_THREADS = 256;
constexpr int NA_WARPS = NA_THREADS / 32;
constexpr int NA_BLOCK = 8;   // plain FP32 partial over <= 8 sources, then compensated add

struct NaUnit {
    uint32_t task, t0, tn, pad;
};

struct NaScratch {
    unsigned long long queue;          // work-queue head (zeroed by every call)
    unsigned long long n_units;        // work units of the current call
    unsigned int bad;                  // a task of this call has bad offsets
    unsigned int status;               // 0: consistent call; 1: bad offsets (NaN rows)
    uint32_t unit_cnt[NA_MAX_TASKS + 1];
    uint32_t unit_off[NA_MAX_TASKS + 1];
    NaUnit unit[NA_MAX_TARGETS];       // <= one unit per target
};

static __device__ __align__(256) NaScratch g_na_scratch;

constexpr int NA_MAX_DEVICES = 64;
std::mutex g_na_mutex;
NaScratch *g_na_ptr[NA_MAX_DEVICES] = {};
int g_na_sms[NA_MAX_DEVICES] = {};

int na_setup(NaScratch **ptr, int *sms)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return GC_ERR_CUDA;
    if (dev < 0 || dev >= NA_MAX_DEVICES) return GC_ERR_ARG;
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_ptr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return GC_ERR_CUDA;
        }
        int n = 0;
        if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess ||
            n < 1)
            return GC_ERR_CUDA;
        g_na_ptr[dev] = static_cast<NaScratch *>(p);
        g_na_sms[dev] = n;
    }
    *ptr = g_na_ptr[dev];
    *sms = g_na_sms[dev];
    return GC_OK;
}

// work units per task: blocks of <= 16 targets
__global__ void k_na_count(uint64_t n_tasks, const uint64_t *tgt_off, const uint64_t *src_off,
                           NaScratch *S)
{
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n_tasks;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint64_t a = tgt_off[t], b = tgt_off[t + 1];
        const uint64_t sa = src_off[t], sb = src_off[t + 1];
        if (b < a || sb < sa || sb - sa > 0xFFFFFFFFull || b - a > NA_MAX_TARGETS) {
            S->bad = 1u;
            S->unit_cnt[t] = 0u;
            continue;
        }
        S->unit_cnt[t] = (uint32_t)((b - a + 15) / 16);
    }
}

// single block: exclusive scan of the unit counts, unit total, queue reset;
// a call whose target total disagrees with its offsets runs no unit and is
// marked for NaN output
__global__ void k_na_scan(uint64_t n_tasks, const uint64_t *tgt_off, uint64_t n_tgt_total,
                          NaScratch *S)
{
    __shared__ uint32_t warp_sums[32];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t carry = 0;
    for (uint64_t b = 0; b < n_tasks; b += blockDim.x) {
        const uint64_t i = b + threadIdx.x;
        const uint32_t v = (i < n_tasks) ? S->unit_cnt[i] : 0u;
        uint32_t x = v;
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) warp_sums[w] = x;
        __syncthreads();
        uint32_t before = carry;
        for (int q = 0; q < w; ++q) before += warp_sums[q];
        uint32_t total = 0;
        for (int q = 0; q < nw; ++q) total += warp_sums[q];
        if (i < n_tasks) S->unit_off[i] = before + x - v;
        __syncthreads();
        carry += total;
    }
    if (threadIdx.x == 0) {
        const bool consistent = tgt_off[n_tasks] == n_tgt_total && tgt_off[0] == 0 &&
                                S->bad == 0u && carry <= NA_MAX_TARGETS;
        S->unit_off[n_tasks] = carry;
        S->n_units = consistent ? carry : 0ull;
        S->status = consistent ? 0u : 1u;
        S->queue = 0ull;
        S->bad = 0u;
    }
}

__global__ void k_na_fill(uint64_t n_tasks, const uint64_t *tgt_off, NaScratch *S)
{
    if (S->n_units == 0) return;   // empty or inconsistent call: nothing to run
    for (uint64_t t = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; t < n_tasks;
         t += (uint64_t)gridDim.x * blockDim.x) {
        const uint32_t nt = (uint32_t)(tgt_off[t + 1] - tgt_off[t]);
        const uint32_t nb = (nt + 15u) / 16u;
        const uint32_t bs = nb ? (nt + nb - 1u) / nb : 0u;
        for (uint32_t b = 0; b < nb; ++b) {
            NaUnit u;
            u.task = (uint32_t)t;
            u.t0 = b * bs;
            u.tn = min(bs, nt - b * bs);
            u.pad = 0;
            const uint32_t at = S->unit_off[t] + b;
            if (at < NA_MAX_TARGETS) S->unit[at] = u;
        }
    }
}

__device__ __forceinline__ void na_kahan(float &s, float &c, float v)
{
    const float y = v - c;
    const float t = s + y;
    c = (t - s) - y;
    s = t;
}

// One warp per work unit (task, block of <= 16 targets), T targets x
// S = 32 / T source lanes, sources read in place (float4 x, y, z, m), the
// same softened-gravity terms and compensated accumulation as the batched
// kernel; lane results combined in FP64 in lane order; row r of target
// tgt_off[task] + k gets (s0..s3, c0..c3) with value s - c.  A call with
// bad offsets instead fills its n_tgt_total rows with NaN.
__global__ void __launch_bounds__(NA_THREADS) k_na_gravity(const NaScratch *S,
                                                           const uint64_t *tgt_off,
                                                           const float4 *tgt,
                                                           const uint64_t *src_off,
                                                           const float4 *src, float eps2,
                                                           float4 *out, uint64_t n_tgt_total,
                                                           unsigned long long *queue)
{
    __shared__ double red[NA_WARPS][32][4];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    if (S->status != 0u) {
        const float q = __int_as_float(0x7fc00000);
        const float4 nan4 = make_float4(q, q, q, q);
        for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < 2 * n_tgt_total;
             i += (uint64_t)gridDim.x * blockDim.x)
            out[i] = nan4;
        return;
    }
    const unsigned long long n_units = S->n_units;
    for (;;) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(queue, 1ull);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= n_units) break;
        const NaUnit u = S->unit[w];
        const int T = (int)u.tn, Sl = 32 / T;
        const int t = lane % T, sl = lane / T;
        const uint64_t tb = tgt_off[u.task], s0 = src_off[u.task];
        const uint32_t ns = (uint32_t)(src_off[u.task + 1] - s0);
        const float4 xi = tgt[tb + u.t0 + t];
        float sx = 0.f, sy = 0.f, sz = 0.f, sp = 0.f, cx = 0.f, cy = 0.f, cz = 0.f, cp = 0.f;
        if (sl < Sl) {
            uint32_t j = (uint32_t)sl;
            while (j < ns) {
                float bx = 0.f, by = 0.f, bz = 0.f, bp = 0.f;
                for (int k = 0; k < NA_BLOCK && j < ns; ++k, j += (uint32_t)Sl) {
                    const float4 pj = __ldg(src + s0 + j);
                    const float dx = pj.x - xi.x, dy = pj.y - xi.y, dz = pj.z - xi.z;
                    const float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, eps2)));
                    const float ri = rsqrtf(r2);
                    const float mr = pj.w * ri;
                    const float mr3 = mr * ri * ri;
                    bx = fmaf(mr3, dx, bx);
                    by = fmaf(mr3, dy, by);
                    bz = fmaf(mr3, dz, bz);
                    bp -= mr;
                }
                na_kahan(sx, cx, bx);
                na_kahan(sy, cy, by);
                na_kahan(sz, cz, bz);
                na_kahan(sp, cp, bp);
            }
        }
        red[wib][lane][0] = (double)sx - (double)cx;
        red[wib][lane][1] = (double)sy - (double)cy;
        red[wib][lane][2] = (double)sz - (double)cz;
        red[wib][lane][3] = (double)sp - (double)cp;
        __syncwarp();
        if (sl == 0) {
            double v[4] = {0, 0, 0, 0};
            for (int q = 0; q < Sl; ++q)
                for (int c = 0; c < 4; ++c) v[c] += red[wib][q * T + t][c];
            float4 s4, c4;
            s4.x = (float)v[0]; c4.x = (float)((double)s4.x - v[0]);
            s4.y = (float)v[1]; c4.y = (float)((double)s4.y - v[1]);
            s4.z = (float)v[2]; c4.z = (float)((double)s4.z - v[2]);
            s4.w = (float)v[3]; c4.w = (float)((double)s4.w - v[3]);
            const uint64_t row = tb + u.t0 + t;
            out[2 * row] = s4;
            out[2 * row + 1] = c4;
        }
        __syncwarp();
    }
}

}  // namespace

extern "C" int gc_gravity_noalloc(uint64_t n_tasks, const uint64_t *tgt_off, const float *tgt_xyzm,
                                  const uint64_t *src_off, const float *src_xyzm,
                                  uint64_t n_tgt_total, float eps2, float *out_rows,
                                  void *cuda_stream)
{
    if (n_tasks > NA_MAX_TASKS || n_tgt_total > NA_MAX_TARGETS) return GC_ERR_TOO_LARGE;
    if (!(eps2 > 0.0f)) return GC_ERR_ARG;
    if (n_tasks == 0) return GC_OK;
    if (!tgt_off || !src_off || !tgt_xyzm || !src_xyzm || !out_rows) return GC_ERR_ARG;
    if (((uintptr_t)tgt_xyzm | (uintptr_t)src_xyzm | (uintptr_t)out_rows) % 16) return GC_ERR_ARG;
    // an error left pending by earlier work is the caller's: report it
    // without clearing it and launch nothing
    if (cudaPeekAtLastError() != cudaSuccess) return GC_ERR_CUDA;
    NaScratch *S = nullptr;
    int sms = 0;
    int rc = na_setup(&S, &sms);
    if (rc != GC_OK) return rc;
    cudaStream_t s = (cudaStream_t)cuda_stream;
    const unsigned g = (unsigned)((n_tasks + 255) / 256 < (uint64_t)sms * 8 ? (n_tasks + 255) / 256
                                                                          : (uint64_t)sms * 8);
    k_na_count<<<g, 256, 0, s>>>(n_tasks, tgt_off, src_off, S);
    if (cudaGetLastError() != cudaSuccess) return GC_ERR_CUDA;
    k_na_scan<<<1, 1024, 0, s>>>(n_tasks, tgt_off, n_tgt_total, S);
    if (cudaGetLastError() != cudaSuccess) return GC_ERR_CUDA;
    k_na_fill<<<g, 256, 0, s>>>(n_tasks, tgt_off, S);
    if (cudaGetLastError() != cudaSuccess) return GC_ERR_CUDA;
    k_na_gravity<<<(unsigned)sms * 4, NA_THREADS, 0, s>>>(
        S, tgt_off, (const float4 *)tgt_xyzm, src_off, (const float4 *)src_xyzm, eps2,
        (float4 *)out_rows, n_tgt_total, &S->queue);
    if (cudaGetLastError() != cudaSuccess) return GC_ERR_CUDA;
    return GC_OK;
}
