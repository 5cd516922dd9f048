// gc_api.cu -- C ABI of libgcharm: pool lifetime, uploads, batching
// (submit/flush/wait), result read-back and introspection.  The batched
// step itself is split across gc_residency.cu (chare table), gc_kernels.cu
// (pack, interaction, scatter) and the task builders.
#include <cmath>
#include <cstring>
#include <ctime>
#include <unordered_map>
#include <vector>

#include "gc_common.cuh"

// ---- helpers declared in other translation units ----------------------------

// ---- DBuf ---------------------------------------------------------------------
int DBuf::reserve(size_t bytes)
{
    if (bytes <= cap) return GC_OK;
    release();
    size_t want = bytes + bytes / 4 + 256;
    if (cudaMalloc(&p, want) != cudaSuccess) {
        cudaGetLastError();
        p = nullptr;
        cap = 0;
        return GC_ERR_OOM;
    }
    cap = want;
    return GC_OK;
}

void DBuf::release()
{
    if (p) cudaFree(p);
    p = nullptr;
    cap = 0;
}

// Grow keeping the first `used` bytes.
static int grow_keep(DBuf &b, size_t bytes, size_t used, cudaStream_t s)
{
    if (bytes <= b.cap) return GC_OK;
    size_t want = bytes + bytes / 2 + 256;
    void *np = nullptr;
    if (cudaMalloc(&np, want) != cudaSuccess) {
        cudaGetLastError();
        return GC_ERR_OOM;
    }
    if (used && b.p) {
        if (cudaMemcpyAsync(np, b.p, used, cudaMemcpyDeviceToDevice, s) != cudaSuccess) {
            cudaFree(np);
            return GC_ERR_CUDA;
        }
        cudaStreamSynchronize(s);
    }
    b.release();
    b.p = np;
    b.cap = want;
    return GC_OK;
}

const void *gc_device_view(gc_pool *p, const void *ptr, size_t bytes, DBuf &buf, int *rc)
{
    *rc = GC_OK;
    cudaPointerAttributes at;
    if (cudaPointerGetAttributes(&at, ptr) != cudaSuccess) {
        cudaGetLastError();
        at.type = cudaMemoryTypeUnregistered;
    }
    if (at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged) return ptr;
    if ((*rc = buf.reserve(bytes)) != GC_OK) return nullptr;
    if (cudaMemcpyAsync(buf.p, ptr, bytes, cudaMemcpyHostToDevice, p->s) != cudaSuccess ||
        cudaStreamSynchronize(p->s) != cudaSuccess) {
        *rc = GC_ERR_CUDA;
        return nullptr;
    }
    p->stats.h2d_bytes += bytes;
    return buf.p;
}

int gc_reserve_batch(gc_pool *p, uint64_t add_tasks, uint64_t add_tgt, uint64_t add_src)
{
    GC_TRY(grow_keep(p->tasks, (p->nb_tasks + add_tasks + 1) * sizeof(TaskRec),
                     p->nb_tasks * sizeof(TaskRec), p->s));
    GC_TRY(grow_keep(p->tgt_ids, (p->nb_tgt + add_tgt + 1) * sizeof(uint32_t),
                     p->nb_tgt * sizeof(uint32_t), p->s));
    GC_TRY(grow_keep(p->src_ids, (p->nb_src + add_src + 1) * sizeof(uint32_t),
                     p->nb_src * sizeof(uint32_t), p->s));
    return GC_OK;
}

namespace {

__global__ void k_gather_totals(const gcd4 *totals, const uint32_t *ids, uint64_t n,
                                uint64_t id_cap, gcd4 *out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t id = ids[i];
        out[i] = (id < id_cap) ? totals[id] : gcd4{0, 0, 0, 0};
    }
}

// FP64 value s - c of compensated result rows (sum float4, compensation
// float4 per row), one row per thread
__global__ void k_row_values(const float4 *res, uint64_t n, gcd4 *out)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        const float4 s = res[2 * i], c = res[2 * i + 1];
        out[i] = gcd4{(double)s.x - (double)c.x, (double)s.y - (double)c.y,
                      (double)s.z - (double)c.z, (double)s.w - (double)c.w};
    }
}

}  // namespace

void free_ctx(FlushCtx &c)
{
    for (cudaStream_t q : c.ps)   // the pack's side streams read the buffers below
        if (q) cudaStreamSynchronize(q);
    DBuf *bufs[] = {&c.tasks, &c.tgt_ids, &c.src_ids, &c.tgt_perm, &c.src_perm, &c.stg_tgt,
                    &c.stg_src, &c.wu, &c.wu_cnt, &c.wu_off, &c.rowcnt, &c.lj_list, &c.res,
                    &c.row_id, &c.rid_sorted, &c.row_sorted, &c.rows_tmp, &c.runs, &c.tiles,
                    &c.merge_a, &c.merge_b, &c.cub_tmp, &c.lpt, &c.ent};
    for (DBuf *b : bufs) b->release();
    for (int i = 0; i < 6; ++i)
        if (c.ev_stage[i]) cudaEventDestroy(c.ev_stage[i]);
    if (c.ev_done) cudaEventDestroy(c.ev_done);
    if (c.ev_packed) cudaEventDestroy(c.ev_packed);
    if (c.ev_scattered) cudaEventDestroy(c.ev_scattered);
    if (c.d_ctr) cudaFree(c.d_ctr);
    if (c.h_ctr) cudaFreeHost(c.h_ctr);
    for (cudaStream_t q : c.ps)
        if (q) cudaStreamDestroy(q);
    for (cudaEvent_t e : c.pev)
        if (e) cudaEventDestroy(e);
    if (c.owns_stream && c.s) cudaStreamDestroy(c.s);
}

static void free_pool(gc_pool *p)
{
    if (!p) return;
    for (cudaStream_t cs : {p->cs_in, p->cs_out, p->cs_sub})
        if (cs) cudaStreamSynchronize(cs);
    cudaFree(p->d_pool);
    cudaFree(p->d_slot_of_id);
    cudaFree(p->d_id_of_slot);
    cudaFree(p->d_last_use);
    cudaFree(p->d_ref_epoch);
    cudaFree(p->d_ref_count);
    cudaFree(p->d_totals);
    cudaFree(p->d_ctr);
    if (p->d_ewald_h) cudaFree(p->d_ewald_h);
    if (p->h_mirror) cudaFreeHost(p->h_mirror);
    if (p->h_ctr) cudaFreeHost(p->h_ctr);
    DBuf *bufs[] = {&p->tasks, &p->tgt_ids, &p->src_ids, &p->uniq, &p->miss, &p->miss_sorted,
                    &p->freel,
                    &p->tiles, &p->ekeys, &p->ekeys2, &p->evicted, &p->cub_tmp, &p->io_a,
                    &p->io_b, &p->nb.keys, &p->nb.keys2, &p->nb.ids, &p->nb.ids2, &p->nb.lcp,
                    &p->nb.win, &p->nb.dmax, &p->nb.nnode, &p->nb.node_off, &p->nb.node_a,
                    &p->nb.node_b, &p->nb.node_val, &p->nb.bucket, &p->nb.bbox,
                    &p->nb.list_off, &p->nb.list_len, &p->nb.list, &p->nb.bounds,
                    &p->nb.cub_tmp, &p->nb.mono, &p->nb.hostcopy, &p->nb.wnode, &p->nb.seed_tiles,
                    &p->nb.seed_a, &p->nb.seed_m, &p->nb.seed_key, &p->au_ids, &p->au_vals,
                    &p->at_ids, &p->at_out, &p->sub_desc, &p->md.hostcopy,
                    &p->md.keys,
                    &p->md.keys2, &p->md.ids, &p->md.ids2, &p->md.cell_start, &p->md.cnt_t,
                    &p->md.cnt_s, &p->md.cub_tmp};
    for (DBuf *b : bufs) b->release();
    for (cudaEvent_t &e : p->nb.ev)
        if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : {p->ev_au, p->ev_au_in, p->ev_at_in, p->ev_at_g, p->ev_at,
                          p->ev_pend_free, p->ev_sub_copied, p->ev_sub_done})
        if (e) cudaEventDestroy(e);
    if (p->h_sub) cudaFreeHost(p->h_sub);
    for (cudaStream_t cs : {p->cs_in, p->cs_out, p->cs_sub})
        if (cs) cudaStreamDestroy(cs);
    for (int i = 0; i < 2; ++i) free_ctx(p->ctx[i]);
    delete p;
}

int init_ctx(FlushCtx &c, cudaStream_t given)
{
    if (given) {
        c.s = given;
        c.owns_stream = false;
    } else {
        if (cudaStreamCreateWithFlags(&c.s, cudaStreamNonBlocking) != cudaSuccess)
            return GC_ERR_CUDA;
        c.owns_stream = true;
    }
    if (cudaMalloc((void **)&c.d_ctr, sizeof(unsigned long long) * FC_COUNT) != cudaSuccess ||
        cudaHostAlloc((void **)&c.h_ctr, sizeof(unsigned long long) * FH_COUNT,
                      cudaHostAllocDefault) != cudaSuccess)
        return GC_ERR_OOM;
    for (int i = 0; i < 6; ++i)
        if (cudaEventCreate(&c.ev_stage[i]) != cudaSuccess) return GC_ERR_CUDA;
    if (cudaEventCreateWithFlags(&c.ev_done, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c.ev_packed, cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&c.ev_scattered, cudaEventDisableTiming) != cudaSuccess)
        return GC_ERR_CUDA;
    for (cudaStream_t &q : c.ps)
        if (cudaStreamCreateWithFlags(&q, cudaStreamNonBlocking) != cudaSuccess)
            return GC_ERR_CUDA;
    for (cudaEvent_t &e : c.pev)
        if (cudaEventCreateWithFlags(&e, cudaEventDisableTiming) != cudaSuccess)
            return GC_ERR_CUDA;
    if (cudaMemsetAsync(c.d_ctr, 0, sizeof(unsigned long long) * FC_COUNT, c.s) != cudaSuccess)
        return GC_ERR_CUDA;
    return GC_OK;
}

// The context holding batch `batch`, or null if neither does.
static FlushCtx *ctx_of(gc_pool *p, uint64_t batch)
{
    for (int i = 0; i < 2; ++i)
        if (p->ctx[i].valid && p->ctx[i].batch == batch) return &p->ctx[i];
    return nullptr;
}

static FlushCtx *last_ctx(gc_pool *p) { return p->last >= 0 ? &p->ctx[p->last] : nullptr; }

namespace {
__global__ void k_clear_flags(unsigned long long *flags, unsigned long long mask)
{
    if (threadIdx.x == 0 && blockIdx.x == 0) atomicAnd(flags, ~mask);
}
}  // namespace

int gc_clear_flags(gc_pool *p, cudaStream_t s, unsigned long long mask)
{
    k_clear_flags<<<1, 32, 0, s>>>(p->d_ctr + CTR_FLAGS, mask);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

int gc_apply_totals_reset(gc_pool *p, cudaStream_t s)
{
    if (!p->totals_reset_pending) return GC_OK;
    GC_CUDA_TRY(cudaMemsetAsync(p->d_totals, 0, sizeof(gcd4) * p->cfg.id_capacity, s));
    p->totals_reset_pending = false;
    return GC_OK;
}

// Make the issue stream wait for every scatter in flight (per-id totals).
int order_after_scatters(gc_pool *p)
{
    for (int i = 0; i < 2; ++i)
        if (p->ctx[i].valid && p->ctx[i].s != p->s)
            GC_CUDA_TRY(cudaStreamWaitEvent(p->s, p->ctx[i].ev_scattered, 0));
    return GC_OK;
}

template <class T>
static int dmalloc(T **ptr, uint64_t count)
{
    if (cudaMalloc((void **)ptr, sizeof(T) * (count ? count : 1)) != cudaSuccess) {
        cudaGetLastError();
        *ptr = nullptr;
        return GC_ERR_OOM;
    }
    return GC_OK;
}

static bool on_grid(double v, double scale, int64_t *out)
{
    double g = v * scale;
    if (!(g >= 0) || g > 9.0e18 || std::floor(g) != g) return false;
    *out = (int64_t)g;
    return true;
}

static void clear_last_stats(gc_pool *p)
{
    gc_stats_t &s = p->stats;
    s.last_unique = s.last_hits = s.last_misses = s.last_evictions = 0;
    s.last_staging_bytes = s.last_waves = 0;
    s.lj_pairs_in_cutoff = 0;
    for (int b = 0; b < 8; ++b) s.reuse_hist[b] = 0;
}

extern "C" {

const char *gc_strerror(int status)
{
    switch (status) {
    case GC_OK: return "ok";
    case GC_ERR_ARG: return "invalid argument";
    case GC_ERR_OOM: return "out of memory";
    case GC_ERR_POOL_FULL: return "pool full: batch references more ids than fit";
    case GC_ERR_UNKNOWN_ID: return "unknown id: a task references an id never uploaded";
    case GC_ERR_BUDGET: return "one task exceeds the staging budget";
    case GC_ERR_NOT_READY: return "not ready";
    case GC_ERR_TIMEOUT: return "timeout";
    case GC_ERR_CUDA: return "CUDA error";
    case GC_ERR_STATE: return "invalid state";
    case GC_ERR_TOO_LARGE: return "request exceeds a fixed size limit";
    default: return "unknown status";
    }
}

int gc_pool_create(const gc_config *cfg, gc_pool_t **out)
{
    if (!cfg || !out) return GC_ERR_ARG;
    *out = nullptr;
    if (cfg->id_capacity == 0 || cfg->pool_capacity == 0 || !(cfg->eps2 > 0.0f) ||
        cfg->id_capacity > 0xFFFFFFFEull || cfg->pool_capacity > 0xFFFFFFFEull)
        return GC_ERR_ARG;
    gc_pool *p = new gc_pool();
    std::memset(&p->stats, 0, sizeof p->stats);
    p->cfg = *cfg;
    int64_t rc2g = 0, eg = 0;
    if (cfg->lj_rc2 > 0.0f) {
        if (!on_grid((double)cfg->lj_rc2, 4398046511104.0, &rc2g)) { delete p; return GC_ERR_ARG; }
    }
    if (cfg->md_edge > 0.0f) {
        if (!on_grid((double)cfg->md_edge, 2097152.0, &eg) || eg >= (1 << 23)) {
            delete p;
            return GC_ERR_ARG;
        }
    }
    p->rc2_grid = rc2g;
    p->md_edge_grid = (int32_t)eg;
    if (cfg->ewald_box < 0.0f || !(cfg->ewald_box == cfg->ewald_box)) {
        delete p;
        return GC_ERR_ARG;
    }
    if (cudaGetDevice(&p->device) != cudaSuccess ||
        cudaDeviceGetAttribute(&p->num_sms, cudaDevAttrMultiProcessorCount, p->device) !=
            cudaSuccess) {
        cudaGetLastError();
        delete p;
        return GC_ERR_CUDA;
    }
    // flush context 0 issues on the caller's stream (or an owned one), context
    // 1 on an owned stream; consecutive batches alternate between them
    {
        int rc0 = init_ctx(p->ctx[0], (cudaStream_t)cfg->cuda_stream);
        if (rc0 == GC_OK) rc0 = init_ctx(p->ctx[1], nullptr);
        if (rc0 != GC_OK) {
            cudaGetLastError();
            free_pool(p);
            return rc0;
        }
        p->cur = 0;
        p->last = -1;
        p->s = p->ctx[0].s;
    }
    const uint64_t idc = cfg->id_capacity, cap = cfg->pool_capacity;
    int rc = GC_OK;
    if (rc == GC_OK) rc = dmalloc(&p->d_pool, cap);
    if (rc == GC_OK) rc = dmalloc(&p->d_slot_of_id, idc);
    if (rc == GC_OK) rc = dmalloc(&p->d_id_of_slot, cap);
    if (rc == GC_OK) rc = dmalloc(&p->d_last_use, cap);
    if (rc == GC_OK) rc = dmalloc(&p->d_ref_epoch, idc);
    if (rc == GC_OK) rc = dmalloc(&p->d_ref_count, idc);
    if (rc == GC_OK) rc = dmalloc(&p->d_totals, idc);
    if (rc == GC_OK) rc = dmalloc(&p->d_ctr, (uint64_t)CTR_COUNT);
    if (rc == GC_OK && cfg->ewald_box > 0.0f) {
        // reciprocal vectors with 0 < |h|^2 <= 10, one of each pair +-h (the
        // pair's cos and h sin terms are equal: the coefficient is doubled)
        const double L = cfg->ewald_box, alpha = 2.0 / L, pi = 3.14159265358979323846;
        std::vector<float4> hv;
        for (int hx = -3; hx <= 3; ++hx)
            for (int hy = -3; hy <= 3; ++hy)
                for (int hz = -3; hz <= 3; ++hz) {
                    const int h2 = hx * hx + hy * hy + hz * hz;
                    if (h2 == 0 || h2 > 10) continue;
                    const bool upper = hx > 0 || (hx == 0 && (hy > 0 || (hy == 0 && hz > 0)));
                    if (!upper) continue;
                    const double c = 2.0 * std::exp(-pi * pi * h2 / (alpha * alpha * L * L)) / h2;
                    hv.push_back(make_float4((float)hx, (float)hy, (float)hz, (float)c));
                }
        rc = dmalloc(&p->d_ewald_h, (uint64_t)hv.size());
        if (rc == GC_OK &&
            cudaMemcpy(p->d_ewald_h, hv.data(), hv.size() * sizeof(float4),
                       cudaMemcpyHostToDevice) != cudaSuccess)
            rc = GC_ERR_CUDA;
        p->n_ewald_h = (int)hv.size();
    }
    if (rc == GC_OK) {
        if (cudaHostAlloc((void **)&p->h_mirror, sizeof(float4) * idc, cudaHostAllocMapped) !=
                cudaSuccess ||
            cudaHostGetDevicePointer((void **)&p->d_mirror, p->h_mirror, 0) != cudaSuccess ||
            cudaHostAlloc((void **)&p->h_ctr, sizeof(unsigned long long) * CTR_COUNT,
                          cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            rc = GC_ERR_OOM;
        }
    }
    if (rc == GC_OK) {
        cudaMemsetAsync(p->d_slot_of_id, 0xFF, sizeof(uint32_t) * idc, p->s);
        cudaMemsetAsync(p->d_id_of_slot, 0xFF, sizeof(uint32_t) * cap, p->s);
        p->free_slots = cap;
        cudaMemsetAsync(p->d_last_use, 0, sizeof(uint32_t) * cap, p->s);
        cudaMemsetAsync(p->d_ref_epoch, 0xFF, sizeof(uint32_t) * idc, p->s);   // unknown
        cudaMemsetAsync(p->d_ref_count, 0, sizeof(uint32_t) * idc, p->s);
        cudaMemsetAsync(p->d_totals, 0, sizeof(gcd4) * idc, p->s);
        cudaMemsetAsync(p->d_ctr, 0, sizeof(unsigned long long) * CTR_COUNT, p->s);
        std::memset(p->h_mirror, 0, sizeof(float4) * idc);
        if (rc == GC_OK && cudaStreamSynchronize(p->s) != cudaSuccess) rc = GC_ERR_CUDA;
    }
    if (rc != GC_OK) {
        free_pool(p);
        return rc;
    }
    *out = p;
    return GC_OK;
}

int gc_pool_destroy(gc_pool_t *p)
{
    if (!p) return GC_ERR_ARG;
    cudaStreamSynchronize(p->ctx[0].s);
    cudaStreamSynchronize(p->ctx[1].s);
    free_pool(p);
    return GC_OK;
}

int gc_pool_upload(gc_pool_t *p, const uint32_t *ids, const float *xyzm, uint64_t n)
{
    if (!p || (n && (!ids || !xyzm))) return GC_ERR_ARG;
    if (n == 0) return GC_OK;
    uint32_t bad = 0;
    for (uint64_t i = 0; i < n; ++i) bad |= (uint64_t)ids[i] >= p->cfg.id_capacity;
    if (bad) return GC_ERR_ARG;
    // the device writes resident ids' slots and non-resident ids' mirror
    // entries (a resident id's mirror entry is refreshed when it is evicted),
    // in stream order after the batches already flushed have packed
    GC_TRY(grow_keep(p->io_a, n * sizeof(uint32_t) + 16, 0, p->s));
    GC_TRY(grow_keep(p->io_b, n * sizeof(float4) + 16, 0, p->s));
    int rc = GC_OK;
    if (cudaMemcpyAsync(p->io_a.p, ids, n * sizeof(uint32_t), cudaMemcpyHostToDevice, p->s) !=
            cudaSuccess ||
        cudaMemcpyAsync(p->io_b.p, xyzm, n * sizeof(float4), cudaMemcpyHostToDevice, p->s) !=
            cudaSuccess)
        rc = GC_ERR_CUDA;
    if (rc == GC_OK) rc = gc_launch_upload(p, p->io_a.as<uint32_t>(), p->io_b.as<float4>(), n, 1);
    if (cudaStreamSynchronize(p->s) != cudaSuccess) rc = GC_ERR_CUDA;
    p->stats.h2d_bytes += n * (sizeof(uint32_t) + sizeof(float4));
    return rc;
}

// Copy streams and events of the stream-ordered upload and totals read.
static int async_init(gc_pool *p)
{
    for (cudaStream_t *cs : {&p->cs_in, &p->cs_out})
        if (!*cs) GC_CUDA_TRY(cudaStreamCreateWithFlags(cs, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&p->ev_au, &p->ev_au_in, &p->ev_at_in, &p->ev_at_g, &p->ev_at})
        if (!*e) GC_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    return GC_OK;
}

int gc_pool_upload_async(gc_pool_t *p, const uint32_t *ids, const float *xyzm, uint64_t n)
{
    if (!p || (n && (!ids || !xyzm))) return GC_ERR_ARG;
    if (n == 0) return GC_OK;
    GC_TRY(async_init(p));
    // a reallocation frees the old buffers, which waits for the device
    GC_TRY(grow_keep(p->au_ids, n * sizeof(uint32_t) + 16, 0, p->s));
    GC_TRY(grow_keep(p->au_vals, n * sizeof(float4) + 16, 0, p->s));
    // the copies wait only for the previous upload kernel to have read the
    // buffers, not for the batches queued on the pool's stream
    if (p->au_used) GC_CUDA_TRY(cudaStreamWaitEvent(p->cs_in, p->ev_au, 0));
    GC_CUDA_TRY(cudaMemcpyAsync(p->au_ids.p, ids, n * sizeof(uint32_t), cudaMemcpyHostToDevice,
                                p->cs_in));
    GC_CUDA_TRY(cudaMemcpyAsync(p->au_vals.p, xyzm, n * sizeof(float4), cudaMemcpyHostToDevice,
                                p->cs_in));
    GC_CUDA_TRY(cudaEventRecord(p->ev_au_in, p->cs_in));
    GC_CUDA_TRY(cudaStreamWaitEvent(p->s, p->ev_au_in, 0));
    GC_TRY(gc_launch_upload(p, p->au_ids.as<uint32_t>(), p->au_vals.as<float4>(), n, 1));
    GC_CUDA_TRY(cudaEventRecord(p->ev_au, p->s));
    p->au_used = true;
    p->stats.h2d_bytes += n * (sizeof(uint32_t) + sizeof(float4));
    return GC_OK;
}

int gc_pool_upload_device(gc_pool_t *p, const uint32_t *ids_dev, const float *xyzm_dev,
                          uint64_t n)
{
    if (!p || (n && (!ids_dev || !xyzm_dev))) return GC_ERR_ARG;
    if (((uintptr_t)xyzm_dev) % 16) return GC_ERR_ARG;
    return gc_launch_upload(p, ids_dev, (const float4 *)xyzm_dev, n, 1);
}

// ---- submission ---------------------------------------------------------------

// Host arrays of one submission: descriptors packed into the pinned host
// staging (with the ids too when they are few), copied on the submission
// stream, task records built there; returns once the caller's arrays have
// been read.
static const uint64_t SUB_PACK_IDS = 1u << 18;   // ids packed with the descriptors

static int submit_host(gc_pool *p, uint64_t n_tasks, const uint64_t *task_ids,
                       const uint32_t *kinds, const int8_t *shifts, const uint64_t *tgt_off,
                       const uint32_t *tgt_ids, const uint64_t *src_off,
                       const uint32_t *src_ids, uint64_t n_tgt, uint64_t n_src, uint32_t *dt,
                       uint32_t *ds, uint64_t id_base, TaskRec *recs)
{
    if (!p->cs_sub) GC_CUDA_TRY(cudaStreamCreateWithFlags(&p->cs_sub, cudaStreamNonBlocking));
    for (cudaEvent_t *e : {&p->ev_pend_free, &p->ev_sub_copied, &p->ev_sub_done})
        if (!*e) GC_CUDA_TRY(cudaEventCreateWithFlags(e, cudaEventDisableTiming));
    auto al = [](size_t v) { return (v + 15) & ~(size_t)15; };
    const size_t b_ids = task_ids ? n_tasks * 8 : 0, b_k = n_tasks * 4,
                 b_sh = shifts ? n_tasks * 3 : 0, b_off = (n_tasks + 1) * 8;
    const size_t o_ids = 0, o_k = al(o_ids + b_ids), o_sh = al(o_k + b_k), o_to = al(o_sh + b_sh),
                 o_so = al(o_to + b_off), desc = o_so + b_off;
    const bool pack_ids = n_tgt + n_src <= SUB_PACK_IDS;
    const size_t o_tg = al(desc), o_sr = al(o_tg + n_tgt * 4),
                 host_bytes = pack_ids ? o_sr + n_src * 4 : desc;
    GC_TRY(grow_keep(p->sub_desc, desc + 16, 0, p->s));
    if (host_bytes > p->h_sub_cap) {
        if (p->h_sub) cudaFreeHost(p->h_sub);
        p->h_sub = nullptr;
        p->h_sub_cap = 0;
        const size_t want = host_bytes + host_bytes / 2 + 4096;
        if (cudaHostAlloc(&p->h_sub, want, cudaHostAllocDefault) != cudaSuccess) {
            cudaGetLastError();
            p->h_sub = nullptr;
            return GC_ERR_OOM;
        }
        p->h_sub_cap = want;
    }
    char *h = (char *)p->h_sub;
    if (b_ids) std::memcpy(h + o_ids, task_ids, b_ids);
    std::memcpy(h + o_k, kinds, b_k);
    if (b_sh) std::memcpy(h + o_sh, shifts, b_sh);
    std::memcpy(h + o_to, tgt_off, b_off);
    std::memcpy(h + o_so, src_off, b_off);
    if (pack_ids) {
        if (n_tgt) std::memcpy(h + o_tg, tgt_ids, n_tgt * 4);
        if (n_src) std::memcpy(h + o_sr, src_ids, n_src * 4);
    }
    // the pending arrays' last readers (the batch that held them before the
    // flush handed them over); the previous submission's task records ran
    // earlier on this stream, so the descriptor buffer is free
    const cudaStream_t cs = p->cs_sub;
    char *d = (char *)p->sub_desc.p;
    int rc = GC_OK;
    auto cp = [&](void *dst, const void *src, size_t bytes) {
        if (rc == GC_OK && bytes &&
            cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, cs) != cudaSuccess)
            rc = GC_ERR_CUDA;
    };
    if (cudaStreamWaitEvent(cs, p->ev_pend_free, 0) != cudaSuccess) rc = GC_ERR_CUDA;
    cp(d, h, desc);
    cp(dt, pack_ids ? (const void *)(h + o_tg) : (const void *)tgt_ids, n_tgt * 4);
    cp(ds, pack_ids ? (const void *)(h + o_sr) : (const void *)src_ids, n_src * 4);
    if (rc == GC_OK && cudaEventRecord(p->ev_sub_copied, cs) != cudaSuccess) rc = GC_ERR_CUDA;
    if (rc == GC_OK)
        rc = gc_make_task_recs(p, n_tasks, task_ids ? (uint64_t *)(d + o_ids) : nullptr,
                               (uint32_t *)(d + o_k), shifts ? (int8_t *)(d + o_sh) : nullptr,
                               (uint64_t *)(d + o_to), (uint64_t *)(d + o_so), p->nb_tgt,
                               p->nb_src, id_base, recs, cs);
    if (rc == GC_OK && (cudaEventRecord(p->ev_sub_done, cs) != cudaSuccess ||
                        cudaStreamWaitEvent(p->s, p->ev_sub_done, 0) != cudaSuccess))
        rc = GC_ERR_CUDA;
    // the caller's arrays and the host staging have been read once the
    // copies are done (a bad task is reported by the flush)
    if (rc == GC_OK && cudaEventSynchronize(p->ev_sub_copied) != cudaSuccess) rc = GC_ERR_CUDA;
    if (rc != GC_OK) {
        cudaStreamSynchronize(cs);
        return rc;
    }
    p->stats.h2d_bytes += desc + 4 * (n_tgt + n_src);
    return GC_OK;
}

static int gc_submit_csr_impl(gc_pool *p, uint64_t n_tasks, const uint64_t *task_ids,
                       const uint32_t *kinds, const int8_t *shifts, const uint64_t *tgt_off,
                       const uint32_t *tgt_ids, const uint64_t *src_off,
                       const uint32_t *src_ids, uint64_t n_tgt_total, uint64_t n_src_total,
                       int on_device, uint64_t *batch_out)
{
    if (!p || (n_tasks && (!kinds || !tgt_off || !src_off))) return GC_ERR_ARG;
    if (batch_out) *batch_out = p->submitted_batches;
    if (n_tasks == 0) return GC_OK;
    const uint64_t budget = p->cfg.staging_budget_bytes;
    if (!on_device) {
        if (tgt_off[0] != 0 || src_off[0] != 0) return GC_ERR_ARG;
        for (uint64_t t = 0; t < n_tasks; ++t) {
            if (tgt_off[t + 1] < tgt_off[t] || src_off[t + 1] < src_off[t]) return GC_ERR_ARG;
            uint64_t nt = tgt_off[t + 1] - tgt_off[t], ns = src_off[t + 1] - src_off[t];
            if (nt > 0xFFFFFFFFull || ns > 0xFFFFFFFFull) return GC_ERR_ARG;
            if (kinds[t] > GC_EWALD || (kinds[t] == GC_LJ_SELF && ns) ||
                (kinds[t] == GC_EWALD && p->n_ewald_h == 0))
                return GC_ERR_ARG;
            if (budget && (nt + ns) * sizeof(float4) > budget) return GC_ERR_BUDGET;
        }
        n_tgt_total = tgt_off[n_tasks];
        n_src_total = src_off[n_tasks];
        if (n_tgt_total && !tgt_ids) return GC_ERR_ARG;
        if (n_src_total && !src_ids) return GC_ERR_ARG;
    }
    GC_TRY(gc_reserve_batch(p, n_tasks, n_tgt_total, n_src_total));
    TaskRec *recs = p->tasks.as<TaskRec>() + p->nb_tasks;
    uint32_t *dt = p->tgt_ids.as<uint32_t>() + p->nb_tgt;
    uint32_t *ds = p->src_ids.as<uint32_t>() + p->nb_src;
    const uint64_t id_base = p->stats.tasks + p->nb_tasks;
    if (on_device) {
        if (n_tgt_total)
            GC_CUDA_TRY(cudaMemcpyAsync(dt, tgt_ids, n_tgt_total * sizeof(uint32_t),
                                        cudaMemcpyDeviceToDevice, p->s));
        if (n_src_total)
            GC_CUDA_TRY(cudaMemcpyAsync(ds, src_ids, n_src_total * sizeof(uint32_t),
                                        cudaMemcpyDeviceToDevice, p->s));
        GC_TRY(gc_make_task_recs(p, n_tasks, task_ids, kinds, shifts, tgt_off, src_off,
                                 p->nb_tgt, p->nb_src, id_base, recs, p->s));
    } else {
        GC_TRY(submit_host(p, n_tasks, task_ids, kinds, shifts, tgt_off, tgt_ids, src_off,
                           src_ids, n_tgt_total, n_src_total, dt, ds, id_base, recs));
    }
    p->nb_tasks += n_tasks;
    p->nb_tgt += n_tgt_total;
    p->nb_src += n_src_total;
    return GC_OK;
}

int gc_submit_csr(gc_pool_t *p, uint64_t n_tasks, const uint64_t *task_ids,
                  const uint32_t *kinds, const int8_t *shifts, const uint64_t *tgt_off,
                  const uint32_t *tgt_ids, const uint64_t *src_off, const uint32_t *src_ids,
                  uint64_t n_tgt_total, uint64_t n_src_total, int on_device,
                  uint64_t *batch_out)
{
    return gc_submit_csr_impl(p, n_tasks, task_ids, kinds, shifts, tgt_off, tgt_ids, src_off,
                              src_ids, n_tgt_total, n_src_total, on_device, batch_out);
}

int gc_submit(gc_pool_t *p, const gc_task *tasks, uint64_t n, uint64_t *batch_out)
{
    if (!p || (n && !tasks)) return GC_ERR_ARG;
    std::vector<uint64_t> ids(n), to(n + 1), so(n + 1);
    std::vector<uint32_t> kinds(n), tg, sr;
    std::vector<int8_t> sh(3 * n);
    to[0] = so[0] = 0;
    for (uint64_t t = 0; t < n; ++t) {
        const gc_task &k = tasks[t];
        if ((k.n_targets && !k.target_ids) || (k.n_sources && !k.source_ids)) return GC_ERR_ARG;
        ids[t] = k.task_id;
        kinds[t] = k.kind;
        for (int a = 0; a < 3; ++a) sh[3 * t + a] = k.shift[a];
        tg.insert(tg.end(), k.target_ids, k.target_ids + k.n_targets);
        sr.insert(sr.end(), k.source_ids, k.source_ids + k.n_sources);
        to[t + 1] = to[t] + k.n_targets;
        so[t + 1] = so[t] + k.n_sources;
    }
    return gc_submit_csr_impl(p, n, ids.data(), kinds.data(), sh.data(), to.data(), tg.data(),
                              so.data(), sr.data(), 0, 0, 0, batch_out);
}

// ---- flush ----------------------------------------------------------------------
//
// Batch k runs on flush context ctx[k % 2] and its stream.  Two event edges
// keep consecutive batches correct while they overlap on the device:
//   - the next batch's chare-table step (which may move or refill pool
//     slots) and any upload or task build issued after gc_flush returns wait
//     for this batch's pack (the last reader of the pool);
//   - the next batch's scatter waits for this batch's scatter (per-id totals
//     accumulate in admission order).
// The interaction of batch k thus runs while batch k+1 is residency-checked
// and packed.  A context is reused by batch k+2, in stream order after
// batch k, so results of a batch stay readable until batch k+2 is flushed.

static void count_timing(gc_pool *p, FlushCtx &c, bool block);

static int flush_impl(gc_pool *p, int per_task)
{
    if (!p) return GC_ERR_ARG;
    if (p->nb_tasks == 0) return GC_OK;
    FlushCtx &c = p->ctx[p->cur];
    FlushCtx *prev = last_ctx(p);
    count_timing(p, c, true);   // the context's previous batch (two batches ago)
    // the batch becomes this context's batch; the context's previous batch
    // arrays become the next pending arrays (every later write to them is
    // ordered after this context's stream passes the point below, or, for
    // the copies of a host submission, after the previous batch's work on
    // this stream: ev_pend_free)
    if (!p->ev_pend_free)
        GC_CUDA_TRY(cudaEventCreateWithFlags(&p->ev_pend_free, cudaEventDisableTiming));
    GC_CUDA_TRY(cudaEventRecord(p->ev_pend_free, c.s));
    std::swap(p->tasks, c.tasks);
    std::swap(p->tgt_ids, c.tgt_ids);
    std::swap(p->src_ids, c.src_ids);
    c.n_tasks = p->nb_tasks;
    c.n_tgt = p->nb_tgt;
    c.n_src = p->nb_src;
    c.batch = p->submitted_batches;
    c.md_struct = p->md_pending && c.n_tasks == gc_md_tasks(p->md_pend_m, p->md_pend_dim);
    c.md_m = p->md_pend_m;
    c.md_dim = p->md_pend_dim;
    p->md_pending = false;
    // one N-body build alone: its rows are the bucket particles, each once
    c.unique_rows = p->nb_pend_tasks != 0 && c.n_tasks == p->nb_pend_tasks;
    p->nb_pend_tasks = 0;
    c.valid = false;
    c.host_tasks_valid = false;
    c.timing_valid = false;
    c.timing_counted = false;
    p->nb_tasks = p->nb_tgt = p->nb_src = 0;
    const uint64_t T = c.n_tasks, NT = c.n_tgt, NS = c.n_src;
    clear_last_stats(p);

    uint64_t info[5];
    const uint64_t budget = p->cfg.staging_budget_bytes;
    // A batch that fits the staging budget runs as one wave: its chare-table
    // step is issued with the preparation, and the task-flag word, the
    // preparation's sizes and the chare-table counters come back in one host
    // round trip (the task records were written on this stream).
    const bool one_wave = !(budget && (NT + NS) * sizeof(float4) > budget);
    GC_CUDA_TRY(cudaMemcpyAsync(p->h_ctr + CTR_FLAGS, p->d_ctr + CTR_FLAGS,
                                sizeof(unsigned long long), cudaMemcpyDeviceToHost, c.s));
    int rc = gc_prepare_issue(p, c);
    if (rc != GC_OK) return rc;
    if (one_wave) {
        GC_TRY(c.ent.reserve((NT + NS + 1) * sizeof(uint32_t)));
        GC_CUDA_TRY(cudaEventRecord(c.ev_stage[0], c.s));
        rc = gc_residency_issue(p, c.tgt_ids.as<uint32_t>(), NT, c.src_ids.as<uint32_t>(), NS,
                                c.ent.as<uint32_t>());
        if (rc != GC_OK) return rc;
    }
    GC_CUDA_TRY(cudaStreamSynchronize(c.s));
    rc = gc_prepare_finish(p, c, info);
    if (rc != GC_OK) return rc;
    if (p->h_ctr[CTR_FLAGS] & GC_FLAG_BAD_TASK) {
        gc_clear_flags(p, c.s, GC_FLAG_BAD_TASK);
        return GC_ERR_ARG;
    }
    const uint64_t R = info[0], W = info[1], L = info[2], inter = info[3], max_list = info[4];
    c.n_rows = R;
    c.max_list = max_list;

    GC_TRY(c.tgt_perm.reserve((NT + 1) * 4));
    GC_TRY(c.src_perm.reserve((NS + 1) * 4));
    GC_TRY(c.res.reserve((R + 1) * 2 * sizeof(float4)));
    GC_TRY(c.row_id.reserve((R + 1) * 4));

    // waves under the staging budget
    struct Wave { uint64_t t0, t1, tg0, tg1, s0, s1; };
    std::vector<Wave> waves;
    std::vector<uint32_t> wu_off, lj_off;
    bool need_offsets = per_task != 0;
    if (!one_wave) {
        std::vector<TaskRec> h(T);
        GC_CUDA_TRY(cudaMemcpy(h.data(), c.tasks.p, T * sizeof(TaskRec), cudaMemcpyDeviceToHost));
        uint64_t t0 = 0;
        while (t0 < T) {
            uint64_t t1 = t0, bytes = 0;
            while (t1 < T && bytes + (uint64_t)(h[t1].nt + h[t1].ns) * sizeof(float4) <= budget) {
                bytes += (uint64_t)(h[t1].nt + h[t1].ns) * sizeof(float4);
                ++t1;
            }
            if (t1 == t0) return GC_ERR_BUDGET;
            Wave w;
            w.t0 = t0; w.t1 = t1;
            w.tg0 = h[t0].tgt_off; w.tg1 = (t1 < T) ? h[t1].tgt_off : NT;
            w.s0 = h[t0].src_off; w.s1 = (t1 < T) ? h[t1].src_off : NS;
            waves.push_back(w);
            t0 = t1;
        }
        need_offsets = true;
    } else {
        waves.push_back(Wave{0, T, 0, NT, 0, NS});
    }
    if (need_offsets) GC_TRY(gc_read_wu_offsets(p, c, wu_off, lj_off));

    // source staging holds one extra float4 per task (pad of odd gravity lists)
    uint64_t max_wt = 0, max_ws = 0;
    for (const Wave &w : waves) {
        if (w.tg1 - w.tg0 > max_wt) max_wt = w.tg1 - w.tg0;
        if (w.s1 - w.s0 + (w.t1 - w.t0) > max_ws) max_ws = w.s1 - w.s0 + (w.t1 - w.t0);
    }
    GC_TRY(c.stg_tgt.reserve((max_wt + 1) * sizeof(float4)));
    GC_TRY(c.stg_src.reserve((max_ws + 1) * sizeof(float4)));
    uint64_t max_we = 0;   // entries of the largest wave (entry slots)
    for (const Wave &w : waves)
        if (w.tg1 - w.tg0 + w.s1 - w.s0 > max_we) max_we = w.tg1 - w.tg0 + w.s1 - w.s0;
    if (!one_wave) GC_TRY(c.ent.reserve((max_we + 1) * sizeof(uint32_t)));
    if (max_list > 16384) {   // lists beyond one shared-memory sort: chunk + merge
        GC_TRY(c.merge_a.reserve((max_wt + max_ws + 1) * sizeof(uint64_t)));
        GC_TRY(c.merge_b.reserve((max_wt + max_ws + 1) * sizeof(uint64_t)));
    }

    c.waves.clear();
    for (const Wave &w : waves) {
        WaveRange r{w.t0, w.t1, w.tg0, w.tg1, w.s0, w.s1, 0, W, 0, L};
        if (need_offsets) {
            r.w0 = wu_off[w.t0]; r.w1 = wu_off[w.t1];
            r.l0 = lj_off[w.t0]; r.l1 = lj_off[w.t1];
        }
        c.waves.push_back(r);
    }
    c.msrc = max_wt + 1;

    float ms_res = 0, ms_pack = 0, ms_int = 0;
    const uint32_t *tgt_ids = c.tgt_ids.as<uint32_t>();
    const uint32_t *src_ids = c.src_ids.as<uint32_t>();
    for (size_t k = 0; k < waves.size(); ++k) {
        const Wave &w = waves[k];
        if (one_wave) {
            rc = gc_residency_finish(p);   // issued with the preparation
        } else {
            GC_CUDA_TRY(cudaEventRecord(c.ev_stage[0], c.s));
            rc = gc_residency(p, tgt_ids + w.tg0, w.tg1 - w.tg0, src_ids + w.s0, w.s1 - w.s0,
                              c.ent.as<uint32_t>());
        }
        if (rc != GC_OK) return rc;
        GC_CUDA_TRY(cudaEventRecord(c.ev_stage[1], c.s));
        GC_TRY(gc_pack(p, c, w.t0, w.t1, w.tg0, w.s0, max_wt + 1, c.ent.as<uint32_t>(),
                       w.tg1 - w.tg0));
        GC_CUDA_TRY(cudaEventRecord(c.ev_stage[2], c.s));
        uint64_t w0 = 0, w1 = W, l0 = 0, l1 = L;
        if (need_offsets) {
            w0 = wu_off[w.t0]; w1 = wu_off[w.t1];
            l0 = lj_off[w.t0]; l1 = lj_off[w.t1];
        }
        if (!per_task) {
            GC_TRY(gc_interact_range(p, c, w0, w1, l0, l1, w.tg0, w.s0, w.t0));
        } else {
            for (uint64_t t = w.t0; t < w.t1; ++t)
                GC_TRY(gc_interact_one_task(p, c, wu_off[t], wu_off[t + 1], lj_off[t],
                                            lj_off[t + 1], w.tg0, w.s0, w.t0));
        }
        GC_CUDA_TRY(cudaEventRecord(c.ev_stage[3], c.s));
        if (waves.size() > 1) {
            float a = 0, b = 0, d = 0;
            GC_CUDA_TRY(cudaEventSynchronize(c.ev_stage[3]));
            cudaEventElapsedTime(&a, c.ev_stage[0], c.ev_stage[1]);
            cudaEventElapsedTime(&b, c.ev_stage[1], c.ev_stage[2]);
            cudaEventElapsedTime(&d, c.ev_stage[2], c.ev_stage[3]);
            ms_res += a; ms_pack += b; ms_int += d;
        }
    }
    // pack done: later pool changes may proceed
    GC_CUDA_TRY(cudaEventRecord(c.ev_packed, c.s));
    if (prev && prev != &c && prev->valid) GC_CUDA_TRY(cudaStreamWaitEvent(c.s, prev->ev_scattered, 0));
    GC_TRY(gc_apply_totals_reset(p, c.s));
    GC_TRY(gc_scatter(p, c));
    GC_CUDA_TRY(cudaEventRecord(c.ev_scattered, c.s));
    GC_CUDA_TRY(cudaEventRecord(c.ev_stage[4], c.s));
    GC_CUDA_TRY(cudaEventRecord(c.ev_done, c.s));
    c.multiwave_ms[0] = ms_res;
    c.multiwave_ms[1] = ms_pack;
    c.multiwave_ms[2] = ms_int;
    c.n_waves = waves.size();
    c.timing_valid = true;
    c.valid = true;

    gc_stats_t &st = p->stats;
    st.flushes += 1;
    st.tasks += T;
    st.interactions += inter;
    st.last_waves = waves.size();
    st.last_staging_bytes = (NT + NS) * sizeof(float4);

    p->last = p->cur;
    p->submitted_batches += 1;
    p->cur ^= 1;
    p->s = p->ctx[p->cur].s;
    GC_CUDA_TRY(cudaStreamWaitEvent(p->s, c.ev_packed, 0));
    return GC_OK;
}

int gc_flush(gc_pool_t *p) { return flush_impl(p, 0); }

int gc_flush_per_task(gc_pool_t *p) { return flush_impl(p, 1); }

int gc_wait(gc_pool_t *p, uint64_t batch, uint64_t timeout_ns)
{
    if (!p) return GC_ERR_ARG;
    if (p->last < 0 || batch >= p->submitted_batches) return GC_ERR_NOT_READY;
    auto device_status = [p]() -> int {
        unsigned long long f = 0;
        if (cudaMemcpy(&f, p->d_ctr + CTR_FLAGS, sizeof f, cudaMemcpyDeviceToHost) != cudaSuccess)
            return GC_ERR_CUDA;
        if (f & GC_FLAG_TIMEOUT) {
            if (gc_clear_flags(p, p->s, GC_FLAG_TIMEOUT) != GC_OK ||
                cudaStreamSynchronize(p->s) != cudaSuccess)
                return GC_ERR_CUDA;
            return GC_ERR_TIMEOUT;
        }
        return GC_OK;
    };
    // the batch's context, or (an older batch) both: stream order makes a
    // later batch on the same context complete after it
    std::vector<cudaEvent_t> evs;
    if (FlushCtx *c = ctx_of(p, batch)) {
        evs.push_back(c->ev_done);
    } else {
        for (int i = 0; i < 2; ++i)
            if (p->ctx[i].valid) evs.push_back(p->ctx[i].ev_done);
    }
    struct timespec t0, t1;
    clock_gettime(CLOCK_MONOTONIC, &t0);
    for (cudaEvent_t e : evs) {
        if (timeout_ns == 0) {
            GC_CUDA_TRY(cudaEventSynchronize(e));
            continue;
        }
        for (;;) {
            cudaError_t q = cudaEventQuery(e);
            if (q == cudaSuccess) break;
            if (q != cudaErrorNotReady) return GC_ERR_CUDA;
            clock_gettime(CLOCK_MONOTONIC, &t1);
            uint64_t el = (uint64_t)(t1.tv_sec - t0.tv_sec) * 1000000000ull +
                          (uint64_t)(t1.tv_nsec - t0.tv_nsec);
            if (el >= timeout_ns) return GC_ERR_TIMEOUT;
        }
    }
    return device_status();
}

int gc_join(gc_pool_t *p, void *stream)
{
    if (!p) return GC_ERR_ARG;
    cudaStream_t s = (cudaStream_t)stream;
    for (int i = 0; i < 2; ++i)
        if (p->ctx[i].ev_done && p->ctx[i].s != s)
            GC_CUDA_TRY(cudaStreamWaitEvent(s, p->ctx[i].ev_done, 0));
    // the last stream-ordered totals read's copy out
    if (p->at_used) GC_CUDA_TRY(cudaStreamWaitEvent(s, p->ev_at, 0));
    if (p->s != s) {
        // work issued on the pool's stream after the last flush (uploads,
        // task builds, graph replays)
        cudaEvent_t e = nullptr;
        GC_CUDA_TRY(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
        int rc = GC_OK;
        if (cudaEventRecord(e, p->s) != cudaSuccess || cudaStreamWaitEvent(s, e, 0) != cudaSuccess)
            rc = GC_ERR_CUDA;
        cudaEventDestroy(e);
        return rc;
    }
    return GC_OK;
}

int gc_batch_done(gc_pool_t *p, uint64_t batch, int *done_out)
{
    if (!p || !done_out) return GC_ERR_ARG;
    *done_out = 0;
    if (p->last < 0 || batch >= p->submitted_batches) return GC_OK;
    FlushCtx *c = ctx_of(p, batch);
    cudaError_t q = cudaSuccess;
    if (c) {
        q = cudaEventQuery(c->ev_done);
    } else {
        for (int i = 0; i < 2 && q == cudaSuccess; ++i)
            if (p->ctx[i].valid) q = cudaEventQuery(p->ctx[i].ev_done);
    }
    if (q == cudaSuccess) *done_out = 1;
    else if (q != cudaErrorNotReady) return GC_ERR_CUDA;
    return GC_OK;
}

// ---- results -----------------------------------------------------------------------

static FlushCtx *result_ctx(gc_pool *p)
{
    FlushCtx *c = last_ctx(p);
    return (c && c->valid) ? c : nullptr;
}

int gc_result_rows(gc_pool_t *p, uint64_t *rows_out)
{
    if (!p || !rows_out) return GC_ERR_ARG;
    FlushCtx *c = result_ctx(p);
    *rows_out = c ? c->n_rows : 0;
    return GC_OK;
}

int gc_read_batch_results(gc_pool_t *p, uint64_t first_row, uint64_t n_rows, float *out)
{
    if (!p || (n_rows && !out)) return GC_ERR_ARG;
    FlushCtx *c = result_ctx(p);
    if (!c || first_row + n_rows > c->n_rows) return GC_ERR_ARG;
    GC_CUDA_TRY(cudaEventSynchronize(c->ev_done));
    GC_CUDA_TRY(cudaMemcpy(out, c->res.as<float4>() + 2 * first_row, n_rows * 2 * sizeof(float4),
                           cudaMemcpyDeviceToHost));
    return GC_OK;
}

int gc_read_batch_values(gc_pool_t *p, uint64_t first_row, uint64_t n_rows, double *values4)
{
    if (!p || (n_rows && !values4)) return GC_ERR_ARG;
    FlushCtx *c = result_ctx(p);
    if (!c || first_row + n_rows > c->n_rows) return GC_ERR_ARG;
    if (n_rows == 0) return GC_OK;
    GC_TRY(grow_keep(p->io_b, n_rows * sizeof(gcd4) + 32, 0, p->s));
    GC_CUDA_TRY(cudaStreamWaitEvent(p->s, c->ev_done, 0));
    unsigned g = (unsigned)((n_rows + 255) / 256);
    if (g > 65535u * 8) g = 65535u * 8;
    ++p->stats.kernel_launches;
    k_row_values<<<g, 256, 0, p->s>>>(c->res.as<float4>() + 2 * first_row, n_rows,
                                      p->io_b.as<gcd4>());
    GC_CUDA_TRY(cudaGetLastError());
    GC_CUDA_TRY(cudaMemcpyAsync(values4, p->io_b.p, n_rows * sizeof(gcd4),
                                cudaMemcpyDeviceToHost, p->s));
    GC_CUDA_TRY(cudaStreamSynchronize(p->s));
    return GC_OK;
}

int gc_row_values(const float *rows, uint64_t n_rows, double *values4)
{
    if (n_rows && (!rows || !values4)) return GC_ERR_ARG;
    for (uint64_t i = 0; i < n_rows; ++i)
        for (int k = 0; k < 4; ++k)
            values4[4 * i + k] = (double)rows[8 * i + k] - (double)rows[8 * i + 4 + k];
    return GC_OK;
}

int gc_read_batch_rows(gc_pool_t *p, uint64_t batch, uint64_t first_row, uint64_t n_rows,
                       float *out)
{
    if (!p || (n_rows && !out)) return GC_ERR_ARG;
    FlushCtx *c = ctx_of(p, batch);
    if (!c || !c->valid) return GC_ERR_ARG;
    if (first_row + n_rows > c->n_rows) return GC_ERR_ARG;
    GC_CUDA_TRY(cudaEventSynchronize(c->ev_done));
    if (n_rows)
        GC_CUDA_TRY(cudaMemcpy(out, c->res.as<float4>() + 2 * first_row,
                               n_rows * 2 * sizeof(float4), cudaMemcpyDeviceToHost));
    return GC_OK;
}

static int ensure_host_tasks(FlushCtx &c)
{
    if (c.host_tasks_valid) return GC_OK;
    c.host_tasks.resize(c.n_tasks);
    GC_CUDA_TRY(cudaEventSynchronize(c.ev_done));
    GC_CUDA_TRY(cudaMemcpy(c.host_tasks.data(), c.tasks.p, c.n_tasks * sizeof(TaskRec),
                           cudaMemcpyDeviceToHost));
    c.task_index.clear();
    c.task_index.reserve(c.n_tasks * 2);
    for (uint64_t t = 0; t < c.n_tasks; ++t) c.task_index[c.host_tasks[t].task_id] = t;
    c.host_tasks_valid = true;
    return GC_OK;
}

int gc_read_results(gc_pool_t *p, const uint64_t *task_ids, uint64_t n, float *out)
{
    if (!p || (n && (!task_ids || !out))) return GC_ERR_ARG;
    FlushCtx *c = result_ctx(p);
    if (!c) return GC_ERR_NOT_READY;
    GC_TRY(ensure_host_tasks(*c));
    std::vector<float4> all(2 * c->n_rows + 2);
    if (c->n_rows)
        GC_CUDA_TRY(cudaMemcpy(all.data(), c->res.p, c->n_rows * 2 * sizeof(float4),
                               cudaMemcpyDeviceToHost));
    uint64_t w = 0;
    for (uint64_t i = 0; i < n; ++i) {
        auto it = c->task_index.find(task_ids[i]);
        if (it == c->task_index.end()) return GC_ERR_ARG;
        const TaskRec &r = c->host_tasks[it->second];
        uint64_t rows = r.nt + (r.kind == GC_LJ_PAIR ? r.ns : 0u);
        std::memcpy(out + 8 * w, &all[2 * r.row_off], rows * 2 * sizeof(float4));
        w += rows;
    }
    return GC_OK;
}

int gc_read_totals(gc_pool_t *p, const uint32_t *ids, uint64_t n, double *acc4)
{
    if (!p || (n && (!ids || !acc4))) return GC_ERR_ARG;
    if (n == 0) return GC_OK;
    GC_TRY(order_after_scatters(p));
    GC_TRY(gc_apply_totals_reset(p, p->s));
    GC_TRY(grow_keep(p->io_a, n * 4 + 16, 0, p->s));
    GC_TRY(grow_keep(p->io_b, n * sizeof(gcd4) + 32, 0, p->s));
    int rc = GC_OK;
    if (cudaMemcpyAsync(p->io_a.p, ids, n * 4, cudaMemcpyHostToDevice, p->s) != cudaSuccess)
        rc = GC_ERR_CUDA;
    if (rc == GC_OK) {
        unsigned g = (unsigned)((n + 255) / 256);
        if (g > 65535u * 8) g = 65535u * 8;
        ++p->stats.kernel_launches;
        k_gather_totals<<<g, 256, 0, p->s>>>(p->d_totals, p->io_a.as<uint32_t>(), n,
                                             p->cfg.id_capacity, p->io_b.as<gcd4>());
        if (cudaMemcpyAsync(acc4, p->io_b.p, n * sizeof(gcd4), cudaMemcpyDeviceToHost, p->s) !=
                cudaSuccess ||
            cudaStreamSynchronize(p->s) != cudaSuccess)
            rc = GC_ERR_CUDA;
    }
    return rc;
}

int gc_read_totals_async(gc_pool_t *p, const uint32_t *ids, uint64_t n, double *acc4)
{
    if (!p || (n && (!ids || !acc4))) return GC_ERR_ARG;
    if (n == 0) return GC_OK;
    GC_TRY(async_init(p));
    GC_TRY(order_after_scatters(p));
    GC_TRY(gc_apply_totals_reset(p, p->s));
    GC_TRY(grow_keep(p->at_ids, n * 4 + 16, 0, p->s));
    GC_TRY(grow_keep(p->at_out, n * sizeof(gcd4) + 32, 0, p->s));
    // ids in: after the previous gather has read at_ids
    if (p->at_used) GC_CUDA_TRY(cudaStreamWaitEvent(p->cs_in, p->ev_at_g, 0));
    GC_CUDA_TRY(cudaMemcpyAsync(p->at_ids.p, ids, n * 4, cudaMemcpyHostToDevice, p->cs_in));
    GC_CUDA_TRY(cudaEventRecord(p->ev_at_in, p->cs_in));
    // gather on the pool's stream (after every scatter queued so far, before
    // any later one): after the ids are in and the previous totals copied out
    GC_CUDA_TRY(cudaStreamWaitEvent(p->s, p->ev_at_in, 0));
    if (p->at_used) GC_CUDA_TRY(cudaStreamWaitEvent(p->s, p->ev_at, 0));
    unsigned g = (unsigned)((n + 255) / 256);
    if (g > 65535u * 8) g = 65535u * 8;
    ++p->stats.kernel_launches;
    k_gather_totals<<<g, 256, 0, p->s>>>(p->d_totals, p->at_ids.as<uint32_t>(), n,
                                         p->cfg.id_capacity, p->at_out.as<gcd4>());
    GC_CUDA_TRY(cudaGetLastError());
    GC_CUDA_TRY(cudaEventRecord(p->ev_at_g, p->s));
    // totals out on their own stream: the work queued next on the pool's
    // stream does not wait for this copy
    GC_CUDA_TRY(cudaStreamWaitEvent(p->cs_out, p->ev_at_g, 0));
    GC_CUDA_TRY(cudaMemcpyAsync(acc4, p->at_out.p, n * sizeof(gcd4), cudaMemcpyDeviceToHost,
                                p->cs_out));
    GC_CUDA_TRY(cudaEventRecord(p->ev_at, p->cs_out));
    p->at_used = true;
    return GC_OK;
}

int gc_totals_device(gc_pool_t *p, const double **totals_dev)
{
    if (!p || !totals_dev) return GC_ERR_ARG;
    if (p->totals_reset_pending) {
        GC_TRY(order_after_scatters(p));
        GC_TRY(gc_apply_totals_reset(p, p->s));
    }
    *totals_dev = (const double *)p->d_totals;
    return GC_OK;
}

// The zeroing is deferred to the next consumer of the totals: the next
// batch's scatter (on its own stream, after the previous batch's scatter),
// a read, a graph replay or a kick-drift.  Work issued meanwhile (uploads,
// task builds) therefore does not wait for the batches in flight.
int gc_reset_totals(gc_pool_t *p)
{
    if (!p) return GC_ERR_ARG;
    p->totals_reset_pending = true;
    return GC_OK;
}

int gc_stats(gc_pool_t *p, gc_stats_t *out)
{
    if (!p || !out) return GC_ERR_ARG;
    GC_CUDA_TRY(cudaStreamSynchronize(p->ctx[0].s));
    GC_CUDA_TRY(cudaStreamSynchronize(p->ctx[1].s));
    unsigned long long c[CTR_COUNT];
    GC_CUDA_TRY(cudaMemcpy(c, p->d_ctr, sizeof c, cudaMemcpyDeviceToHost));
    for (int i = 0; i < 2; ++i) count_timing(p, p->ctx[i], false);
    *out = p->stats;
    out->updates = c[CTR_UPDATES];
    FlushCtx *l = result_ctx(p);
    out->lj_pairs_in_cutoff = 0;
    if (l) {
        unsigned long long v = 0;
        GC_CUDA_TRY(cudaMemcpy(&v, l->d_ctr + FC_LJ_IN, sizeof v, cudaMemcpyDeviceToHost));
        out->lj_pairs_in_cutoff = v;
    }
    return GC_OK;
}

// Stage times of a context's completed batch (its events have fired).
static void timings_of(const FlushCtx &c, float ms[5])
{
    if (c.n_waves > 1) {
        ms[0] = c.multiwave_ms[0];
        ms[1] = c.multiwave_ms[1];
        ms[2] = c.multiwave_ms[2];
        cudaEventElapsedTime(&ms[3], c.ev_stage[3], c.ev_stage[4]);
        ms[4] = ms[0] + ms[1] + ms[2] + ms[3];
        return;
    }
    cudaEventElapsedTime(&ms[0], c.ev_stage[0], c.ev_stage[1]);
    cudaEventElapsedTime(&ms[1], c.ev_stage[1], c.ev_stage[2]);
    cudaEventElapsedTime(&ms[2], c.ev_stage[2], c.ev_stage[3]);
    cudaEventElapsedTime(&ms[3], c.ev_stage[3], c.ev_stage[4]);
    cudaEventElapsedTime(&ms[4], c.ev_stage[0], c.ev_stage[4]);
}

// Add a completed batch's stage times to the pool's sums, once.  block:
// wait for the batch; otherwise count it only if it has completed.
static void count_timing(gc_pool *p, FlushCtx &c, bool block)
{
    if (!c.timing_valid || c.timing_counted) return;
    if (block) {
        if (cudaEventSynchronize(c.ev_stage[4]) != cudaSuccess) return;
    } else if (cudaEventQuery(c.ev_stage[4]) != cudaSuccess) {
        cudaGetLastError();
        return;
    }
    float ms[5];
    timings_of(c, ms);
    for (int i = 0; i < 5; ++i) p->stats.stage_ms_sum[i] += ms[i];
    ++p->stats.timed_batches;
    c.timing_counted = true;
}

int gc_last_timings(gc_pool_t *p, float ms[5])
{
    if (!p || !ms) return GC_ERR_ARG;
    FlushCtx *c = result_ctx(p);
    if (!c || !c->timing_valid) return GC_ERR_NOT_READY;
    GC_CUDA_TRY(cudaEventSynchronize(c->ev_stage[4]));
    timings_of(*c, ms);
    count_timing(p, *c, true);
    return GC_OK;
}

// ---- introspection -----------------------------------------------------------------

int gc_batch_sizes(gc_pool_t *p, uint64_t *n_tasks, uint64_t *n_tgt, uint64_t *n_src)
{
    if (!p) return GC_ERR_ARG;
    FlushCtx *c = result_ctx(p);
    if (n_tasks) *n_tasks = c ? c->n_tasks : 0;
    if (n_tgt) *n_tgt = c ? c->n_tgt : 0;
    if (n_src) *n_src = c ? c->n_src : 0;
    return GC_OK;
}

int gc_read_entry_slots(gc_pool_t *p, uint32_t *tgt_slots, uint32_t *src_slots)
{
    FlushCtx *c = p ? result_ctx(p) : nullptr;
    if (!c) return GC_ERR_STATE;
    GC_CUDA_TRY(cudaEventSynchronize(c->ev_done));
    // looked up in the chare table now (the pack reads the table directly)
    GC_TRY(grow_keep(p->io_a, (c->n_tgt + c->n_src + 1) * 4, 0, c->s));
    uint32_t *d = p->io_a.as<uint32_t>();
    int rc = gc_entry_slots(p, c->s, c->tgt_ids.as<uint32_t>(), c->n_tgt, d);
    if (rc == GC_OK) rc = gc_entry_slots(p, c->s, c->src_ids.as<uint32_t>(), c->n_src, d + c->n_tgt);
    if (rc == GC_OK && cudaStreamSynchronize(c->s) != cudaSuccess) rc = GC_ERR_CUDA;
    if (rc == GC_OK && tgt_slots && c->n_tgt &&
        cudaMemcpy(tgt_slots, d, c->n_tgt * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = GC_ERR_CUDA;
    if (rc == GC_OK && src_slots && c->n_src &&
        cudaMemcpy(src_slots, d + c->n_tgt, c->n_src * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
        rc = GC_ERR_CUDA;
    return rc;
}

int gc_read_pack_perm(gc_pool_t *p, uint32_t *tgt_perm, uint32_t *src_perm)
{
    FlushCtx *c = p ? result_ctx(p) : nullptr;
    if (!c) return GC_ERR_STATE;
    GC_CUDA_TRY(cudaEventSynchronize(c->ev_done));
    if (tgt_perm && c->n_tgt)
        GC_CUDA_TRY(cudaMemcpy(tgt_perm, c->tgt_perm.p, c->n_tgt * 4, cudaMemcpyDeviceToHost));
    if (src_perm && c->n_src)
        GC_CUDA_TRY(cudaMemcpy(src_perm, c->src_perm.p, c->n_src * 4, cudaMemcpyDeviceToHost));
    return GC_OK;
}

int gc_read_residency(gc_pool_t *p, uint32_t *slot_of_id, uint32_t *id_of_slot,
                      uint32_t *last_use)
{
    if (!p) return GC_ERR_ARG;
    GC_CUDA_TRY(cudaStreamSynchronize(p->ctx[0].s));
    GC_CUDA_TRY(cudaStreamSynchronize(p->ctx[1].s));
    if (slot_of_id)
        GC_CUDA_TRY(cudaMemcpy(slot_of_id, p->d_slot_of_id, p->cfg.id_capacity * 4,
                               cudaMemcpyDeviceToHost));
    if (id_of_slot)
        GC_CUDA_TRY(cudaMemcpy(id_of_slot, p->d_id_of_slot, p->cfg.pool_capacity * 4,
                               cudaMemcpyDeviceToHost));
    if (last_use)
        GC_CUDA_TRY(cudaMemcpy(last_use, p->d_last_use, p->cfg.pool_capacity * 4,
                               cudaMemcpyDeviceToHost));
    return GC_OK;
}

int gc_read_evicted(gc_pool_t *p, uint32_t *ids, uint64_t cap, uint64_t *n_out)
{
    if (!p || !n_out) return GC_ERR_ARG;
    GC_CUDA_TRY(cudaStreamSynchronize(p->ctx[0].s));
    GC_CUDA_TRY(cudaStreamSynchronize(p->ctx[1].s));
    *n_out = p->n_evicted_last;
    uint64_t k = p->n_evicted_last < cap ? p->n_evicted_last : cap;
    if (k && ids) GC_CUDA_TRY(cudaMemcpy(ids, p->evicted.p, k * 4, cudaMemcpyDeviceToHost));
    return GC_OK;
}

}  // extern "C"
