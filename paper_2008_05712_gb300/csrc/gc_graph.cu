// gc_graph.cu -- a combined batch captured once and replayed as a CUDA graph
// (the persistent + graph form of the Section 3.1 combined launch).
//
// Capture runs the pending batch as an ordinary flush, which settles the
// chare table (every id of the batch resident, Section 3.2) and every size
// that a flush otherwise reads back to the host.  The graph then records the
// device work of one more execution of the same batch on buffers it owns:
// the last-use update of the batch's distinct ids, and per wave the pack and
// the interaction kernels, and the per-id FP64 accumulation in the order the
// capture run established.  A replay reads the current pool values, so
// values re-uploaded in place between replays are used; it is valid while no
// slot has been assigned or freed since capture.
#include <cub/cub.cuh>

#include "gc_common.cuh"

struct gc_graph {
    gc_pool *p = nullptr;
    FlushCtx c;                       // the graph's own batch buffers and stream
    DBuf uniq;                        // distinct ids of the batch
    DBuf ent;                         // slot of every entry (targets, then sources)
    uint64_t n_uniq = 0;
    uint32_t *d_epoch = nullptr;      // epoch of the current replay (device)
    uint32_t *h_epoch = nullptr;      // pinned staging of it
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    cudaEvent_t ev_done = nullptr;
    uint64_t version = 0;             // pool table version at capture
    uint64_t tasks = 0, entries = 0, interactions = 0, launches = 0;
};

namespace {

__global__ void k_flag_first(const uint32_t *sorted, uint64_t n, uint32_t *flag)
{
    GRID_STRIDE(i, n) flag[i] = (i == 0 || sorted[i] != sorted[i - 1]) ? 1u : 0u;
}

__global__ void k_scatter_first(const uint32_t *sorted, const uint32_t *flag,
                                const uint32_t *pos, uint64_t n, uint32_t *out)
{
    GRID_STRIDE(i, n) if (flag[i]) out[pos[i]] = sorted[i];
}

__global__ void k_count_missing(const uint32_t *ids, uint64_t n, const uint32_t *slot_of_id,
                                unsigned long long *missing)
{
    unsigned long long m = 0;
    GRID_STRIDE(i, n) m += (slot_of_id[ids[i]] == GC_NONE) ? 1ull : 0ull;
    for (int o = 16; o; o >>= 1) m += __shfl_xor_sync(0xffffffffu, m, o);
    if ((threadIdx.x & 31) == 0 && m) atomicAdd(missing, m);
}

__global__ void k_touch_epoch(const uint32_t *uniq, uint64_t U, const uint32_t *slot_of_id,
                              uint32_t *last_use, const uint32_t *epoch)
{
    const uint32_t e = *epoch;
    GRID_STRIDE(k, U) last_use[slot_of_id[uniq[k]]] = e;
}

void destroy_graph(gc_graph *g)
{
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->ev_done) cudaEventDestroy(g->ev_done);
    if (g->d_epoch) cudaFree(g->d_epoch);
    if (g->h_epoch) cudaFreeHost(g->h_epoch);
    g->uniq.release();
    g->ent.release();
    free_ctx(g->c);
    delete g;
}

// The batch's distinct ids (sorted) into g->uniq, and a check that every
// entry is resident.
int distinct_ids(gc_pool *p, gc_graph *g, uint64_t *missing_out)
{
    FlushCtx &c = g->c;
    const uint64_t n = c.n_tgt + c.n_src;
    const int maxb = p->num_sms * 16;
    // all entry ids, contiguous: targets then sources
    DBuf all, sorted, vals, flag, pos, cub_tmp;
    int rc = GC_OK;
    auto cleanup = [&]() {
        all.release(); sorted.release(); vals.release(); flag.release(); pos.release();
        cub_tmp.release();
    };
    if ((rc = all.reserve((n + 1) * 4)) != GC_OK || (rc = sorted.reserve((n + 1) * 4)) != GC_OK ||
        (rc = vals.reserve((n + 1) * 8)) != GC_OK || (rc = flag.reserve((n + 1) * 4)) != GC_OK ||
        (rc = pos.reserve((n + 2) * 4)) != GC_OK) {
        cleanup();
        return rc;
    }
    uint32_t *a = all.as<uint32_t>();
    if (c.n_tgt && cudaMemcpyAsync(a, c.tgt_ids.p, c.n_tgt * 4, cudaMemcpyDeviceToDevice, c.s))
        rc = GC_ERR_CUDA;
    if (rc == GC_OK && c.n_src &&
        cudaMemcpyAsync(a + c.n_tgt, c.src_ids.p, c.n_src * 4, cudaMemcpyDeviceToDevice, c.s))
        rc = GC_ERR_CUDA;
    unsigned long long *miss = (unsigned long long *)vals.p;   // scratch word first
    if (rc == GC_OK && cudaMemsetAsync(miss, 0, sizeof *miss, c.s)) rc = GC_ERR_CUDA;
    if (rc == GC_OK)
        k_count_missing<<<grid_for(n, 256, maxb), 256, 0, c.s>>>(a, n, p->d_slot_of_id, miss);
    unsigned long long h_miss = 0;
    if (rc == GC_OK &&
        (cudaMemcpyAsync(&h_miss, miss, sizeof h_miss, cudaMemcpyDeviceToHost, c.s) ||
         cudaStreamSynchronize(c.s)))
        rc = GC_ERR_CUDA;
    if (rc == GC_OK && h_miss == 0) {
        int bits = 1;
        while (bits < 32 && ((uint64_t)1 << bits) < p->cfg.id_capacity) ++bits;
        uint32_t *vin = (uint32_t *)vals.p, *vout = vin + (n + 1);
        k_flag_first<<<grid_for(n, 256, maxb), 256, 0, c.s>>>(a, n, flag.as<uint32_t>());
        rc = gc_sort_pairs_u32(cub_tmp, a, sorted.as<uint32_t>(), flag.as<uint32_t>(), vout, n,
                               bits, c.s);   // values unused
        uint32_t *srt = sorted.as<uint32_t>();
        if (rc == GC_OK) {
            k_flag_first<<<grid_for(n, 256, maxb), 256, 0, c.s>>>(srt, n, flag.as<uint32_t>());
            rc = gc_exclusive_scan_u32(cub_tmp, flag.as<uint32_t>(), pos.as<uint32_t>(), n + 1,
                                       c.s);
        }
        uint32_t h_u = 0;
        if (rc == GC_OK &&
            (cudaMemcpyAsync(&h_u, pos.as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, c.s) ||
             cudaStreamSynchronize(c.s)))
            rc = GC_ERR_CUDA;
        if (rc == GC_OK) rc = g->uniq.reserve(((uint64_t)h_u + 1) * 4);
        if (rc == GC_OK) {
            k_scatter_first<<<grid_for(n, 256, maxb), 256, 0, c.s>>>(
                srt, flag.as<uint32_t>(), pos.as<uint32_t>(), n, g->uniq.as<uint32_t>());
            g->n_uniq = h_u;
            if (cudaStreamSynchronize(c.s) != cudaSuccess) rc = GC_ERR_CUDA;
        }
    }
    if (rc == GC_OK && cudaGetLastError() != cudaSuccess) rc = GC_ERR_CUDA;
    cleanup();
    *missing_out = h_miss;
    return rc;
}

}  // namespace

extern "C" int gc_graph_capture(gc_pool_t *p, gc_graph_t **out)
{
    if (!p || !out) return GC_ERR_ARG;
    *out = nullptr;
    if (p->nb_tasks == 0) return GC_ERR_STATE;
    GC_TRY(gc_flush(p));
    FlushCtx &src = p->ctx[p->last];
    GC_CUDA_TRY(cudaEventSynchronize(src.ev_done));
    {
        unsigned long long f = 0;
        GC_CUDA_TRY(cudaMemcpy(&f, p->d_ctr + CTR_FLAGS, sizeof f, cudaMemcpyDeviceToHost));
        if (f & GC_FLAG_TIMEOUT) {   // reported once, like gc_wait
            GC_TRY(gc_clear_flags(p, p->s, GC_FLAG_TIMEOUT));
            GC_CUDA_TRY(cudaStreamSynchronize(p->s));
            return GC_ERR_TIMEOUT;
        }
    }
    gc_graph *g = new gc_graph();
    g->p = p;
    int rc = init_ctx(g->c, nullptr);
    if (rc == GC_OK && (cudaMalloc((void **)&g->d_epoch, 4) != cudaSuccess ||
                        cudaHostAlloc((void **)&g->h_epoch, 4, cudaHostAllocDefault) !=
                            cudaSuccess ||
                        cudaEventCreateWithFlags(&g->ev_done, cudaEventDisableTiming) !=
                            cudaSuccess))
        rc = GC_ERR_CUDA;
    if (rc != GC_OK) {
        destroy_graph(g);
        return rc;
    }
    FlushCtx &c = g->c;
    // take over the capture run's buffers (its batch is complete)
    std::swap(c.tasks, src.tasks);
    std::swap(c.tgt_ids, src.tgt_ids);
    std::swap(c.src_ids, src.src_ids);
    std::swap(c.tgt_perm, src.tgt_perm);
    std::swap(c.src_perm, src.src_perm);
    std::swap(c.stg_tgt, src.stg_tgt);
    std::swap(c.stg_src, src.stg_src);
    std::swap(c.wu, src.wu);
    std::swap(c.lj_list, src.lj_list);
    std::swap(c.res, src.res);
    std::swap(c.row_id, src.row_id);
    std::swap(c.rid_sorted, src.rid_sorted);
    std::swap(c.row_sorted, src.row_sorted);
    std::swap(c.runs, src.runs);
    std::swap(c.merge_a, src.merge_a);
    std::swap(c.merge_b, src.merge_b);
    c.n_tasks = src.n_tasks;
    c.n_tgt = src.n_tgt;
    c.n_src = src.n_src;
    c.n_rows = src.n_rows;
    c.waves = src.waves;
    c.msrc = src.msrc;
    c.max_list = src.max_list;
    c.md_struct = src.md_struct;
    c.md_m = src.md_m;
    c.md_dim = src.md_dim;
    c.unique_rows = src.unique_rows;
    c.n_waves = src.n_waves;
    c.valid = true;
    src.valid = false;    // its arrays now belong to the graph
    src.host_tasks_valid = false;
    GC_CUDA_TRY(cudaMemcpyAsync(c.d_ctr + FC_RUNS, src.d_ctr + FC_RUNS,
                                sizeof(unsigned long long), cudaMemcpyDeviceToDevice, c.s));
    GC_CUDA_TRY(cudaStreamWaitEvent(c.s, src.ev_done, 0));
    uint64_t missing = 0;
    rc = distinct_ids(p, g, &missing);
    if (rc == GC_OK && missing) rc = GC_ERR_POOL_FULL;   // the batch does not fit the pool
    g->tasks = c.n_tasks;
    g->entries = c.n_tgt + c.n_src;
    if (rc != GC_OK) {
        destroy_graph(g);
        return rc;
    }
    // the slot of every entry, fixed for the graph's lifetime (a replay is
    // refused once any slot has been assigned or freed)
    if (rc == GC_OK) rc = g->ent.reserve((g->entries + 1) * sizeof(uint32_t));
    if (rc == GC_OK && c.n_tgt)
        rc = gc_entry_slots(p, c.s, c.tgt_ids.as<uint32_t>(), c.n_tgt, g->ent.as<uint32_t>());
    if (rc == GC_OK && c.n_src)
        rc = gc_entry_slots(p, c.s, c.src_ids.as<uint32_t>(), c.n_src,
                            g->ent.as<uint32_t>() + c.n_tgt);
    if (rc != GC_OK) {
        destroy_graph(g);
        return rc;
    }
    {
        // interactions of the batch, as the flush counted them
        unsigned long long inter = 0;
        GC_CUDA_TRY(cudaMemcpy(&inter, src.d_ctr + FC_INTER, sizeof inter,
                               cudaMemcpyDeviceToHost));
        g->interactions = inter;
    }

    // record one execution of the batch's device work
    const gc_stats_t saved = p->stats;
    const uint32_t saved_sched = p->wu_schedule;
    p->wu_schedule = GC_SCHED_FIFO;   // the work units keep the capture run's order
    const int maxb = p->num_sms * 16;
    if (cudaStreamBeginCapture(c.s, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        p->wu_schedule = saved_sched;
        destroy_graph(g);
        return GC_ERR_CUDA;
    }
    if (g->n_uniq)
        k_touch_epoch<<<grid_for(g->n_uniq, 256, maxb), 256, 0, c.s>>>(
            g->uniq.as<uint32_t>(), g->n_uniq, p->d_slot_of_id, p->d_last_use, g->d_epoch);
    for (const WaveRange &w : c.waves) {
        if (rc == GC_OK) {
            // per-wave views of the batch-wide entry slots: targets of the
            // wave, then (at ent_t + ent_nt) its sources
            const uint32_t *et = g->ent.as<uint32_t>() + w.tg0;
            const uint32_t *es = g->ent.as<uint32_t>() + c.n_tgt + w.s0;
            rc = gc_pack(p, c, w.t0, w.t1, w.tg0, w.s0, c.msrc, et, (uint64_t)(es - et));
        }
        if (rc == GC_OK) rc = gc_interact_range(p, c, w.w0, w.w1, w.l0, w.l1, w.tg0, w.s0, w.t0);
    }
    if (rc == GC_OK) rc = gc_scatter_replay(p, c);
    cudaGraph_t graph = nullptr;
    cudaError_t ce = cudaStreamEndCapture(c.s, &graph);
    p->wu_schedule = saved_sched;
    g->launches = p->stats.kernel_launches - saved.kernel_launches;
    p->stats = saved;
    if (rc == GC_OK && ce != cudaSuccess) rc = GC_ERR_CUDA;
    g->graph = graph;
    if (rc == GC_OK && cudaGraphInstantiate(&g->exec, graph, 0) != cudaSuccess) rc = GC_ERR_CUDA;
    if (rc != GC_OK) {
        cudaGetLastError();
        destroy_graph(g);
        return rc;
    }
    g->version = p->table_version;
    *out = g;
    return GC_OK;
}

extern "C" int gc_graph_launch(gc_graph_t *g)
{
    if (!g) return GC_ERR_ARG;
    gc_pool *p = g->p;
    if (p->table_version != g->version) return GC_ERR_STATE;
    p->epoch += 1;
    if (p->epoch == 0 || p->epoch == GC_EPOCH_UNKNOWN) p->epoch = 1;
    // totals accumulate in admission order: after every scatter in flight;
    // the pool's issue stream then waits for this replay
    GC_TRY(order_after_scatters(p));
    GC_TRY(gc_apply_totals_reset(p, p->s));
    cudaEvent_t issue = nullptr;
    GC_CUDA_TRY(cudaEventCreateWithFlags(&issue, cudaEventDisableTiming));
    int rc = GC_OK;
    if (cudaEventRecord(issue, p->s) != cudaSuccess ||
        cudaStreamWaitEvent(g->c.s, issue, 0) != cudaSuccess)
        rc = GC_ERR_CUDA;
    cudaEventDestroy(issue);
    if (rc != GC_OK) return rc;
    *g->h_epoch = p->epoch;
    GC_CUDA_TRY(cudaMemcpyAsync(g->d_epoch, g->h_epoch, 4, cudaMemcpyHostToDevice, g->c.s));
    GC_CUDA_TRY(cudaGraphLaunch(g->exec, g->c.s));
    GC_CUDA_TRY(cudaEventRecord(g->ev_done, g->c.s));
    GC_CUDA_TRY(cudaStreamWaitEvent(p->s, g->ev_done, 0));
    gc_stats_t &st = p->stats;
    st.flushes += 1;
    st.tasks += g->tasks;
    st.entries += g->entries;
    st.interactions += g->interactions;
    st.unique += g->n_uniq;
    st.hits += g->n_uniq;
    st.kernel_launches += g->launches;
    return GC_OK;
}

extern "C" int gc_graph_wait(gc_graph_t *g)
{
    if (!g) return GC_ERR_ARG;
    GC_CUDA_TRY(cudaEventSynchronize(g->ev_done));
    unsigned long long f = 0;
    GC_CUDA_TRY(cudaMemcpy(&f, g->p->d_ctr + CTR_FLAGS, sizeof f, cudaMemcpyDeviceToHost));
    if (f & GC_FLAG_TIMEOUT) {   // reported once, like gc_wait
        GC_TRY(gc_clear_flags(g->p, g->c.s, GC_FLAG_TIMEOUT));
        GC_CUDA_TRY(cudaStreamSynchronize(g->c.s));
        return GC_ERR_TIMEOUT;
    }
    return GC_OK;
}

extern "C" int gc_graph_rows(gc_graph_t *g, uint64_t *rows_out)
{
    if (!g || !rows_out) return GC_ERR_ARG;
    *rows_out = g->c.n_rows;
    return GC_OK;
}

extern "C" int gc_graph_results(gc_graph_t *g, uint64_t first_row, uint64_t n_rows, float *out)
{
    if (!g || (n_rows && !out) || first_row + n_rows > g->c.n_rows) return GC_ERR_ARG;
    GC_CUDA_TRY(cudaEventSynchronize(g->ev_done));
    GC_CUDA_TRY(cudaStreamSynchronize(g->c.s));
    if (n_rows)
        GC_CUDA_TRY(cudaMemcpy(out, g->c.res.as<float4>() + 2 * first_row,
                               n_rows * 2 * sizeof(float4), cudaMemcpyDeviceToHost));
    return GC_OK;
}

extern "C" int gc_graph_destroy(gc_graph_t *g)
{
    if (!g) return GC_ERR_ARG;
    cudaStreamSynchronize(g->c.s);
    destroy_graph(g);
    return GC_OK;
}
