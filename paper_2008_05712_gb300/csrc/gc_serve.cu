// gc_serve.cu -- continuous-batching request loop (the runtime side of
// Section 3.1 of Rengasamy & Vadhiyar, arXiv 2008.05712: requests arrive
// over time, are combined by the adaptive rule and run as combined batches
// while the host keeps admitting new ones).
//
// The loop replays an open-loop arrival schedule in real time.  At every
// iteration it (1) moves arrived requests into the pending queue and tells
// the combiner, (2) retires batches whose completion event has fired,
// stamping each task's latency from its scheduled arrival (so a slow server
// cannot hide queueing delay), (3) when a flush context is free, asks the
// combiner how many pending requests to combine, cuts that number to the
// staging budget, submits the oldest ones and flushes.  Two batches can be
// in flight: the chare-table step and pack of one overlap the interaction
// kernel of the other on the device.  Host-side only; all device work goes
// through the pool API.
#include <algorithm>
#include <cstring>
#include <ctime>
#include <deque>
#include <vector>

#include "gc_common.cuh"

namespace {

uint64_t now_ns()
{
    struct timespec t;
    clock_gettime(CLOCK_MONOTONIC, &t);
    return (uint64_t)t.tv_sec * 1000000000ull + (uint64_t)t.tv_nsec;
}

struct InFlight {
    uint64_t batch;
    uint64_t t0, t1;      // task range [t0, t1)
    uint64_t t_flush;     // loop time of the flush
};

double percentile(std::vector<uint64_t> v, double q)
{
    if (v.empty()) return 0.0;
    std::sort(v.begin(), v.end());
    const double pos = q * (double)(v.size() - 1);
    const size_t i = (size_t)pos;
    const double f = pos - (double)i;
    if (i + 1 >= v.size()) return (double)v.back();
    return (1.0 - f) * (double)v[i] + f * (double)v[i + 1];
}

}  // namespace

extern "C" int gc_serve(gc_pool_t *p, uint64_t n, const uint64_t *arrival_ns,
                        const uint32_t *kinds, const int8_t *shifts, const uint64_t *tgt_off,
                        const uint32_t *tgt_ids, const uint64_t *src_off,
                        const uint32_t *src_ids, const gc_serve_config *cfg,
                        uint64_t *latency_ns_out, float *results_out, gc_serve_report *report)
{
    if (!p || !cfg || !report || (n && (!arrival_ns || !kinds || !tgt_off || !src_off)))
        return GC_ERR_ARG;
    if (cfg->max_in_flight < 1 || cfg->max_in_flight > 2) return GC_ERR_ARG;
    std::memset(report, 0, sizeof *report);
    if (n == 0) return GC_OK;
    for (uint64_t i = 1; i < n; ++i)
        if (arrival_ns[i] < arrival_ns[i - 1]) return GC_ERR_ARG;
    if (p->nb_tasks) return GC_ERR_STATE;   // a pending batch would mix in
    // arrival k is task k mod m
    const uint64_t m = (cfg->task_set && cfg->task_set < n) ? cfg->task_set : n;
    if (m < n && results_out) return GC_ERR_ARG;
    auto task_of = [m](uint64_t k) { return k % m; };

    uint64_t max_size = cfg->max_size;
    if (!max_size) GC_TRY(gc_max_combine_size(p, &max_size));
    gc_combiner_t *comb = nullptr;
    GC_TRY(gc_combiner_create(cfg->policy, max_size, cfg->static_n, cfg->window, &comb));

    // result rows of each task (targets, plus sources of LJ pair tasks)
    std::vector<uint64_t> row_off(m + 1, 0);
    for (uint64_t t = 0; t < m; ++t) {
        const uint64_t nt = tgt_off[t + 1] - tgt_off[t], ns = src_off[t + 1] - src_off[t];
        row_off[t + 1] = row_off[t] + nt + (kinds[t] == GC_LJ_PAIR ? ns : 0);
    }
    // page-lock the caller's id arrays for the call (unless they already
    // are): the per-batch host-to-device copies then run as direct DMA
    // instead of through the driver's pageable staging
    std::vector<void *> pinned;
    uint64_t pinned_bytes = 0;
    auto pin = [&](const void *ptr, uint64_t bytes) {
        if (!ptr || !bytes) return;
        cudaPointerAttributes at;
        if (cudaPointerGetAttributes(&at, ptr) == cudaSuccess &&
            at.type != cudaMemoryTypeUnregistered) {
            pinned_bytes += bytes;
            return;
        }
        cudaGetLastError();
        if (cudaHostRegister(const_cast<void *>(ptr), bytes, cudaHostRegisterDefault) ==
            cudaSuccess) {
            pinned.push_back(const_cast<void *>(ptr));
            pinned_bytes += bytes;
        } else {
            cudaGetLastError();   // stays pageable: slower copies, same results
        }
    };
    if (!cfg->keep_pageable) {
        pin(tgt_ids, tgt_off[m] * sizeof(uint32_t));
        pin(src_ids, src_off[m] * sizeof(uint32_t));
    }
    const uint64_t budget = p->cfg.staging_budget_bytes;
    const uint64_t none = ~0ull;
    std::vector<uint64_t> lat(n, none);
    std::vector<uint64_t> to, so;
    std::deque<InFlight> inflight;
    uint64_t next = 0, head = 0, done = 0;   // arrivals [0,next) queued from `head`
    uint64_t batches = 0, taken_total = 0, busy_ns = 0, last_iter = 0;
    uint64_t submit_ns = 0, flush_ns = 0, retire_ns = 0;
    const uint64_t limit = cfg->timeout_ns ? cfg->timeout_ns : 60000000000ull;
    const uint64_t last_arrival = arrival_ns[n - 1];
    gc_stats_t s0;
    int rc = gc_stats(p, &s0);
    const uint64_t start = now_ns();

    while (rc == GC_OK && done < n) {
        const uint64_t now = now_ns() - start;
        if (!inflight.empty() && now - inflight.front().t_flush > limit) {
            rc = GC_ERR_TIMEOUT;   // a batch did not complete in time
            break;
        }
        while (next < n && arrival_ns[next] <= now) {
            gc_combiner_arrive(comb, arrival_ns[next], 1);
            ++next;
        }
        // retire completed batches, oldest first
        const uint64_t r0 = now_ns();
        while (!inflight.empty()) {
            int fin = 0;
            rc = gc_batch_done(p, inflight.front().batch, &fin);
            if (rc != GC_OK || !fin) break;
            const InFlight f = inflight.front();
            const uint64_t t_done = now_ns() - start;
            rc = gc_wait(p, f.batch, 0);   // device-side status of the batch
            if (rc != GC_OK) break;
            for (uint64_t t = f.t0; t < f.t1; ++t) lat[t] = t_done - arrival_ns[t];
            if (results_out) {
                const uint64_t rows = row_off[f.t1] - row_off[f.t0];
                rc = gc_read_batch_rows(p, f.batch, 0, rows, results_out + 8 * row_off[f.t0]);
                if (rc != GC_OK) break;
            }
            done += f.t1 - f.t0;
            inflight.pop_front();
        }
        retire_ns += now_ns() - r0;
        if (rc != GC_OK) break;
        // past the drain limit: start nothing more, finish what runs
        const bool closed = cfg->drain_ns && next == n && now > last_arrival + cfg->drain_ns;
        if (closed && inflight.empty()) break;
        const uint64_t queued = next - head;
        bool acted = false;
        if (!closed && queued && inflight.size() < cfg->max_in_flight) {
            uint64_t take = 0;
            gc_combiner_poll(comb, now, queued, &take);
            // the static rule fires only on arrivals: drain what is left once
            // the schedule has ended
            if (!take && next == n && cfg->policy == GC_COMBINE_STATIC) take = queued;
            if (take > queued) take = queued;
            if (take) {
                // admission by staging memory: the oldest requests that fit
                uint64_t t1 = head, bytes = 0;
                while (t1 < head + take) {
                    const uint64_t q = task_of(t1);
                    const uint64_t b = ((tgt_off[q + 1] - tgt_off[q]) +
                                        (src_off[q + 1] - src_off[q])) * sizeof(float4);
                    if (budget && bytes + b > budget && t1 > head) break;
                    bytes += b;
                    ++t1;
                }
                // arrivals head .. t1-1: contiguous runs of the task arrays
                uint64_t b_idx = 0;
                const uint64_t s0_ns = now_ns();
                for (uint64_t k = head; k < t1 && rc == GC_OK;) {
                    const uint64_t q0 = task_of(k);
                    const uint64_t len = std::min(t1 - k, m - q0);
                    to.assign(len + 1, 0);
                    so.assign(len + 1, 0);
                    for (uint64_t j = 0; j <= len; ++j) {
                        to[j] = tgt_off[q0 + j] - tgt_off[q0];
                        so[j] = src_off[q0 + j] - src_off[q0];
                    }
                    rc = gc_submit_csr(p, len, nullptr, kinds + q0,
                                       shifts ? shifts + 3 * q0 : nullptr, to.data(),
                                       tgt_ids + tgt_off[q0], so.data(), src_ids + src_off[q0],
                                       0, 0, 0, &b_idx);
                    k += len;
                }
                const uint64_t f0_ns = now_ns();
                submit_ns += f0_ns - s0_ns;
                if (rc == GC_OK) rc = gc_flush(p);
                flush_ns += now_ns() - f0_ns;
                if (rc != GC_OK) break;
                inflight.push_back(InFlight{b_idx, head, t1, now_ns() - start});
                taken_total += t1 - head;
                head = t1;
                ++batches;
                acted = true;
            }
        } else if (queued && !closed) {
            busy_ns += now - last_iter;   // requests ready, no free flush context
        }
        last_iter = now;
        if (!acted && inflight.empty() && next < n && head == next) {
            // idle until the next arrival (or the next poll)
            const uint64_t wake = std::min(arrival_ns[next], now + cfg->poll_ns);
            const uint64_t cur = now_ns() - start;
            if (wake > cur) {
                struct timespec ts;
                const uint64_t d = wake - cur;
                ts.tv_sec = (time_t)(d / 1000000000ull);
                ts.tv_nsec = (long)(d % 1000000000ull);
                nanosleep(&ts, nullptr);
            }
        }
    }
    const uint64_t wall = now_ns() - start;
    gc_combiner_destroy(comb);
    for (void *ptr : pinned) cudaHostUnregister(ptr);
    if (rc != GC_OK) return rc;
    gc_stats_t s1;
    GC_TRY(gc_stats(p, &s1));
    // latency statistics over the served arrivals after the warm-up
    std::vector<uint64_t> meas;
    meas.reserve(n);
    for (uint64_t k = 0; k < n; ++k)
        if (lat[k] != none && arrival_ns[k] >= cfg->warmup_ns) meas.push_back(lat[k]);
    report->tasks = n;
    report->batches = batches;
    report->interactions = s1.interactions - s0.interactions;
    report->wall_s = (double)wall * 1e-9;
    report->interactions_per_s = (double)report->interactions / report->wall_s;
    report->measured = meas.size();
    report->unserved = n - done;
    if (!meas.empty()) {
        report->lat_p50_us = percentile(meas, 0.50) * 1e-3;
        report->lat_p99_us = percentile(meas, 0.99) * 1e-3;
        report->lat_max_us = (double)*std::max_element(meas.begin(), meas.end()) * 1e-3;
        double sum = 0;
        for (uint64_t v : meas) sum += (double)v;
        report->lat_mean_us = sum / (double)meas.size() * 1e-3;
    }
    report->mean_batch = batches ? (double)taken_total / (double)batches : 0.0;
    report->busy_s = (double)busy_ns * 1e-9;
    report->max_size = max_size;
    report->pinned_bytes = pinned_bytes;
    report->submit_s = (double)submit_ns * 1e-9;
    report->flush_s = (double)flush_ns * 1e-9;
    report->retire_s = (double)retire_ns * 1e-9;
    if (latency_ns_out) std::memcpy(latency_ns_out, lat.data(), n * sizeof(uint64_t));
    return GC_OK;
}
