// gc_policy.cu -- when to combine pending work requests into one batch
// (Section 3.1 of Rengasamy & Vadhiyar, arXiv 2008.05712).
//
// The paper's adaptive rule: maxSize is the number of requests one combined
// launch runs at full occupancy (from the occupancy calculator); the runtime
// keeps a running maximum maxInterval of the intervals between request
// arrivals and polls the pending list periodically: with at least maxSize
// pending it combines maxSize of them; with fewer, it combines everything
// pending once the time since the last arrival exceeds 2 x maxInterval.
// The paper's static baseline (Section 4.3) combines whatever is pending
// after every 100 requests.  The greedy rule (no counterpart in the paper)
// is the work-conserving form for a caller that polls only when it has room
// for another batch on the device: combine everything pending at every
// poll (the caller's admission still bounds a batch by the staging budget),
// so under a load above what maxSize-request batches sustain the batches
// grow with the queue instead of the queue growing without end.  Host-side
// logic only (no device work).
#include <cmath>
#include <deque>

#include "gc_common.cuh"

struct gc_combiner {
    int policy;
    uint64_t max_size;
    uint64_t static_n;
    uint64_t window;
    bool have_arrival = false;
    uint64_t last_arrival = 0;
    uint64_t max_interval = 0;
    // windowed variant: the last `window` intervals as a decreasing deque of
    // (arrival number, interval), so the front is their maximum
    std::deque<std::pair<uint64_t, uint64_t>> recent;
    uint64_t n_gaps = 0;
    uint64_t since_combine = 0;      // arrivals since the last combine (static rule)
};

extern "C" {

int gc_combiner_create(int policy, uint64_t max_size, uint64_t static_n, uint64_t window,
                       gc_combiner_t **out)
{
    if (!out) return GC_ERR_ARG;
    *out = nullptr;
    if (policy < GC_COMBINE_ADAPTIVE || policy > GC_COMBINE_GREEDY) return GC_ERR_ARG;
    if ((policy == GC_COMBINE_ADAPTIVE || policy == GC_COMBINE_ADAPTIVE_WINDOW) &&
        max_size == 0)
        return GC_ERR_ARG;
    if (policy == GC_COMBINE_STATIC && static_n == 0) return GC_ERR_ARG;
    if (policy == GC_COMBINE_ADAPTIVE_WINDOW && window == 0) return GC_ERR_ARG;
    gc_combiner *c = new gc_combiner();
    c->policy = policy;
    c->max_size = max_size;
    c->static_n = static_n;
    c->window = window;
    *out = c;
    return GC_OK;
}

int gc_combiner_destroy(gc_combiner_t *c)
{
    if (!c) return GC_ERR_ARG;
    delete c;
    return GC_OK;
}

int gc_combiner_arrive(gc_combiner_t *c, uint64_t t_ns, uint64_t count)
{
    if (!c) return GC_ERR_ARG;
    for (uint64_t i = 0; i < count; ++i) {
        if (c->have_arrival) {
            const uint64_t gap = t_ns >= c->last_arrival ? t_ns - c->last_arrival : 0;
            if (c->policy == GC_COMBINE_ADAPTIVE_WINDOW) {
                // maximum of the last `window` intervals, amortised O(1)
                const uint64_t k = c->n_gaps++;
                while (!c->recent.empty() && c->recent.back().second <= gap)
                    c->recent.pop_back();
                c->recent.emplace_back(k, gap);
                while (c->recent.front().first + c->window <= k) c->recent.pop_front();
                c->max_interval = c->recent.front().second;
            } else if (gap > c->max_interval) {
                c->max_interval = gap;
            }
        }
        c->have_arrival = true;
        c->last_arrival = t_ns;
        c->since_combine += 1;
    }
    return GC_OK;
}

int gc_combiner_poll(gc_combiner_t *c, uint64_t t_ns, uint64_t queued, uint64_t *take_out)
{
    if (!c || !take_out) return GC_ERR_ARG;
    uint64_t take = 0;
    if (queued > 0) {
        switch (c->policy) {
        case GC_COMBINE_ADAPTIVE:
        case GC_COMBINE_ADAPTIVE_WINDOW: {
            if (queued >= c->max_size) {
                take = c->max_size;
            } else {
                const uint64_t idle = t_ns >= c->last_arrival ? t_ns - c->last_arrival : 0;
                if (idle > 2 * c->max_interval) take = queued;
            }
            break;
        }
        case GC_COMBINE_STATIC:
            if (c->since_combine >= c->static_n) take = queued;
            break;
        case GC_COMBINE_GREEDY:
            take = queued;
            break;
        default:   // GC_COMBINE_PER_TASK
            take = 1;
            break;
        }
    }
    if (take) c->since_combine = 0;
    *take_out = take;
    return GC_OK;
}

int gc_combiner_max_interval(gc_combiner_t *c, uint64_t *ns_out)
{
    if (!c || !ns_out) return GC_ERR_ARG;
    *ns_out = c->max_interval;
    return GC_OK;
}

uint64_t gc_combine_size_from_occupancy(double occupancy, uint32_t max_blocks_per_sm,
                                        uint32_t n_sm)
{
    if (!(occupancy > 0.0) || max_blocks_per_sm == 0 || n_sm == 0) return 0;
    return (uint64_t)std::llround(occupancy * (double)max_blocks_per_sm) * (uint64_t)n_sm;
}

}  // extern "C"
