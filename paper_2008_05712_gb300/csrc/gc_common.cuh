// gc_common.cuh -- internal declarations shared by the libgcharm translation
// units (not part of the public ABI; see include/gcharm.h for that).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>
#include <stddef.h>

#include <unordered_map>
#include <vector>

#include "gcharm.h"

#define GC_NONE 0xFFFFFFFFu
// ref_epoch[id]: GC_EPOCH_UNKNOWN until the id's value is first uploaded,
// 0 until first referenced, then the epoch of the last wave referencing it
#define GC_EPOCH_UNKNOWN 0xFFFFFFFFu

// Four doubles, 32-byte aligned (one per-id FP64 total).
struct __align__(32) gcd4 {
    double x, y, z, w;
};

// Device error-flag bits (pool->d_ctr[CTR_FLAGS]).
#define GC_FLAG_UNKNOWN_ID 1u     // a batch entry names an id never uploaded
#define GC_FLAG_ID_RANGE 2u       // an id >= id_capacity (device upload/build)
#define GC_FLAG_BAD_TASK 4u       // unknown kind, or LJ_SELF with sources
#define GC_FLAG_TIMEOUT 8u        // a device-side wait ran out of its limit

// Indices into the pool's device counter block (pool->d_ctr, uint64 each).
// The residency counters (CTR_UNIQUE .. end) are cleared at every wave.
enum {
    CTR_FLAGS = 0,      // error bits
    CTR_UPDATES,        // uploads that hit a resident slot
    CTR_UNIQUE,         // distinct ids in the current wave
    CTR_HITS,
    CTR_MISSES,
    CTR_FREE,
    CTR_HIST0,          // 8 reuse-histogram bins
    CTR_COUNT = CTR_HIST0 + 8
};

// Indices into a flush context's counter block (ctx.d_ctr).
enum {
    FC_QUEUE = 0,       // work-queue head of the persistent interaction kernel
    FC_INTER,           // pair interactions of the batch
    FC_NGRAV_WU,        // gravity work units of the batch
    FC_NLJ,             // LJ tasks of the batch
    FC_MAXLIST,         // longest list of the batch
    FC_RUNS,            // distinct ids among result rows
    FC_LJ_IN,           // LJ pairs inside the cutoff
    FC_PACK_WORK,       // list claims of the block-per-list pack kernels (4 counters)
    FC_COUNT = FC_PACK_WORK + 4
};
// Host-only words after the FC_COUNT counters of a context's pinned block:
// the batch sizes the preparation reads back (rows, gravity work units, LJ
// tasks; 4-byte values land in the low half of a zeroed word).
enum { FH_ROWS = FC_COUNT, FH_WU, FH_LJ, FH_COUNT };

// One task as the kernels see it (48 bytes).
struct TaskRec {
    uint64_t task_id;
    uint64_t tgt_off;   // first target entry (batch-global)
    uint64_t src_off;   // first source entry (batch-global)
    uint64_t row_off;   // first result row (batch-global)
    uint32_t kind;
    uint32_t nt, ns;
    int8_t shift[4];
};
static_assert(sizeof(TaskRec) == 48, "TaskRec layout");

// Growable device buffer.  Growing frees the old storage (contents lost).
struct DBuf {
    void *p = nullptr;
    size_t cap = 0;
    int reserve(size_t bytes);
    void release();
    template <class T> T *as() const { return static_cast<T *>(p); }
};

// Work unit of the gravity kernel: one task and a block of <= 16 targets.
struct GravWU {
    uint32_t task;
    uint32_t t0;     // first target (staged order)
    uint32_t tn;     // targets in the block
    uint32_t pad;
};

struct NBodyState {
    uint64_t n = 0, n_nodes = 0, n_buckets = 0, n_list = 0, max_list = 0;
    DBuf keys, keys2, ids, ids2, lcp, win, dmax, nnode, node_off;
    DBuf node_a, node_b, node_val, bucket, bbox, list_off, list_len, list, wnode;
    uint64_t n_walk_items = 0;       // (bucket, walk range) pairs of the last build
    DBuf bounds, cub_tmp, mono, hostcopy;
    // Morton order: seeded from the previous build's order (ids2) when it
    // holds a permutation of the same n particles
    int order_mode = 1;              // GC_ORDER_SEEDED
    uint64_t order_n = 0;            // particles of the permutation in ids2 (0: none)
    DBuf seed_tiles, seed_a, seed_m, seed_key;
    // build timing: events {start, order done, end}, folded into the sums
    // once the end event has completed
    cudaEvent_t ev[3] = {nullptr, nullptr, nullptr};
    bool ev_pending = false, pending_seeded = false;
    uint64_t builds = 0, seeded_builds = 0, timed_builds = 0, last_resorted = 0;
    double last_order_ms = 0, last_tree_ms = 0, order_ms_sum = 0, tree_ms_sum = 0;
};

struct MDState {
    uint64_t n = 0;
    int m = 0;
    int dim = 3;
    DBuf keys, keys2, ids, ids2, cell_start, cnt_t, cnt_s, cub_tmp, hostcopy;
};

// Blocks for n items at `threads` per block, at most max_blocks (grid-stride
// loops cover the rest).
static inline unsigned grid_for(uint64_t n, int threads, int max_blocks)
{
    uint64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (uint64_t)max_blocks) b = max_blocks;
    return (unsigned)b;
}

#define GRID_STRIDE(i, n)                                                       \
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (n); \
         i += (uint64_t)gridDim.x * blockDim.x)

// One wave of a flush: tasks [t0, t1), their target / source entries, and
// their gravity work units and LJ task slots.
struct WaveRange {
    uint64_t t0, t1, tg0, tg1, s0, s1, w0, w1, l0, l1;
};

// Everything one in-flight batch owns: its stream, its batch arrays, work
// buffers, counters and events.
struct FlushCtx {
    cudaStream_t s = nullptr;
    bool owns_stream = false;
    // side streams of the pack's size classes and their fork / join events
    cudaStream_t ps[3] = {nullptr, nullptr, nullptr};
    cudaEvent_t pev[4] = {nullptr, nullptr, nullptr, nullptr};
    unsigned long long *d_ctr = nullptr;   // [FC_COUNT]
    unsigned long long *h_ctr = nullptr;   // pinned copy
    DBuf tasks, tgt_ids, src_ids;          // the executed batch
    uint64_t n_tasks = 0, n_tgt = 0, n_src = 0, n_rows = 0, batch = 0;
    bool valid = false;
    DBuf tgt_perm, src_perm, stg_tgt, stg_src;
    DBuf wu, wu_cnt, wu_off, rowcnt, lj_list, res, row_id;
    DBuf lpt;                          // longest-first ordering scratch
    DBuf rid_sorted, row_sorted, rows_tmp, runs, tiles, merge_a, merge_b, cub_tmp;
    DBuf ent;                          // the current wave's entry slots
    cudaEvent_t ev_stage[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaEvent_t ev_done = nullptr, ev_packed = nullptr, ev_scattered = nullptr;
    bool timing_valid = false;
    bool timing_counted = false;   // stage times added to the pool's sums
    float multiwave_ms[3] = {0, 0, 0};
    uint64_t n_waves = 0;
    std::vector<WaveRange> waves;          // the waves of the batch
    uint64_t msrc = 0;                     // source offset in the merge scratch
    uint64_t max_list = 0;                 // longest target or source list
    bool md_struct = false;                // the batch is one MD build: rows reduced per cell
    int md_m = 0, md_dim = 3;
    bool unique_rows = false;              // every row id occurs once (one N-body build)
    std::vector<TaskRec> host_tasks;       // for gc_read_results
    std::unordered_map<uint64_t, uint64_t> task_index;
    bool host_tasks_valid = false;
};

struct gc_pool {
    gc_config cfg;
    cudaStream_t s = nullptr;         // issue stream = ctx[cur].s
    int device = 0;
    int num_sms = 0;
    int64_t rc2_grid = 0;       // cutoff^2 in (2^-21)^2 units
    int32_t md_edge_grid = 0;   // cell edge in 2^-21 units

    // chare table and data
    float4 *d_pool = nullptr;          // [pool_capacity]
    uint32_t *d_slot_of_id = nullptr;  // [id_capacity]
    uint32_t *d_id_of_slot = nullptr;  // [pool_capacity]
    uint64_t free_slots = 0;           // slots holding no id (kept on the host)
    uint64_t res_n = 0;                // entries of the chare-table step issued last
    bool res_few = false;              // it listed its distinct ids while marking
    uint32_t *d_last_use = nullptr;    // [pool_capacity]
    uint32_t *d_ref_epoch = nullptr;   // [id_capacity]
    uint32_t *d_ref_count = nullptr;   // [id_capacity]
    float4 *h_mirror = nullptr;        // pinned, mapped [id_capacity]
    float4 *d_mirror = nullptr;        // device alias of h_mirror
    gcd4 *d_totals = nullptr;       // [id_capacity]
    unsigned long long *d_ctr = nullptr;   // [CTR_COUNT]
    unsigned long long *h_ctr = nullptr;   // pinned copy

    // pending batch (device-resident), swapped into a flush context by gc_flush
    uint64_t nb_tasks = 0, nb_tgt = 0, nb_src = 0;
    DBuf tasks, tgt_ids, src_ids;
    uint64_t submitted_batches = 0;   // index of the pending batch
    bool md_pending = false;          // the pending batch began with an MD build
    uint64_t nb_pend_tasks = 0;       // tasks of an N-body build that began the pending batch
    bool totals_reset_pending = false;   // gc_reset_totals not yet applied on the device
    int md_pend_m = 0, md_pend_dim = 3;

    // two flush contexts: batch k runs on ctx[k % 2]; `cur` takes the next
    // flush, `last` holds the last flushed batch (-1: none yet)
    FlushCtx ctx[2];
    int cur = 0, last = -1;

    // residency work buffers (the chare-table step is serialised)
    DBuf uniq, miss, miss_sorted, freel, tiles, ekeys, ekeys2, evicted, cub_tmp;
    DBuf io_a, io_b;                  // host <-> device staging of uploads and reads
    // stream-ordered uploads and totals reads (gc_pool_upload_async,
    // gc_read_totals_async): own device buffers, and one copy stream per
    // direction, so that a step's input copies overlap the batch before it
    // and its totals copy the tree build after it; events order each copy
    // or kernel after the last use of the buffer it overwrites
    DBuf au_ids, au_vals, at_ids, at_out;
    cudaStream_t cs_in = nullptr, cs_out = nullptr;
    cudaEvent_t ev_au = nullptr;      // upload kernel has read au_*
    cudaEvent_t ev_au_in = nullptr;   // au_* copied in
    cudaEvent_t ev_at_in = nullptr;   // at_ids copied in
    cudaEvent_t ev_at_g = nullptr;    // gather has read at_ids and written at_out
    cudaEvent_t ev_at = nullptr;      // at_out copied out
    bool au_used = false, at_used = false;
    // host-array submissions: descriptors (and the ids of a small
    // submission) packed into a pinned host buffer, copied and turned into
    // task records on a stream of their own.  The copies wait only for the
    // last readers of the pending arrays (ev_pend_free, recorded by the flush
    // that handed them over) -- not for the batch in flight -- and the host
    // waits for the copies alone (ev_sub_copied); the pool's stream waits
    // for the task records (ev_sub_done)
    cudaStream_t cs_sub = nullptr;
    cudaEvent_t ev_pend_free = nullptr, ev_sub_copied = nullptr, ev_sub_done = nullptr;
    DBuf sub_desc;                    // device copy of the descriptors
    void *h_sub = nullptr;            // pinned host staging
    size_t h_sub_cap = 0;
    uint64_t n_evicted_last = 0;
    uint32_t epoch = 0;

    gc_stats_t stats;
    // interaction schedule (gc_set_tuning / gc_autotune)
    uint32_t wu_max_targets = 16;      // targets per gravity work unit: 8, 16 or 32
    uint32_t wu_schedule = GC_SCHED_FIFO;
    uint32_t wu_tile = 128;            // gravity tile shape: source pairs per staged tile
    uint32_t wu_kb = 8;                // and pairs per plain partial sum
    uint32_t wu_tpl = 1;               // and targets per lane
    uint64_t table_version = 0;        // bumped whenever a slot is assigned or freed
    // Ewald correction (GC_EWALD tasks): half of the reciprocal vectors
    // (hx, hy, hz, 2 exp(-pi^2 h^2 / (alpha L)^2) / h^2)
    float4 *d_ewald_h = nullptr;
    int n_ewald_h = 0;
    NBodyState nb;
    MDState md;
};

// ---- error helper ----------------------------------------------------------
#define GC_CUDA_TRY(expr)                                    \
    do {                                                     \
        cudaError_t _e = (expr);                             \
        if (_e != cudaSuccess) return GC_ERR_CUDA;           \
    } while (0)

#define GC_TRY(expr)                                         \
    do {                                                     \
        int _r = (expr);                                     \
        if (_r != GC_OK) return _r;                          \
    } while (0)

// ---- CUB-backed primitives (gc_sort.cu) -------------------------------------
int gc_sort_pairs_u64(DBuf &tmp, const uint64_t *kin, uint64_t *kout, const uint32_t *vin,
                      uint32_t *vout, uint64_t n, int end_bit, cudaStream_t s);
int gc_sort_pairs_u32(DBuf &tmp, const uint32_t *kin, uint32_t *kout, const uint32_t *vin,
                      uint32_t *vout, uint64_t n, int end_bit, cudaStream_t s);
int gc_sort_keys_u32(DBuf &tmp, const uint32_t *kin, uint32_t *kout, uint64_t n, int end_bit,
                     cudaStream_t s);
int gc_sort_keys_u64(DBuf &tmp, const uint64_t *kin, uint64_t *kout, uint64_t n,
                     cudaStream_t s);
int gc_exclusive_scan_u64(DBuf &tmp, const uint64_t *in, uint64_t *out, uint64_t n,
                          cudaStream_t s);
int gc_exclusive_scan_u32(DBuf &tmp, const uint32_t *in, uint32_t *out, uint64_t n,
                          cudaStream_t s);

// ---- residency (gc_residency.cu) -----------------------------------------------
// Runs the chare-table step for the entries tgt[0..nt) and src[0..ns): after
// it every referenced id is resident.  With `ent` (nt + ns words, may be
// null) it also records each entry's slot as found before any miss was
// placed (NONE for a miss).  Returns GC_OK, GC_ERR_UNKNOWN_ID or
// GC_ERR_POOL_FULL.
int gc_entry_slots(gc_pool *p, cudaStream_t s, const uint32_t *ids, uint64_t n, uint32_t *out);
int gc_residency(gc_pool *p, const uint32_t *tgt, uint64_t nt, const uint32_t *src,
                 uint64_t ns, uint32_t *ent);
// The same in two halves around a wait for the pool's stream (so that the
// wait can serve other read-backs too): the device steps and the counters'
// copy, then what follows from the counters.
int gc_residency_issue(gc_pool *p, const uint32_t *tgt, uint64_t nt, const uint32_t *src,
                       uint64_t ns, uint32_t *ent);
int gc_residency_finish(gc_pool *p);
int gc_launch_upload(gc_pool *p, const uint32_t *ids, const float4 *vals, uint64_t n,
                     int write_mirror);

// ---- pack / interaction / scatter (gc_kernels.cu) -----------------------------
int gc_prepare(gc_pool *p, FlushCtx &c, uint64_t info[5]);
// The same in two halves around a wait for the context's stream: the
// counting kernels and the sizes' copy into the context's pinned words,
// then the buffers and work lists sized from them.
int gc_prepare_issue(gc_pool *p, FlushCtx &c);
int gc_prepare_finish(gc_pool *p, FlushCtx &c, uint64_t info[5]);
int gc_scatter_replay(gc_pool *p, FlushCtx &c);
int init_ctx(FlushCtx &c, cudaStream_t given);
void free_ctx(FlushCtx &c);
int order_after_scatters(gc_pool *p);
// Clear the status bits `mask` of the pool's flag word, stream-ordered and
// atomically (kernels of another batch may be setting other bits meanwhile).
int gc_clear_flags(gc_pool *p, cudaStream_t s, unsigned long long mask);
// Apply a pending reset of the per-id totals on stream s (the caller orders
// s after every scatter already issued).
int gc_apply_totals_reset(gc_pool *p, cudaStream_t s);
int gc_read_wu_offsets(gc_pool *p, FlushCtx &c, std::vector<uint32_t> &wu_off,
                       std::vector<uint32_t> &lj_off);
// `ent` (may be null): the wave's entry slots (as gc_residency records
// them), the wave's ent_nt target entries first, then its source entries.
int gc_pack(gc_pool *p, FlushCtx &c, uint64_t t0, uint64_t t1, uint64_t tgt_base,
            uint64_t src_base, uint64_t msrc, const uint32_t *ent, uint64_t ent_nt);
int gc_interact_range(gc_pool *p, FlushCtx &c, uint64_t w0, uint64_t w1, uint64_t l0,
                      uint64_t l1, uint64_t tgt_base, uint64_t src_base, uint64_t task_base);
int gc_interact_one_task(gc_pool *p, FlushCtx &c, uint64_t w0, uint64_t w1, uint64_t l0,
                         uint64_t l1, uint64_t tgt_base, uint64_t src_base, uint64_t task_base);
int gc_scatter(gc_pool *p, FlushCtx &c);
// ---- MD batches (gc_md.cu) ----------------------------------------------------
uint64_t gc_md_tasks(int m, int dim);
int gc_md_reduce(gc_pool *p, FlushCtx &c);
int gc_make_task_recs(gc_pool *p, uint64_t n_tasks, const uint64_t *task_ids,
                      const uint32_t *kinds, const int8_t *shifts, const uint64_t *tgt_off,
                      const uint64_t *src_off, uint64_t tgt_base, uint64_t src_base,
                      uint64_t task_id_base, TaskRec *out, cudaStream_t s);

// ---- compaction helper (gc_residency.cu) ---------------------------------------
// Writes, in ascending order, every i in [0, n) with flags-kind predicate.
enum CompactKind {
    CK_REF_EPOCH = 0,   // i: ref_epoch[i] == epoch           (id space)
    CK_MISS,            // k < count: slot_of_id[uniq[k]] == NONE   (value uniq[k])
    CK_FREE,            // s: id_of_slot[s] == NONE           (slot space)
    CK_RUN_START        // i < count: i == 0 || key[i] != key[i-1]
};
int gc_compact(gc_pool *p, DBuf &tiles, cudaStream_t s, int kind, uint64_t n_bound,
               const uint64_t *count_dev, const uint32_t *arr, uint32_t *out,
               unsigned long long *count_out);

// ---- builders --------------------------------------------------------------------
// If ptr is host memory, copy bytes of it into buf (stream-ordered, then
// synchronised) and return the device copy; device pointers pass through.
const void *gc_device_view(gc_pool *p, const void *ptr, size_t bytes, DBuf &buf, int *rc);
int gc_reserve_batch(gc_pool *p, uint64_t add_tasks, uint64_t add_tgt, uint64_t add_src);
