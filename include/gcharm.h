/*
 * gcharm.h -- C ABI of libgcharm, a GB300 (sm_103a) engine for batches of
 * many small, irregular pair-interaction work requests, after the G-Charm
 * runtime strategies of Rengasamy & Vadhiyar (arXiv 2008.05712).
 *
 * Model (Section 2.2, Section 3.1, Section 3.2 of the paper):
 *   - Application objects create work requests ("tasks"), each naming the
 *     data items it reads by index (Section 2.2, Section 3.2: a workRequest
 *     carries the buffer indices of its data).
 *   - Pending tasks are combined into one batch and executed by one set of
 *     kernel launches instead of one launch per task (Section 3.1).
 *   - A chare table maps data ids to device-memory slots so that data
 *     already resident is reused and only missing data is transferred
 *     (Section 3.2); the data each task reads is then gathered in sorted
 *     slot order into contiguous staging so the interaction kernel reads it
 *     coalesced (Section 3.2, Fig. 1d).
 *
 * Two interaction kinds are provided, from the paper's two applications:
 *   GC_GRAVITY  (Section 4.1, ChaNGa buckets): for every target i of the
 *               task and every source j of its interaction list,
 *               a_i += m_j r_ij / (|r_ij|^2 + eps2)^(3/2),
 *               phi_i -= m_j / (|r_ij|^2 + eps2)^(1/2),  r_ij = x_j - x_i.
 *   GC_LJ_PAIR / GC_LJ_SELF (Section 4.2, interact() of a compute object
 *               on two patches, updating the forces of both): truncated
 *               Lennard-Jones forces between the atoms of cell A (targets)
 *               and cell B (sources, shifted by the task's cell offset);
 *               a self task uses the pairs i < j of cell A.
 *
 * Conventions for every function:
 *   - Return GC_OK (0) or a negative GC_ERR_* code; on any error the pool
 *     stays valid and the pending batch is unchanged unless stated.
 *   - Host pointers are caller-owned and only read (or written, for
 *     outputs) during the call.  "Device" pointers are CUDA device
 *     addresses on the pool's device; they are read in stream order on the
 *     pool's stream and must stay valid until the operation completes.
 *   - A pool is not thread-safe: one host thread at a time.
 *   - Data values are float4 records (x, y, z, w): for gravity w is the
 *     mass; for LJ atoms xyz is the atom's offset from its cell's origin (an
 *     exact multiple of 2^-21) and w is ignored.
 */
#ifndef GCHARM_H
#define GCHARM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Opaque pool handle (library-owned). */
typedef struct gc_pool gc_pool_t;

/* ---- status codes ------------------------------------------------------ */
#define GC_OK 0
#define GC_ERR_ARG (-1)         /* bad argument or configuration           */
#define GC_ERR_OOM (-2)         /* device or pinned host allocation failed */
#define GC_ERR_POOL_FULL (-3)   /* batch references more distinct ids than
                                   the pool can hold at once               */
#define GC_ERR_UNKNOWN_ID (-4)  /* a task references an id >= id_capacity or
                                   never uploaded; the batch is dropped    */
#define GC_ERR_BUDGET (-5)      /* one task alone exceeds the staging budget */
#define GC_ERR_NOT_READY (-6)   /* results requested before completion     */
#define GC_ERR_TIMEOUT (-7)     /* wait or device-side poll ran out        */
#define GC_ERR_CUDA (-8)        /* a CUDA runtime call failed              */
#define GC_ERR_STATE (-9)       /* call not valid in the pool's state      */
#define GC_ERR_TOO_LARGE (-10)  /* request exceeds a fixed size limit      */

/* ---- task kinds -------------------------------------------------------- */
#define GC_GRAVITY 0u
#define GC_LJ_PAIR 1u
#define GC_LJ_SELF 2u
#define GC_EWALD 3u     /* periodic-gravity correction: targets x sources, the
                           Ewald interaction minus the plain point-mass term
                           (needs gc_config.ewald_box > 0)                   */

/* ---- configuration (gc_pool_create) ------------------------------------ */
typedef struct {
    float eps2;                   /* gravity softening squared, > 0        */
    float lj_eps, lj_sigma;       /* LJ well depth and diameter, > 0       */
    float lj_rc2;                 /* LJ cutoff squared; rc2 * 2^42 must be
                                     an integer (cutoff decided exactly on
                                     the 2^-21 grid)                       */
    float md_edge;                /* MD cell edge, a multiple of 2^-21     */
    uint64_t id_capacity;         /* data ids must be < id_capacity        */
    uint64_t pool_capacity;       /* device slots (resident data items)   */
    uint64_t staging_budget_bytes;/* max staging bytes per flush wave; 0 =
                                     no limit                              */
    int deterministic;            /* 1: per-id totals summed in admission
                                     order (always on in this version)     */
    void *cuda_stream;            /* cudaStream_t the pool issues on; NULL =
                                     the legacy default stream             */
    float ewald_box;              /* periodic cube side L for GC_EWALD tasks;
                                     0 = no Ewald tasks.  Splitting alpha =
                                     2/L, real-space images |n_i| <= 2,
                                     reciprocal vectors 0 < |h|^2 <= 10    */
} gc_config;

/* ---- one task (gc_submit) ---------------------------------------------- */
typedef struct {
    uint64_t task_id;             /* caller's tag, returned with results   */
    uint32_t kind;                /* GC_GRAVITY | GC_LJ_PAIR | GC_LJ_SELF   */
    uint32_t n_targets, n_sources;
    const uint32_t *target_ids;   /* host, n_targets ids                   */
    const uint32_t *source_ids;   /* host, n_sources ids (LJ_SELF: none)   */
    int8_t shift[3];              /* LJ: cell offset of B from A, in cells  */
} gc_task;

/* ---- statistics -------------------------------------------------------- */
typedef struct {
    uint64_t flushes;             /* batches executed                       */
    uint64_t tasks;               /* tasks executed                         */
    uint64_t entries;             /* id references (targets + sources)      */
    uint64_t unique;              /* distinct ids referenced, summed/flush  */
    uint64_t hits;                /* distinct ids found resident            */
    uint64_t misses;              /* distinct ids fetched from host memory  */
    uint64_t updates;             /* uploads that overwrote a resident slot */
    uint64_t evictions;           /* resident ids evicted                   */
    uint64_t h2d_bytes;           /* bytes moved host -> device             */
    uint64_t interactions;        /* pair interactions evaluated            */
    uint64_t lj_pairs_in_cutoff;  /* LJ pairs inside the cutoff (last flush) */
    uint64_t last_unique, last_hits, last_misses, last_evictions;
    uint64_t last_staging_bytes;  /* staging bytes of the last flush        */
    uint64_t last_waves;          /* waves the last flush was split into    */
    uint64_t reuse_hist[8];       /* last flush: distinct ids referenced
                                     1, 2, 3-4, 5-8, 9-16, 17-32, 33-64,
                                     >64 times                             */
    uint64_t kernel_launches;     /* kernels of this library launched      */
    uint64_t primitive_calls;     /* device-wide sort/scan calls (CUB), each
                                     a few launches of its own              */
    double stage_ms_sum[5];       /* device time of every completed flush,
                                     summed per stage {residency, pack,
                                     interaction, scatter, total} (CUDA
                                     events on the flush's stream)          */
    uint64_t timed_batches;       /* flushes counted in stage_ms_sum        */
} gc_stats_t;

/* ---- pool lifetime and data -------------------------------------------- */

/* Create a pool (Section 2.2: the runtime keeps the data it has sent to the
 * GPU; Section 3.2: the chare table maps chare buffers to device slots):
 * device slots, the chare table (id -> slot), a pinned host mirror holding
 * the value of every id that is not resident (a slot's value is written
 * back to it when the id is evicted), and per-id FP64 totals.
 * *out receives the handle.  Errors: GC_ERR_ARG (zero capacities, eps2 <= 0, bad LJ values),
 * GC_ERR_OOM, GC_ERR_CUDA. */
int gc_pool_create(const gc_config *cfg, gc_pool_t **out);

/* Release everything the pool owns (no counterpart in the paper: resource
 * release).  Waits for its stream first. */
int gc_pool_destroy(gc_pool_t *pool);

/* Store values for ids (host arrays, n ids and 4n floats; copied before the
 * call returns) -- the chares' data regions (Section 3.2: data already on the
 * GPU is not sent again).  A resident id is overwritten in its slot (an update, not a
 * miss); a non-resident id is stored in the host mirror and fetched at the
 * next flush that references it.  Duplicate ids in one call: one of the
 * values wins.  Runs on the pool's stream, after the pack of every batch
 * already flushed.  Errors: GC_ERR_ARG (id >= id_capacity; nothing is
 * stored), GC_ERR_CUDA. */
int gc_pool_upload(gc_pool_t *pool, const uint32_t *ids, const float *xyzm,
                   uint64_t n);

/* As gc_pool_upload (Section 3.2: the chares' data regions on the GPU), in
 * stream order: returns once the copies are queued.
 * The host arrays must stay unchanged until the pool's stream has passed
 * this point (gc_join, then a wait on the joined stream).  The copies run
 * on a host-to-device stream of the pool's own and wait only for the
 * previous asynchronous upload to be applied, so with pinned host memory they
 * overlap the batches still running; the upload itself is applied in the
 * pool's stream order.  Ids are checked on the
 * device, as by gc_pool_upload_device: an id >= id_capacity is skipped and
 * makes the next flush fail with GC_ERR_UNKNOWN_ID.  Errors: GC_ERR_ARG
 * (null arrays), GC_ERR_OOM, GC_ERR_CUDA. */
int gc_pool_upload_async(gc_pool_t *pool, const uint32_t *ids, const float *xyzm,
                         uint64_t n);

/* As gc_pool_upload, with device arrays, in stream order (no host wait).
 * Ids are not checked on the host; an id >= id_capacity sets the pool's
 * device error flag and is skipped (reported by the next flush). */
int gc_pool_upload_device(gc_pool_t *pool, const uint32_t *ids_dev,
                          const float *xyzm_dev, uint64_t n);

/* ---- batching ---------------------------------------------------------- */

/* Append tasks to the pending batch (host descriptors; ids are copied): one
 * workRequest per task, added to the list of combinable requests (Section
 * 2.2's workGroupList; Section 3.1).
 * *batch_out (may be NULL) receives the index the next gc_flush will give
 * this batch.  Errors: GC_ERR_ARG (unknown kind, LJ_SELF with sources),
 * GC_ERR_BUDGET (one task's staging exceeds the budget), GC_ERR_OOM. */
int gc_submit(gc_pool_t *pool, const gc_task *tasks, uint64_t n,
              uint64_t *batch_out);

/* Append n_tasks workRequests (Sections 2.2, 3.1) given as CSR arrays: task t has targets
 * tgt_ids[tgt_off[t] .. tgt_off[t+1]) and sources src_ids[src_off[t] ..
 * src_off[t+1]), kind kinds[t], shift shifts[3t..3t+2] (may be NULL: all
 * zero), tag task_ids[t] (NULL: running task counter).  on_device = 0:
 * all arrays are host arrays.  on_device = 1: all arrays are device arrays
 * and n_tgt_total / n_src_total must equal tgt_off[n_tasks] /
 * src_off[n_tasks] (the offsets are not read on the host); they are read in
 * stream order on the pool's stream, so keep them unchanged until the next
 * gc_flush has returned.  Offsets must start at 0 and not decrease. */
int gc_submit_csr(gc_pool_t *pool, uint64_t n_tasks, const uint64_t *task_ids,
                  const uint32_t *kinds, const int8_t *shifts,
                  const uint64_t *tgt_off, const uint32_t *tgt_ids,
                  const uint64_t *src_off, const uint32_t *src_ids,
                  uint64_t n_tgt_total, uint64_t n_src_total, int on_device,
                  uint64_t *batch_out);

/* Run the pending batch as one combined execution (Section 2.2's
 * workRequestCombined; Section 3.1): residency (chare-table lookup, Section
 * 3.2; slot allocation in
 * ascending id order, eviction of the least recently used unreferenced ids
 * when the pool is full, fetch of misses from the host mirror), pack
 * (per list, entries in ascending (slot, list position) order gathered into
 * contiguous float4 staging), interaction (FP32 pair arithmetic with
 * compensated accumulation), and the FP64 per-id accumulation of totals.
 * Reads a few counters back to the host after the residency step; the rest
 * is queued on the pool's stream.  Errors: GC_ERR_UNKNOWN_ID (batch
 * dropped), GC_ERR_POOL_FULL (batch dropped, pool unchanged),
 * GC_ERR_CUDA.  Flushing an empty batch is a no-op. */
int gc_flush(gc_pool_t *pool);

/* Wait until batch `batch` (as returned by the submit calls) has completed,
 * for at most timeout_ns (0 = forever) -- the runtime's monitoring of kernel
 * status before it notifies the chares (Section 2.2).  GC_ERR_TIMEOUT if it
 * has not. */
int gc_wait(gc_pool_t *pool, uint64_t batch, uint64_t timeout_ns);

/* Non-blocking completion check of batch `batch` (Section 2.2: periodic
 * monitoring of the kernels' status): *done_out = 1 once it has completed (0
 * while it runs or has not been flushed). */
int gc_batch_done(gc_pool_t *pool, uint64_t batch, int *done_out);

/* (No counterpart in the paper: stream interoperation.)  Make `stream` (a
 * cudaStream_t; NULL = the legacy default stream) wait for
 * all work the pool has issued so far: every batch in flight and anything
 * queued on the pool's streams.  No host wait. */
int gc_join(gc_pool_t *pool, void *stream);

/* Batches run alternately on two flush contexts, each with its own stream:
 * batch k+1's chare-table step and pack overlap batch k's interaction on the
 * device.  Results of batch k stay readable until batch k+2 is flushed. */

/* ---- results ----------------------------------------------------------- */

/* Results of a combined execution go back to the chares that issued the
 * work requests (Section 2.2).  Number of result rows of the last completed batch: one per target, plus
 * one per source for GC_LJ_PAIR tasks (targets first), in admission order. */
int gc_result_rows(gc_pool_t *pool, uint64_t *rows_out);

/* Copy the per-row results of the last batch, 8 floats per row: the
 * compensated partial (s0..s3, c0..c3) whose value is s - c; for gravity
 * (ax, ay, az, phi), for LJ (fx, fy, fz, U/2).  first_row / n_rows select a
 * range.  Errors: GC_ERR_ARG (range outside the batch). */
int gc_read_batch_results(gc_pool_t *pool, uint64_t first_row, uint64_t n_rows,
                          float *out);

/* The FP64 values of the same rows: 4 doubles per row, value = (double)s -
 * (double)c per component (the compensated partial of Section 2.2's result
 * of one work request, read as the number it stands for), computed on the
 * device and copied to values4 (host, caller-owned).  Waits for the batch.
 * Errors: GC_ERR_ARG (range outside the batch), GC_ERR_CUDA. */
int gc_read_batch_values(gc_pool_t *pool, uint64_t first_row, uint64_t n_rows,
                         double *values4);

/* The same conversion for rows already in host memory (rows read through
 * gc_read_results, gc_graph_results, gc_serve or written by
 * gc_gravity_noalloc): values4[4i + k] = (double)rows[8i + k] -
 * (double)rows[8i + 4 + k].  Host pointers, caller-owned.  Errors:
 * GC_ERR_ARG (null pointer with n_rows > 0). */
int gc_row_values(const float *rows, uint64_t n_rows, double *values4);

/* As gc_read_batch_results, for batch `batch` (one of the two most recently
 * flushed batches).  Waits for that batch.  Errors: GC_ERR_ARG (batch no
 * longer held, range outside the batch). */
int gc_read_batch_rows(gc_pool_t *pool, uint64_t batch, uint64_t first_row, uint64_t n_rows,
                       float *out);

/* Copy the result rows of the tasks with the given tags (each from the last
 * batch), task after task, 8 floats per row.  Errors: GC_ERR_ARG (tag not in
 * the last batch). */
int gc_read_results(gc_pool_t *pool, const uint64_t *task_ids, uint64_t n,
                    float *partial_sum_comp);

/* Per-id FP64 totals accumulated by every batch since the last reset:
 * 4 doubles per id (sum over the id's result rows of s - c) -- a particle's
 * acceleration from all its buckets' work requests (Section 4.1), an atom's
 * force from every cell-pair task that updates both patches (Section 4.2). */
int gc_read_totals(gc_pool_t *pool, const uint32_t *ids, uint64_t n,
                   double *acc4);

/* As gc_read_totals (Section 2.2: results returned to the chares), in stream
 * order: the totals as of every batch flushed
 * so far are copied to acc4 once the pool's stream passes this point
 * (gc_join, then a wait on the joined stream); ids and acc4 must stay valid
 * until then.  The totals are gathered in the pool's stream order; the copy
 * to acc4 runs on a device-to-host stream of the pool's own, so with pinned
 * host memory it overlaps the work queued after it (gc_join waits for it).
 * Errors: GC_ERR_ARG, GC_ERR_OOM, GC_ERR_CUDA. */
int gc_read_totals_async(gc_pool_t *pool, const uint32_t *ids, uint64_t n, double *acc4);

/* Device address of the totals array (double4 per id, id_capacity rows). */
int gc_totals_device(gc_pool_t *pool, const double **totals_dev);

/* (No counterpart in the paper.)  Zero all per-id totals.  Takes effect before the next batch's scatter
 * (and before any read of the totals, graph replay or kick-drift), so work
 * issued in between -- uploads, task builds -- does not wait for the batches
 * still running. */
int gc_reset_totals(gc_pool_t *pool);

/* Counters since creation plus details of the last flush: among them the
 * data-reuse figures of Section 3.2 (distinct ids, hits, misses, reuse
 * histogram). */
int gc_stats(gc_pool_t *pool, gc_stats_t *out);

/* Human-readable text for a status code (static string). */
const char *gc_strerror(int status);

/* ---- introspection of the last batch (integer work, for checking) ----- */

/* Slot of every entry of the last batch: n_tgt target entries then n_src
 * source entries, in admission order. */
int gc_read_entry_slots(gc_pool_t *pool, uint32_t *tgt_slots, uint32_t *src_slots);

/* Pack permutation of the last batch: for each list, perm[k] = list
 * position of the k-th staged entry (ascending (slot, position)). */
int gc_read_pack_perm(gc_pool_t *pool, uint32_t *tgt_perm, uint32_t *src_perm);

/* Sizes of the last batch. */
int gc_batch_sizes(gc_pool_t *pool, uint64_t *n_tasks, uint64_t *n_tgt,
                   uint64_t *n_src);

/* Copy the chare table: slot_of_id (id_capacity), id_of_slot and last_use
 * (pool_capacity each); NONE = 0xFFFFFFFF.  Any pointer may be NULL. */
int gc_read_residency(gc_pool_t *pool, uint32_t *slot_of_id, uint32_t *id_of_slot,
                      uint32_t *last_use);

/* Ids evicted by the last flush, in the order they were chosen. */
int gc_read_evicted(gc_pool_t *pool, uint32_t *ids, uint64_t cap, uint64_t *n_out);

/* ---- task builders on the device --------------------------------------- */

/* N-body tasks (Section 4.1): build the Barnes-Hut octree of the n
 * particles xyzm (4 floats per particle, a device or a host pointer -- host
 * data is first copied to the device; particle p has data id p) and append one GC_GRAVITY task per bucket to the pending batch:
 * targets = the bucket's particles in Morton order, sources = its
 * interaction list.  Tree: 21-bit grid per axis over the bounding cube
 * (power-of-two edge), Morton keys with x in bit 0, stable sort by key;
 * cells with more than bucket_max particles split into their non-empty
 * octants (octant order), a finest-level leaf with more is cut into chunks
 * of bucket_max; nodes numbered in depth-first preorder, node k has data id
 * n + k and value (centre of mass, mass), uploaded to the pool by this
 * call.  Walk: nodes containing the bucket are opened; any other node is
 * accepted iff theta_den^2 s^2 < theta_num^2 d^2 (s node edge, d distance
 * from the node centre to the bucket's box, integer doubled grid units);
 * opened leaves contribute their particles.  theta_num, theta_den in
 * [0, 255], theta_den >= 1.  Requires id_capacity >= n + node count.
 * task_id of bucket b = task_id_base + b.  info_out (may be NULL) receives
 * {n_nodes, n_buckets, list entries, particles sorted afresh}: n after a
 * full sort, the movers after a seeded one (gc_nbody_set_order).  Errors:
 * GC_ERR_ARG, GC_ERR_POOL_FULL (ids would exceed id_capacity), GC_ERR_OOM.
 *
 * Morton order.  The tree is rebuilt at every step of an integration
 * (Section 4.1), and a step moves the particles little.  When the previous
 * build on this pool had the same n, the build (GC_ORDER_SEEDED, the
 * default) computes the new keys in the previous sorted order, keeps a
 * sorted subsequence of it in place, sorts only the other particles (the
 * movers, gathered in id order) and merges the two.  The order, and so
 * every output, is the same as the full stable sort's, for any positions;
 * only the cost depends on how far the particles moved. */
int gc_build_nbody_tasks(gc_pool_t *pool, const float *xyzm_dev, uint64_t n,
                         int bucket_max, int theta_num, int theta_den,
                         uint64_t task_id_base, uint64_t info_out[4]);

/* Morton order of the next N-body builds (Section 4.1: the tree is rebuilt
 * every step): GC_ORDER_FULL sorts every build's
 * keys from scratch; GC_ORDER_SEEDED (default) starts from the previous
 * build's order when it had the same n.  Both give identical trees.
 * Errors: GC_ERR_ARG (unknown mode). */
#define GC_ORDER_FULL 0
#define GC_ORDER_SEEDED 1
int gc_nbody_set_order(gc_pool_t *pool, int mode);

/* N-body build statistics.  Times are CUDA-event intervals on the pool's
 * stream and include the host's waits inside a build (the node, bucket and
 * list counts are read back mid-build). */
typedef struct {
    uint64_t builds;          /* N-body builds completed                    */
    uint64_t seeded_builds;   /* of which started from the previous order   */
    uint64_t last_resorted;   /* particles the last build sorted afresh     */
    uint64_t timed_builds;    /* builds counted in the time sums            */
    double last_order_ms;     /* last build: bounding box to sorted order   */
    double last_tree_ms;      /* last build: whole build, tasks appended    */
    double order_ms_sum;      /* sums over timed builds                     */
    double tree_ms_sum;
} gc_nbody_stats_t;

/* Statistics of this pool's N-body builds (Section 4.1's per-step tree
 * build; waits for the last build's end event).  Errors: GC_ERR_ARG,
 * GC_ERR_CUDA. */
int gc_nbody_stats(gc_pool_t *pool, gc_nbody_stats_t *out);

/* As gc_build_nbody_tasks, with the positions of particles 0..n-1 taken
 * from the pool itself: the values most recently uploaded for ids 0..n-1
 * (gc_pool_upload, gc_pool_upload_device, gc_nbody_kick_drift), read on the
 * device from their slots (or, for an id not resident, from the host
 * mirror), so a caller that has just uploaded a step's positions does not
 * copy them to the device a second time.  Every id 0..n-1 must have been
 * uploaded.  Stream-ordered after those uploads.  Errors as
 * gc_build_nbody_tasks. */
int gc_build_nbody_tasks_resident(gc_pool_t *pool, uint64_t n, int bucket_max, int theta_num,
                                  int theta_den, uint64_t task_id_base, uint64_t info_out[4]);

/* One time step around the force computation (Section 4.1): for particles
 * i = 0..n-1, leapfrog kick then drift,
 *   v' = fl32(v + a dt),  x' = fl32(x + v' dt)   (FP64 arithmetic),
 * with a = acc_dev[4i .. 4i+2] (device FP64, 32-byte aligned; e.g. the
 * pool's per-id totals, gc_totals_device, after the step's flush), state
 * xyzm_dev (x, y, z, m) and vel_dev (vx, vy, vz, unused), device float4
 * arrays updated in place; the new positions are then written into the pool
 * for ids 0..n-1 (in place where resident).  Stream-ordered after every
 * batch in flight; no host wait.  Errors: GC_ERR_ARG (null or misaligned
 * pointers, n > id_capacity), GC_ERR_CUDA. */
int gc_nbody_kick_drift(gc_pool_t *pool, const double *acc_dev, float *xyzm_dev, float *vel_dev,
                        uint64_t n, double dt);

/* Copy the last N-body tree: sorted ids (n) and keys (n); per node (nn):
 * level, cell[3], first, count, leaf, subtree size; per bucket (nb): first,
 * count, leaf node; and the list CSR (nb+1 offsets, entries).  Any pointer
 * may be NULL. */
int gc_read_nbody_tree(gc_pool_t *pool, uint32_t *sorted_ids, uint64_t *sorted_keys,
                       uint8_t *level, uint32_t *cell3, uint32_t *first,
                       uint32_t *count, uint8_t *leaf, uint32_t *size,
                       float *node_xyzm, uint32_t *bucket_first,
                       uint32_t *bucket_count, uint32_t *bucket_node,
                       uint64_t *list_off, uint32_t *list_ids);

/* MD tasks (Section 4.2): group the n atoms by cell (cell_dev: linear cell
 * index x + m (y + m z) per atom, a device or a host pointer) into an m^3 periodic grid, atoms
 * of a cell in ascending atom id (atom a has data id a), and append, for
 * every cell in ascending index, its GC_LJ_SELF task and one GC_LJ_PAIR
 * task per neighbour offset (dx, dy, dz) lexicographically above (0,0,0)
 * (13 offsets), cell B = A + offset wrapped, shift = offset.  Requires
 * m >= 3.  task_id of task t = task_id_base + t.  info_out (may be NULL)
 * receives {tasks, target entries, source entries, max atoms in a cell}. */
int gc_build_md_tasks(gc_pool_t *pool, const uint32_t *cell_dev, uint64_t n, int m,
                      uint64_t task_id_base, uint64_t info_out[4]);

/* The planar case of gc_build_md_tasks (the paper's MD is two-dimensional,
 * Section 4.2): cell_dev[i] = cx + m*cy on a periodic m x m grid (atoms'
 * z offsets 0), m >= 3; per cell in ascending index the self task, then one
 * task per neighbour offset (dx, dy) in {(0,1), (1,-1), (1,0), (1,1)}; the
 * same results and errors as gc_build_md_tasks. */
int gc_build_md_tasks_2d(gc_pool_t *pool, const uint32_t *cell_dev, uint64_t n, int m,
                         uint64_t task_id_base, uint64_t info_out[4]);

/* Copy the last MD cell grouping: cell_start (m^3 + 1, or m^2 + 1 for the
 * planar case), cell_atoms (n). */
int gc_read_md_cells(gc_pool_t *pool, uint32_t *cell_start, uint32_t *cell_atoms);

/* ---- single-task launches (the one-launch-per-task baseline) ----------- */

/* Execute the pending batch like gc_flush, but launch the interaction
 * kernel once per task (same kernel body, one task per launch), as a
 * runtime without kernel combining would (Section 3.1).  Same results. */
int gc_flush_per_task(gc_pool_t *pool);

/* ---- timing of the last flush ------------------------------------------ */

/* Device time in milliseconds of each stage of the last flush, measured
 * with CUDA events on the pool's stream: {residency, pack, interaction,
 * scatter, total}.  Valid after gc_wait. */
int gc_last_timings(gc_pool_t *pool, float ms_out[5]);

/* ---- combining policy (Section 3.1, Section 4.3) ------------------------- */

#define GC_COMBINE_ADAPTIVE 0        /* paper's rule: maxSize, 2 x running-max interval */
#define GC_COMBINE_ADAPTIVE_WINDOW 1 /* same, max over the last `window` intervals      */
#define GC_COMBINE_STATIC 2          /* paper's baseline: all pending every static_n
                                        arrivals (100 in Section 4.3)                    */
#define GC_COMBINE_PER_TASK 3        /* no combining: one task per batch                */
#define GC_COMBINE_GREEDY 4          /* every poll: all pending (no counterpart in the
                                        paper; work-conserving form for a caller that
                                        polls when the device has room for another
                                        batch; batches grow with the queue)              */

typedef struct gc_combiner gc_combiner_t;

/* Decide when pending work requests are combined into a batch (Section
 * 3.1): maxSize = requests one combined launch runs at full occupancy;
 * maxInterval = running maximum of the intervals between arrivals; at each
 * poll, with >= maxSize pending combine maxSize, otherwise combine all
 * pending once the time since the last arrival exceeds 2 x maxInterval.
 * GC_COMBINE_STATIC combines all pending after every static_n arrivals
 * (the paper's static strategy, Section 4.3).  GC_COMBINE_GREEDY combines
 * everything pending at every poll.  Host-side, no device work.
 * Errors: GC_ERR_ARG (unknown policy, max_size 0 for the adaptive rules,
 * static_n 0 for the static rule, window 0 for the windowed rule). */
int gc_combiner_create(int policy, uint64_t max_size, uint64_t static_n, uint64_t window,
                       gc_combiner_t **out);
int gc_combiner_destroy(gc_combiner_t *c);

/* Record `count` requests arriving at time t_ns (monotonic nanoseconds). */
int gc_combiner_arrive(gc_combiner_t *c, uint64_t t_ns, uint64_t count);

/* At time t_ns with `queued` requests pending: *take_out = how many to
 * combine now (0 = keep waiting), oldest first. */
int gc_combiner_poll(gc_combiner_t *c, uint64_t t_ns, uint64_t queued, uint64_t *take_out);

/* Current maxInterval in nanoseconds. */
int gc_combiner_max_interval(gc_combiner_t *c, uint64_t *ns_out);

/* maxSize from an occupancy figure (Section 4.3): round(occupancy x
 * max_blocks_per_sm) x n_sm -- one work request per resident block. */
uint64_t gc_combine_size_from_occupancy(double occupancy, uint32_t max_blocks_per_sm,
                                        uint32_t n_sm);

/* maxSize of this engine on this GPU: work units (one per warp) the gravity
 * kernel keeps resident at once, from cudaOccupancyMaxActiveBlocksPerMultiprocessor
 * x warps per block x SMs. */
int gc_max_combine_size(gc_pool_t *pool, uint64_t *out);

/* ---- serving loop (Section 3.1: requests combined as they arrive) -------- */

typedef struct {
    int policy;               /* GC_COMBINE_*                                  */
    uint64_t max_size;        /* maxSize in requests; 0 = gc_max_combine_size  */
    uint64_t static_n;        /* GC_COMBINE_STATIC: arrivals per combine       */
    uint64_t window;          /* GC_COMBINE_ADAPTIVE_WINDOW: intervals kept    */
    uint32_t max_in_flight;   /* batches on the device at once: 1 or 2         */
    uint32_t keep_pageable;   /* 0: page-lock tgt_ids and src_ids for the call
                                 (cudaHostRegister) unless they already are;
                                 1: copy them from pageable memory as given   */
    uint64_t poll_ns;         /* longest idle sleep while nothing is queued    */
    uint64_t timeout_ns;      /* a batch not complete after this long fails the
                                 call with GC_ERR_TIMEOUT; 0 = 60 s           */
    uint64_t task_set;        /* tasks in the CSR arrays; arrival k is task
                                 k mod task_set (0 = n: arrival k is task k)  */
    uint64_t warmup_ns;       /* arrivals scheduled before this are served but
                                 left out of the latency statistics           */
    uint64_t drain_ns;        /* no batch is started later than this after the
                                 last scheduled arrival; tasks still queued
                                 then are counted as unserved (0 = no limit)  */
} gc_serve_config;

typedef struct {
    uint64_t tasks, batches;
    uint64_t interactions;    /* pair interactions evaluated by the call       */
    uint64_t max_size;        /* maxSize used                                  */
    double wall_s;            /* first scheduled arrival .. last completion    */
    double interactions_per_s;
    double lat_mean_us, lat_p50_us, lat_p99_us, lat_max_us;
    double mean_batch;        /* tasks per batch                               */
    double busy_s;            /* time with requests queued and no free batch
                                 slot (both flush contexts busy)              */
    uint64_t measured;        /* tasks in the latency statistics               */
    uint64_t unserved;        /* arrivals not served within the drain limit    */
    uint64_t pinned_bytes;    /* bytes of tgt_ids and src_ids page-locked for
                                 the call (already, or registered by it)      */
    double submit_s;          /* host time in gc_submit_csr                    */
    double flush_s;           /* host time in gc_flush                         */
    double retire_s;          /* host time retiring completed batches          */
} gc_serve_report;

/* Replay an open-loop arrival schedule in real time on this thread: task t
 * (CSR arrays as in gc_submit_csr, host memory, offsets starting at 0)
 * becomes pending at arrival_ns[t] nanoseconds after the call starts
 * (non-decreasing).  The loop tells the combiner of each arrival, retires
 * completed batches without blocking, and, while fewer than max_in_flight
 * batches run, asks the combiner how many pending tasks to combine, admits
 * the oldest of them that fit the pool's staging budget (at least one) and
 * flushes them: a batch's chare-table step and pack then overlap the
 * interaction of the batch before it.  The static rule drains what is left
 * once the schedule has ended.  Latency of a task = completion observed by
 * the loop - its scheduled arrival (CLOCK_MONOTONIC), so queueing behind a
 * busy device is counted.  latency_ns_out (n values; UINT64_MAX for an
 * unserved arrival) and results_out (8 floats per result row, rows of task
 * after task as gc_read_batch_results gives them; only with task_set = 0 or
 * n) may be NULL.  With task_set = m < n the m tasks are replayed cyclically
 * (a batch of consecutive arrivals is then at most a few contiguous runs of
 * the task arrays), so a long schedule needs no more than one task set.  An
 * offered load the engine cannot sustain leaves a queue behind: drain_ns
 * bounds the time spent after the schedule, and what is still queued then
 * is reported as unserved instead of delaying the call without end.  Unless
 * keep_pageable is set, tgt_ids and src_ids are page-locked for the
 * duration of the call (cudaHostRegister) unless they already are, so that
 * the per-batch copies run as direct DMA.  The pool must have no pending tasks; per-id
 * totals accumulate as for any flush.  Errors: GC_ERR_ARG (bad pointers,
 * decreasing arrivals, max_in_flight not 1 or 2), GC_ERR_STATE (pending
 * tasks), GC_ERR_TIMEOUT, and any error of gc_submit_csr / gc_flush. */
int gc_serve(gc_pool_t *pool, uint64_t n, const uint64_t *arrival_ns, const uint32_t *kinds,
             const int8_t *shifts, const uint64_t *tgt_off, const uint32_t *tgt_ids,
             const uint64_t *src_off, const uint32_t *src_ids, const gc_serve_config *cfg,
             uint64_t *latency_ns_out, float *results_out, gc_serve_report *report);

/* ---- a combined batch as a replayable CUDA graph -------------------------- */

typedef struct gc_graph gc_graph_t;

/* Capture the pending batch as a replayable step (the combined launch of
 * Section 3.1 kept as a CUDA graph).  Runs it once as gc_flush does, which
 * settles the chare table and every size, then records in a CUDA graph the
 * device work of one more execution on buffers the graph owns: last-use
 * update of the batch's distinct ids, per wave the pack and interaction
 * kernels, and the per-id FP64 accumulation in the order the first run
 * established.  The rows of the first run are readable through
 * gc_graph_results (not through the pool's result calls).  *out receives the
 * handle.  Errors: GC_ERR_STATE (no pending task), GC_ERR_POOL_FULL (the
 * batch's ids do not all fit the pool at once), any gc_flush error,
 * GC_ERR_CUDA. */
int gc_graph_capture(gc_pool_t *pool, gc_graph_t **out);

/* Replay the captured step, after the pool's batches in flight and before
 * any later one: same tasks, current pool values (ids re-uploaded in place
 * are used), new rows in the graph's buffers, per-id totals accumulated.
 * Asynchronous.  Errors: GC_ERR_STATE (a slot was assigned or freed since
 * the capture: capture again), GC_ERR_CUDA. */
int gc_graph_launch(gc_graph_t *g);

/* Wait for the last replay; GC_ERR_TIMEOUT if a device wait ran out. */
int gc_graph_wait(gc_graph_t *g);

/* Result rows of the graph's batch (8 floats per row, as
 * gc_read_batch_results) after the last run or replay. */
int gc_graph_rows(gc_graph_t *g, uint64_t *rows_out);
int gc_graph_results(gc_graph_t *g, uint64_t first_row, uint64_t n_rows, float *out);

/* Release the graph and its buffers (waits for its last replay). */
int gc_graph_destroy(gc_graph_t *g);

/* ---- interaction schedule and its autotuner ------------------------------ */
/* How the combined kernel of a batch (Section 3.1: one launch for many work
 * requests) hands its work to warps and stages its sources; the paper fixes
 * one thread block per work request, so these choices have no counterpart
 * there beyond that design. */

#define GC_SCHED_FIFO 0u   /* work units handed out in admission order          */
#define GC_SCHED_LPT 1u    /* longest first (targets x sources, descending;
                              admission order among equals)                    */

typedef struct {
    uint32_t wu_max_targets;  /* targets per gravity work unit (one warp): 8, 16
                                 or 32; a task of nT targets becomes
                                 ceil(nT / wu_max_targets) units of near-equal
                                 size, each run by T targets x 32/T source lanes */
    uint32_t schedule;        /* GC_SCHED_FIFO | GC_SCHED_LPT                  */
    uint32_t tile_pairs;      /* source pairs per tile staged in shared memory
                                 by a bulk copy: 64, 128 or 256 (32 B each;
                                 a block holds 16 tiles, so the size sets
                                 the resident blocks per SM)                   */
    uint32_t comp_block;      /* source pairs summed in plain FP32 before each
                                 compensated add: 8, 16 or 32                  */
    uint32_t targets_per_lane; /* targets each lane accumulates, sharing every
                                 source pair it reads: 1 or 2 (a unit of T
                                 targets then runs ceil(T / 2) target lanes x
                                 32 / ceil(T / 2) source lanes)              */
} gc_tuning;

/* Set / read the interaction schedule and tile shape used by later flushes
 * (default 16, FIFO, 128, 8, 1).  The results change only by FP32 summation
 * order (within the per-result tolerance).  Errors: GC_ERR_ARG (other
 * values). */
int gc_set_tuning(gc_pool_t *pool, const gc_tuning *t);
int gc_get_tuning(gc_pool_t *pool, gc_tuning *t);

/* Autotuner: re-run the interaction stage of the last flushed batch (one
 * wave, gravity tasks) under every schedule and tile shape, work-unit size
 * {8, 16, 32} x {FIFO, LPT} x tile pairs {64, 128, 256} x compensation block
 * {8, 16, 32} x targets per lane {1, 2}, timing each with CUDA events (best
 * of `reps`), and keep the fastest for later flushes -- a two-targets-per-
 * lane shape only when more than 3 % faster than the fastest one-target
 * shape, since it holds fewer warps per SM (a smaller gc_max_combine_size,
 * slower small batches).  ms_out (may be NULL)
 * receives the GC_TUNE_COUNT times, entry (((w * 2 + s) * 3 + t) * 3 + k) *
 * 2 + l - 1 for the w-th work-unit size, schedule s, t-th tile size, k-th
 * block and l targets per lane; *best_out (may be NULL) the choice.  The batch's result rows are rewritten by the re-runs
 * (same values up to summation order); per-id totals are not touched.
 * Errors: GC_ERR_NOT_READY (no batch), GC_ERR_STATE (the batch ran in more
 * than one wave, or has no gravity task), GC_ERR_CUDA. */
#define GC_TUNE_COUNT 108
int gc_autotune(gc_pool_t *pool, int reps, gc_tuning *best_out, float ms_out[GC_TUNE_COUNT]);

/* ---- reuse ablation (Section 3.2, Fig. 3) --------------------------------- */

/* Ways of feeding a batch's sources to the interaction, measured on the last
 * flushed batch (one wave, gravity tasks only), best of `reps`:
 *   out[0] interaction kernel on the packed staging (this engine), ms
 *   out[1] interaction reading every source from the pool through its slot,
 *          in list order (reuse without coalescing: the address buffer), ms
 *   out[2] the same with each list's slots sorted (Fig. 1d without the
 *          gather), ms
 *   out[3] redundant transfer, host side: every list's sources gathered on
 *          the host from the authoritative copy into contiguous staging, ms
 *   out[4] its host-to-device copy (pinned), ms
 *   out[5] bytes of that copy
 *   out[6] bytes the batch fetched with reuse (its misses x 16)
 * The batch's result rows are rewritten by the re-runs (same values up to
 * summation order).  Errors: GC_ERR_NOT_READY, GC_ERR_STATE (several waves,
 * LJ tasks), GC_ERR_OOM, GC_ERR_CUDA. */
int gc_reuse_ablation(gc_pool_t *pool, int reps, double out[7]);

/* ---- measurement ---------------------------------------------------------- */

/* FP32 throughput of the current device, measured: independent paired-FP32
 * FMA chains (2 FMAs = 4 flops per instruction) on every lane of every SM,
 * best of three timed launches (CUDA events).  *tflops_out = TFLOP/s,
 * *ms_out (may be NULL) = the best launch time.  The denominator of the
 * interaction kernel's roofline; no counterpart in the paper.  Allocates a
 * small buffer.  Errors: GC_ERR_ARG, GC_ERR_CUDA. */
int gc_fp32_peak(double *tflops_out, double *ms_out);

/* ---- failure detection ------------------------------------------------------ */

/* Exercise the expiry path of the bounded barrier waits that the interaction
 * kernels use for their bulk copies: one device thread waits, `polls` polls
 * long (1 .. 2^24), on a shared-memory barrier that nothing arrives at, and
 * on expiry sets the pool's timeout status -- the status a stalled copy
 * would set -- instead of spinning on or trapping.  Enqueued on the pool's
 * issue stream; the next gc_wait returns GC_ERR_TIMEOUT and clears the
 * status, and the pool stays usable.  Diagnostics; no counterpart in the
 * paper.  Errors: GC_ERR_ARG, GC_ERR_CUDA. */
int gc_check_wait_expiry(gc_pool_t *pool, uint32_t polls);

/* ---- evaluation without allocation -------------------------------------- */

/* Limits of gc_gravity_noalloc (its scratch is a fixed array). */
#define GC_NOALLOC_MAX_TASKS 65536u
#define GC_NOALLOC_MAX_TARGETS 262144u

/* Softened gravity (the GC_GRAVITY terms) for n_tasks tasks whose values are
 * already in device memory, without allocating anything: no cudaMalloc, no
 * cudaFree, no allocating library call.  The paper has no counterpart; this
 * is for callers that cannot allocate when they need the result -- code
 * inside a framework whose caching allocator already holds the device
 * memory budget (a cudaMalloc beside it can fail or fragment that budget),
 * latency-critical threads that must not take the device-wide
 * synchronisation of cudaMalloc/cudaFree.
 *   tgt_off, src_off : device, n_tasks + 1 offsets each, starting at 0 and
 *                      not decreasing, fewer than 2^32 sources per task;
 *                      tgt_off[n_tasks] must equal n_tgt_total.  Checked on
 *                      the device: a call that breaks any of these computes
 *                      nothing and writes NaN into all n_tgt_total rows of
 *                      out_rows
 *   tgt_xyzm         : device, 4 floats per target (x, y, z, m), 16-byte aligned
 *   src_xyzm         : device, 4 floats per source, 16-byte aligned
 *   out_rows         : device, 8 floats per target, in target order: the
 *                      compensated partial (s0..s3, c0..c3), value s - c =
 *                      (ax, ay, az, phi)
 *   cuda_stream      : cudaStream_t (NULL = legacy default stream)
 * Scratch: one fixed file-scope device array of about 4.5 MiB, kept on
 * every GPU that loads the library until the process exits; shared by all
 * calls, which therefore race if they overlap on the GPU.  The first call
 * on a device (with that device current) performs a one-time set-up
 * (symbol lookup); make it before any stream capture.  Errors:
 * GC_ERR_TOO_LARGE (n_tasks > GC_NOALLOC_MAX_TASKS or n_tgt_total >
 * GC_NOALLOC_MAX_TARGETS), GC_ERR_ARG (eps2 <= 0, null or misaligned
 * pointers), GC_ERR_CUDA (a launch failed, or a CUDA error was already
 * pending when the call began: that error is left pending for its owner and
 * nothing is launched).  Asynchronous: returns after queueing. */
int gc_gravity_noalloc(uint64_t n_tasks, const uint64_t *tgt_off, const float *tgt_xyzm,
                       const uint64_t *src_off, const float *src_xyzm, uint64_t n_tgt_total,
                       float eps2, float *out_rows, void *cuda_stream);

#ifdef __cplusplus
}
#endif

#endif /* GCHARM_H */
