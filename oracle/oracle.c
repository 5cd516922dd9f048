/*
 * oracle.c -- plain, slow, single-threaded FP64 CPU reference ("oracle") for
 * the batched irregular-task path of G-Charm (Rengasamy & Vadhiyar,
 * "Strategies for Efficient Executions of Irregular Message-Driven Parallel
 * Applications on GPU Systems", arXiv 2008.05712).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg may load this library.  The product path
 * (the CUDA library) shares no code, header, table or helper with it.
 *
 * What each function follows:
 *   orc_morton_keys / orc_build_tree  -- Section 4.1: particles grouped into
 *       buckets by a Barnes-Hut octree; buckets share one interaction list.
 *       Quantisation, octant order and bucket size are a fixed reading
 *       (the paper gives none): 21-bit grid per axis, Morton key with
 *       x in bit 0, split while a cell holds more than bucket_max particles.
 *   orc_walk         -- Section 4.1: tree walks produce per-bucket
 *       interaction lists of tree nodes and particles; opening criterion is
 *       the integer form of the Barnes-Hut size/distance test.
 *   orc_gravity      -- Section 4.1 gravity force on a bucket: the plain
 *       Plummer-softened sum over the list (definition, not an algorithm).
 *   orc_md_cells / orc_md_tasks / orc_lj -- Section 4.2: space split into
 *       cells (patches); a compute object evaluates interact() on a pair of
 *       cells and updates the force on the particles of BOTH cells.
 *   orc_residency    -- Section 3.2: the chare table maps data ids to device
 *       slots so that resident data is reused instead of re-transferred.
 *   orc_pack_perm    -- Section 3.2 (Fig. 1d): the data indices of a request
 *       are kept sorted by inserting each new index with a binary search, so
 *       threads read data in sorted index order.
 *   orc_reduce       -- per-id FP64 sum of the per-task contributions in
 *       admission order (the engine's cross-task reduction).
 *
 * Precision: every accumulation is FP64; inputs are FP32 values promoted
 * exactly.  Compile with -ffp-contract=off so that no FMA is formed.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

#define ORC_OK 0
#define ORC_ERR_CAP (-1)
#define ORC_ERR_ARG (-2)
#define ORC_ERR_FULL (-3)

#define GRID_BITS 21
#define GRID_MAX ((1u << GRID_BITS) - 1u)
#define NONE32 0xFFFFFFFFu

/* ------------------------------------------------------------------------ */
/* Quantisation and Morton keys                                             */
/* ------------------------------------------------------------------------ */

/* Smallest power of two >= ext (1.0 when ext == 0). */
static double pow2_at_least(double ext)
{
    double L = 1.0;
    if (ext <= 0.0) return 1.0;
    while (L < ext) L *= 2.0;
    while (L * 0.5 >= ext) L *= 0.5;
    return L;
}

/* Bounding box of the float32 coordinates: lo = per-axis min, L = smallest
 * power of two >= the largest per-axis extent. */
static void bounding_grid(int64_t n, const float *xyzm, double lo[3], double *L)
{
    double hi[3];
    for (int a = 0; a < 3; ++a) { lo[a] = INFINITY; hi[a] = -INFINITY; }
    for (int64_t i = 0; i < n; ++i)
        for (int a = 0; a < 3; ++a) {
            double v = (double)xyzm[4 * i + a];
            if (v < lo[a]) lo[a] = v;
            if (v > hi[a]) hi[a] = v;
        }
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) if (hi[a] - lo[a] > ext) ext = hi[a] - lo[a];
    *L = pow2_at_least(ext);
}

/* q = clamp(floor((x - lo) * 2^21 / L), 0, 2^21 - 1), FP64 subtract then
 * multiply by the exact power of two 2^21/L. */
static uint32_t quantise(float x, double lo, double L)
{
    double scale = 2097152.0 / L;
    double t = ((double)x - lo) * scale;
    double f = floor(t);
    if (f < 0.0) f = 0.0;
    if (f > (double)GRID_MAX) f = (double)GRID_MAX;
    return (uint32_t)f;
}

/* Bit b of qx goes to key bit 3b, qy to 3b+1, qz to 3b+2. */
static uint64_t morton3(uint32_t qx, uint32_t qy, uint32_t qz)
{
    uint64_t k = 0;
    for (int b = 0; b < GRID_BITS; ++b) {
        k |= (uint64_t)((qx >> b) & 1u) << (3 * b);
        k |= (uint64_t)((qy >> b) & 1u) << (3 * b + 1);
        k |= (uint64_t)((qz >> b) & 1u) << (3 * b + 2);
    }
    return k;
}

int orc_morton_keys(int64_t n, const float *xyzm, uint64_t *keys, uint32_t *q3,
                    double *lo3, double *L_out)
{
    double lo[3], L;
    if (n <= 0) return ORC_ERR_ARG;
    bounding_grid(n, xyzm, lo, &L);
    for (int64_t i = 0; i < n; ++i) {
        uint32_t qx = quantise(xyzm[4 * i + 0], lo[0], L);
        uint32_t qy = quantise(xyzm[4 * i + 1], lo[1], L);
        uint32_t qz = quantise(xyzm[4 * i + 2], lo[2], L);
        keys[i] = morton3(qx, qy, qz);
        if (q3) { q3[3 * i] = qx; q3[3 * i + 1] = qy; q3[3 * i + 2] = qz; }
    }
    if (lo3) { lo3[0] = lo[0]; lo3[1] = lo[1]; lo3[2] = lo[2]; }
    if (L_out) *L_out = L;
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Octree (top-down recursive split, nodes numbered in DFS preorder)        */
/* ------------------------------------------------------------------------ */

typedef struct {
    const uint64_t *key;      /* keys in sorted order */
    const uint32_t *ids;      /* ids in sorted order */
    const uint32_t *q3;       /* quantised coords by id */
    const float *xyzm;        /* by id */
    int bucket_max;
    int64_t n;
    /* node outputs */
    int64_t node_cap, nn;
    uint8_t *level; uint32_t *cell; uint32_t *first; uint32_t *count;
    uint8_t *leaf; uint32_t *size; double *mono;
    uint32_t *child; /* 8 per node, NONE32 if absent */
    /* bucket outputs */
    int64_t bucket_cap, nb;
    uint32_t *b_first; uint32_t *b_count; uint32_t *b_node; int32_t *b_box;
    int err;
} tree_ctx;

typedef struct { uint64_t key; uint32_t id; } key_id;

static int cmp_key_id(const void *a, const void *b)
{
    const key_id *x = (const key_id *)a, *y = (const key_id *)b;
    if (x->key < y->key) return -1;
    if (x->key > y->key) return 1;
    if (x->id < y->id) return -1;
    if (x->id > y->id) return 1;
    return 0;
}

static int64_t build_node(tree_ctx *c, int level, uint32_t cx, uint32_t cy,
                          uint32_t cz, uint32_t first, uint32_t count)
{
    if (c->nn >= c->node_cap) { c->err = ORC_ERR_CAP; return -1; }
    int64_t me = c->nn++;
    c->level[me] = (uint8_t)level;
    c->cell[3 * me] = cx; c->cell[3 * me + 1] = cy; c->cell[3 * me + 2] = cz;
    c->first[me] = first;
    c->count[me] = count;
    for (int o = 0; o < 8; ++o) c->child[8 * me + o] = NONE32;

    /* monopole: total mass and mass-weighted mean position, FP64, in sorted
     * particle order */
    double m = 0.0, mx = 0.0, my = 0.0, mz = 0.0;
    for (uint32_t k = first; k < first + count; ++k) {
        uint32_t id = c->ids[k];
        double w = (double)c->xyzm[4 * id + 3];
        m += w;
        mx += w * (double)c->xyzm[4 * id + 0];
        my += w * (double)c->xyzm[4 * id + 1];
        mz += w * (double)c->xyzm[4 * id + 2];
    }
    c->mono[4 * me + 0] = m;
    c->mono[4 * me + 1] = (m != 0.0) ? mx / m : 0.0;
    c->mono[4 * me + 2] = (m != 0.0) ? my / m : 0.0;
    c->mono[4 * me + 3] = (m != 0.0) ? mz / m : 0.0;

    if ((int)count > c->bucket_max && level < GRID_BITS) {
        c->leaf[me] = 0;
        int shift = 3 * (GRID_BITS - (level + 1));
        uint32_t k = first;
        for (int o = 0; o < 8; ++o) {
            uint32_t s = k;
            while (k < first + count && (int)((c->key[k] >> shift) & 7u) == o) ++k;
            if (k > s) {
                uint32_t ccx = 2 * cx + (uint32_t)(o & 1);
                uint32_t ccy = 2 * cy + (uint32_t)((o >> 1) & 1);
                uint32_t ccz = 2 * cz + (uint32_t)((o >> 2) & 1);
                int64_t ch = build_node(c, level + 1, ccx, ccy, ccz, s, k - s);
                if (ch < 0) return -1;
                c->child[8 * me + o] = (uint32_t)ch;
            }
        }
        if (k != first + count) { c->err = ORC_ERR_ARG; return -1; }
    } else {
        c->leaf[me] = 1;
        /* a leaf is one bucket, or consecutive chunks of bucket_max when a
         * finest-level cell holds more than bucket_max particles */
        for (uint32_t s = first; s < first + count; s += (uint32_t)c->bucket_max) {
            uint32_t e = s + (uint32_t)c->bucket_max;
            if (e > first + count) e = first + count;
            if (c->nb >= c->bucket_cap) { c->err = ORC_ERR_CAP; return -1; }
            int64_t b = c->nb++;
            c->b_first[b] = s;
            c->b_count[b] = e - s;
            c->b_node[b] = (uint32_t)me;
            int32_t lo[3] = {INT32_MAX, INT32_MAX, INT32_MAX};
            int32_t hi[3] = {INT32_MIN, INT32_MIN, INT32_MIN};
            for (uint32_t k = s; k < e; ++k) {
                uint32_t id = c->ids[k];
                for (int a = 0; a < 3; ++a) {
                    int32_t v = (int32_t)c->q3[3 * id + a];
                    if (v < lo[a]) lo[a] = v;
                    if (v > hi[a]) hi[a] = v;
                }
            }
            /* doubled grid units: particle cell [q, q+1) -> [2q, 2q+2] */
            for (int a = 0; a < 3; ++a) {
                c->b_box[6 * b + a] = 2 * lo[a];
                c->b_box[6 * b + 3 + a] = 2 * hi[a] + 2;
            }
        }
    }
    c->size[me] = (uint32_t)(c->nn - me);
    return me;
}

/*
 * Build the octree over n particles (ids 0..n-1 are array positions).
 * Outputs: sorted ids/keys; nodes in DFS preorder (children in octant
 * order) with level, integer cell coordinates at that level, particle range
 * [first, first+count) in sorted order, leaf flag, subtree node count,
 * FP64 monopole (mass, com x, y, z) and up to 8 child indices; buckets in
 * DFS order with particle range, leaf node and integer box in doubled grid
 * units.
 */
int orc_build_tree(int64_t n, const float *xyzm, int bucket_max,
                   uint32_t *sorted_ids, uint64_t *sorted_keys,
                   int64_t node_cap, int64_t *n_nodes,
                   uint8_t *node_level, uint32_t *node_cell, uint32_t *node_first,
                   uint32_t *node_count, uint8_t *node_leaf, uint32_t *node_size,
                   double *node_mono, uint32_t *node_child,
                   int64_t bucket_cap, int64_t *n_buckets,
                   uint32_t *bucket_first, uint32_t *bucket_count,
                   uint32_t *bucket_node, int32_t *bucket_box)
{
    if (n <= 0 || bucket_max <= 0) return ORC_ERR_ARG;
    uint64_t *keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)n);
    uint32_t *q3 = (uint32_t *)malloc(sizeof(uint32_t) * 3 * (size_t)n);
    key_id *kv = (key_id *)malloc(sizeof(key_id) * (size_t)n);
    if (!keys || !q3 || !kv) { free(keys); free(q3); free(kv); return ORC_ERR_CAP; }
    orc_morton_keys(n, xyzm, keys, q3, NULL, NULL);
    for (int64_t i = 0; i < n; ++i) { kv[i].key = keys[i]; kv[i].id = (uint32_t)i; }
    qsort(kv, (size_t)n, sizeof(key_id), cmp_key_id);
    for (int64_t i = 0; i < n; ++i) { sorted_keys[i] = kv[i].key; sorted_ids[i] = kv[i].id; }
    free(kv);

    tree_ctx c;
    memset(&c, 0, sizeof c);
    c.key = sorted_keys; c.ids = sorted_ids; c.q3 = q3; c.xyzm = xyzm;
    c.bucket_max = bucket_max; c.n = n;
    c.node_cap = node_cap; c.level = node_level; c.cell = node_cell;
    c.first = node_first; c.count = node_count; c.leaf = node_leaf;
    c.size = node_size; c.mono = node_mono; c.child = node_child;
    c.bucket_cap = bucket_cap; c.b_first = bucket_first; c.b_count = bucket_count;
    c.b_node = bucket_node; c.b_box = bucket_box;
    build_node(&c, 0, 0, 0, 0, 0, (uint32_t)n);
    free(keys); free(q3);
    *n_nodes = c.nn;
    *n_buckets = c.nb;
    return c.err;
}

/* ------------------------------------------------------------------------ */
/* Interaction-list walk                                                    */
/* ------------------------------------------------------------------------ */

typedef struct {
    const uint8_t *level; const uint32_t *cell; const uint32_t *first;
    const uint32_t *count; const uint8_t *leaf; const uint32_t *child;
    const uint32_t *sorted_ids;
    int64_t n;                 /* particles: node k has data id n + k */
    int64_t tn, td;            /* theta = tn / td */
    uint32_t bfirst;
    int64_t blo[3], bhi[3];
    uint32_t *out; int64_t cap, len;
    int err;
} walk_ctx;

static void emit(walk_ctx *w, uint32_t id)
{
    if (w->len < w->cap) w->out[w->len] = id;
    else w->err = ORC_ERR_CAP;
    w->len++;
}

static void visit(walk_ctx *w, uint32_t k)
{
    int contains = (w->first[k] <= w->bfirst) &&
                   (w->bfirst < w->first[k] + w->count[k]);
    if (!contains) {
        /* node cell centre and edge in doubled grid units */
        int64_t s = (int64_t)1 << (22 - w->level[k]);
        int64_t d2 = 0;
        for (int a = 0; a < 3; ++a) {
            int64_t c = (int64_t)w->cell[3 * k + a] * s + s / 2;
            int64_t d = 0;
            if (w->blo[a] - c > d) d = w->blo[a] - c;
            if (c - w->bhi[a] > d) d = c - w->bhi[a];
            d2 += d * d;
        }
        /* accept as a monopole iff (s / d) < theta, i.e. td^2 s^2 < tn^2 d^2 */
        if (w->td * w->td * s * s < w->tn * w->tn * d2) {
            emit(w, (uint32_t)(w->n + k));
            return;
        }
    }
    if (w->leaf[k]) {
        for (uint32_t p = w->first[k]; p < w->first[k] + w->count[k]; ++p)
            emit(w, w->sorted_ids[p]);
        return;
    }
    for (int o = 0; o < 8; ++o)
        if (w->child[8 * k + o] != NONE32) visit(w, w->child[8 * k + o]);
}

/* Interaction list of one bucket: DFS from the root, children in octant
 * order.  Nodes whose particle range contains the bucket are always opened;
 * any other node is accepted as a monopole (id n + node index) iff
 * theta_den^2 * s^2 < theta_num^2 * d^2, where s is the node edge and d the
 * distance from the node centre to the bucket box (doubled grid units);
 * ties and d = 0 open.  An opened leaf contributes its particles in sorted
 * order.  Returns the list length in *len (entries beyond cap are counted
 * but not written; err = ORC_ERR_CAP). */
int orc_walk(int64_t n, const uint8_t *node_level, const uint32_t *node_cell,
             const uint32_t *node_first, const uint32_t *node_count,
             const uint8_t *node_leaf, const uint32_t *node_child,
             const uint32_t *sorted_ids, const uint32_t *bucket_first,
             const int32_t *bucket_box, int64_t bucket, int64_t theta_num,
             int64_t theta_den, uint32_t *out, int64_t cap, int64_t *len)
{
    if (theta_den <= 0 || theta_num < 0 || theta_num > 255 || theta_den > 255)
        return ORC_ERR_ARG;
    walk_ctx w;
    memset(&w, 0, sizeof w);
    w.level = node_level; w.cell = node_cell; w.first = node_first;
    w.count = node_count; w.leaf = node_leaf; w.child = node_child;
    w.sorted_ids = sorted_ids; w.n = n; w.tn = theta_num; w.td = theta_den;
    w.bfirst = bucket_first[bucket];
    for (int a = 0; a < 3; ++a) {
        w.blo[a] = bucket_box[6 * bucket + a];
        w.bhi[a] = bucket_box[6 * bucket + 3 + a];
    }
    w.out = out; w.cap = cap;
    visit(&w, 0);
    *len = w.len;
    return w.err;
}

/* ------------------------------------------------------------------------ */
/* Gravity: plain softened sum                                              */
/* ------------------------------------------------------------------------ */

/* For each target i: a_i = sum_j m_j r_ij / (|r_ij|^2 + eps2)^(3/2),
 * phi_i = -sum_j m_j / (|r_ij|^2 + eps2)^(1/2), r_ij = x_j - x_i, G = 1,
 * summed in list order.  Values are looked up by id in table (4 floats per
 * id: x, y, z, m).  out: 4 doubles per target (ax, ay, az, phi). */
void orc_gravity(const float *table, int64_t nt, const uint32_t *tgt, int64_t ns,
                 const uint32_t *src, double eps2, double *out)
{
    for (int64_t i = 0; i < nt; ++i) {
        const float *pi = table + 4 * (size_t)tgt[i];
        double xi = pi[0], yi = pi[1], zi = pi[2];
        double ax = 0.0, ay = 0.0, az = 0.0, phi = 0.0;
        for (int64_t j = 0; j < ns; ++j) {
            const float *pj = table + 4 * (size_t)src[j];
            double dx = (double)pj[0] - xi;
            double dy = (double)pj[1] - yi;
            double dz = (double)pj[2] - zi;
            double m = (double)pj[3];
            double r2 = dx * dx + dy * dy + dz * dz + eps2;
            double rinv = 1.0 / sqrt(r2);
            double rinv3 = rinv * rinv * rinv;
            ax += m * dx * rinv3;
            ay += m * dy * rinv3;
            az += m * dz * rinv3;
            phi -= m * rinv;
        }
        out[4 * i + 0] = ax; out[4 * i + 1] = ay;
        out[4 * i + 2] = az; out[4 * i + 3] = phi;
    }
}

/* Gravity over a whole CSR batch of tasks (loop of orc_gravity). */
void orc_gravity_batch(const float *table, int64_t ntask, const uint64_t *tgt_off,
                       const uint32_t *tgt, const uint64_t *src_off,
                       const uint32_t *src, double eps2, double *out)
{
    for (int64_t t = 0; t < ntask; ++t)
        orc_gravity(table, (int64_t)(tgt_off[t + 1] - tgt_off[t]), tgt + tgt_off[t],
                    (int64_t)(src_off[t + 1] - src_off[t]), src + src_off[t], eps2,
                    out + 4 * tgt_off[t]);
}

/* ------------------------------------------------------------------------ */
/* MD: cells, cell-pair tasks, Lennard-Jones pair interaction              */
/* ------------------------------------------------------------------------ */

/* Group atoms by cell: cell_start (ncell_total + 1) and cell_atoms (n), the
 * atoms of each cell in ascending atom id. */
int orc_md_cells(int64_t n, const uint32_t *cell_of_atom, int64_t ncell_total,
                 uint32_t *cell_start, uint32_t *cell_atoms)
{
    memset(cell_start, 0, sizeof(uint32_t) * (size_t)(ncell_total + 1));
    for (int64_t i = 0; i < n; ++i) {
        if ((int64_t)cell_of_atom[i] >= ncell_total) return ORC_ERR_ARG;
        cell_start[cell_of_atom[i] + 1]++;
    }
    for (int64_t c = 0; c < ncell_total; ++c) cell_start[c + 1] += cell_start[c];
    uint32_t *fill = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)ncell_total);
    if (!fill) return ORC_ERR_CAP;
    for (int64_t c = 0; c < ncell_total; ++c) fill[c] = cell_start[c];
    for (int64_t i = 0; i < n; ++i) cell_atoms[fill[cell_of_atom[i]]++] = (uint32_t)i;
    free(fill);
    return ORC_OK;
}

/* Tasks of a periodic m^3 cell grid: for every cell c in ascending linear
 * index (c = x + m (y + m z)), first the self task, then one task per
 * neighbour offset d = (dx, dy, dz) in {-1,0,1}^3 that is lexicographically
 * greater than (0,0,0) with dx most significant (13 offsets), in that
 * order.  Cell B = c + d wrapped; d is the unwrapped offset of B from A. */
int orc_md_tasks(int64_t m, uint32_t *cell_a, uint32_t *cell_b, int8_t *d3,
                 uint8_t *is_self)
{
    int64_t t = 0;
    for (int64_t c = 0; c < m * m * m; ++c) {
        int64_t x = c % m, y = (c / m) % m, z = c / (m * m);
        cell_a[t] = (uint32_t)c; cell_b[t] = (uint32_t)c;
        d3[3 * t] = 0; d3[3 * t + 1] = 0; d3[3 * t + 2] = 0; is_self[t] = 1;
        ++t;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy)
                for (int dz = -1; dz <= 1; ++dz) {
                    int later = (dx > 0) || (dx == 0 && dy > 0) ||
                                (dx == 0 && dy == 0 && dz > 0);
                    if (!later) continue;
                    int64_t bx = (x + dx + m) % m, by = (y + dy + m) % m, bz = (z + dz + m) % m;
                    cell_a[t] = (uint32_t)c;
                    cell_b[t] = (uint32_t)(bx + m * (by + m * bz));
                    d3[3 * t] = (int8_t)dx; d3[3 * t + 1] = (int8_t)dy; d3[3 * t + 2] = (int8_t)dz;
                    is_self[t] = 0;
                    ++t;
                }
    }
    return (int)t;
}

/* The planar case (the paper's MD is two-dimensional, Section 4.2): a
 * periodic m x m cell grid, c = x + m y; for every cell, the self task, then
 * one task per offset (dx, dy) in {-1,0,1}^2 lexicographically greater than
 * (0,0) with dx most significant (4 offsets); the z offset is 0. */
int orc_md_tasks_2d(int64_t m, uint32_t *cell_a, uint32_t *cell_b, int8_t *d3,
                    uint8_t *is_self)
{
    int64_t t = 0;
    for (int64_t c = 0; c < m * m; ++c) {
        int64_t x = c % m, y = c / m;
        cell_a[t] = (uint32_t)c; cell_b[t] = (uint32_t)c;
        d3[3 * t] = 0; d3[3 * t + 1] = 0; d3[3 * t + 2] = 0; is_self[t] = 1;
        ++t;
        for (int dx = -1; dx <= 1; ++dx)
            for (int dy = -1; dy <= 1; ++dy) {
                int later = (dx > 0) || (dx == 0 && dy > 0);
                if (!later) continue;
                int64_t bx = (x + dx + m) % m, by = (y + dy + m) % m;
                cell_a[t] = (uint32_t)c;
                cell_b[t] = (uint32_t)(bx + m * by);
                d3[3 * t] = (int8_t)dx; d3[3 * t + 1] = (int8_t)dy; d3[3 * t + 2] = 0;
                is_self[t] = 0;
                ++t;
            }
    }
    return (int)t;
}

/*
 * Lennard-Jones forces of one cell-pair task.  Atoms carry local offsets u
 * (table: 4 floats per id, u exact multiples of 2^-21); atom j of cell B
 * sits at u_j + d * edge relative to cell A's origin.  A pair is inside the
 * cutoff iff |r|^2 < rc^2, decided exactly on the 2^-21 grid (rc2_grid =
 * rc^2 * 2^42, E = edge * 2^21).  For an included pair, with
 * s6 = (sigma^2/r^2)^3:
 *   F_i = 24 eps (2 s6^2 - s6) / r^2 * (x_i - x_j),  F_j = -F_i,
 *   U   = 4 eps (s6^2 - s6), half to each atom (4th component).
 * Self task (is_self != 0): pairs i < j of list A.  outA: 4 doubles per A
 * atom, outB: 4 doubles per B atom (unused for self tasks).
 */
int orc_lj(const float *table, int64_t na, const uint32_t *a, int64_t nb,
           const uint32_t *b, int is_self, const int8_t *d3, int64_t E,
           double eps, double sigma, int64_t rc2_grid, double *outA, double *outB)
{
    const double S = 2097152.0;
    memset(outA, 0, sizeof(double) * 4 * (size_t)na);
    if (!is_self) memset(outB, 0, sizeof(double) * 4 * (size_t)nb);
    int64_t nj = is_self ? na : nb;
    const uint32_t *bl = is_self ? a : b;
    for (int64_t i = 0; i < na; ++i) {
        const float *ui = table + 4 * (size_t)a[i];
        int64_t Ui[3];
        for (int k = 0; k < 3; ++k) Ui[k] = (int64_t)((double)ui[k] * S);
        for (int64_t j = is_self ? i + 1 : 0; j < nj; ++j) {
            const float *uj = table + 4 * (size_t)bl[j];
            int64_t D[3];
            int64_t r2g = 0;
            for (int k = 0; k < 3; ++k) {
                int64_t Uj = (int64_t)((double)uj[k] * S);
                D[k] = Uj + (int64_t)d3[k] * E - Ui[k];   /* x_j - x_i, grid units */
                r2g += D[k] * D[k];
            }
            if (!(r2g < rc2_grid)) continue;
            double rx = (double)D[0] / S, ry = (double)D[1] / S, rz = (double)D[2] / S;
            double r2 = rx * rx + ry * ry + rz * rz;
            double s2 = sigma * sigma / r2;
            double s6 = s2 * s2 * s2;
            double coef = 24.0 * eps * (2.0 * s6 * s6 - s6) / r2;
            double U = 4.0 * eps * (s6 * s6 - s6);
            /* F_i = coef * (x_i - x_j) = -coef * r */
            double fx = -coef * rx, fy = -coef * ry, fz = -coef * rz;
            outA[4 * i + 0] += fx; outA[4 * i + 1] += fy; outA[4 * i + 2] += fz;
            outA[4 * i + 3] += 0.5 * U;
            double *oj = is_self ? outA + 4 * j : outB + 4 * j;
            oj[0] -= fx; oj[1] -= fy; oj[2] -= fz; oj[3] += 0.5 * U;
        }
    }
    return ORC_OK;
}

/* ------------------------------------------------------------------------ */
/* Residency (chare table) and pack permutation                             */
/* ------------------------------------------------------------------------ */

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return (x > y) - (x < y);
}

/*
 * One flush of the residency table.  State (updated in place):
 *   slot_of_id[id_cap]   NONE32 if id not resident
 *   id_of_slot[cap]      NONE32 if slot free
 *   last_use[cap]        epoch of the last flush that referenced the slot
 * Policy for the batch's entry ids:
 *   U = sorted unique ids; hits = resident members of U, misses = the rest.
 *   If misses exceed free slots, evict resident ids not in U in ascending
 *   (last_use, slot) order until enough slots are free; if that is not
 *   possible, return ORC_ERR_FULL with the state untouched.
 *   Misses, in ascending id order, take the free slots in ascending slot
 *   order.  Every slot of U gets last_use = epoch.
 * Outputs: entry_slots[n_entries]; miss_ids (ascending, stats[1] of them);
 * evicted ids (ascending slot order of eviction selection, stats[2]);
 * reuse[k] = multiplicity of the k-th unique id; stats = {hits, misses,
 * evictions, unique}.
 */
int orc_residency(int64_t id_cap, int64_t cap, uint32_t *slot_of_id,
                  uint32_t *id_of_slot, uint32_t *last_use, uint32_t epoch,
                  int64_t n_entries, const uint32_t *entry_ids,
                  uint32_t *entry_slots, uint32_t *uniq_out, uint32_t *reuse,
                  uint32_t *miss_ids, uint32_t *evicted_ids, int64_t *stats)
{
    for (int64_t e = 0; e < n_entries; ++e)
        if ((int64_t)entry_ids[e] >= id_cap) return ORC_ERR_ARG;
    uint32_t *srt = (uint32_t *)malloc(sizeof(uint32_t) * (size_t)(n_entries + 1));
    if (!srt) return ORC_ERR_CAP;
    memcpy(srt, entry_ids, sizeof(uint32_t) * (size_t)n_entries);
    qsort(srt, (size_t)n_entries, sizeof(uint32_t), cmp_u32);
    int64_t nu = 0;
    for (int64_t e = 0; e < n_entries; ++e) {
        if (nu > 0 && uniq_out[nu - 1] == srt[e]) { reuse[nu - 1]++; continue; }
        uniq_out[nu] = srt[e]; reuse[nu] = 1; ++nu;
    }
    free(srt);
    int64_t hits = 0, misses = 0;
    for (int64_t k = 0; k < nu; ++k) {
        if (slot_of_id[uniq_out[k]] != NONE32) ++hits;
        else miss_ids[misses++] = uniq_out[k];
    }
    int64_t nfree = 0;
    for (int64_t s = 0; s < cap; ++s) if (id_of_slot[s] == NONE32) ++nfree;
    int64_t nevict = 0;
    if (misses > nfree) {
        int64_t need = misses - nfree;
        /* candidates: resident slots whose id is not referenced now */
        uint64_t *cand = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(cap + 1));
        if (!cand) return ORC_ERR_CAP;
        int64_t nc = 0;
        for (int64_t s = 0; s < cap; ++s) {
            uint32_t id = id_of_slot[s];
            if (id == NONE32) continue;
            /* is id in U?  binary search */
            int64_t lo = 0, hi = nu;
            while (lo < hi) {
                int64_t mid = (lo + hi) / 2;
                if (uniq_out[mid] < id) lo = mid + 1; else hi = mid;
            }
            if (lo < nu && uniq_out[lo] == id) continue;
            cand[nc++] = ((uint64_t)last_use[s] << 32) | (uint64_t)s;
        }
        if (nc < need) { free(cand); return ORC_ERR_FULL; }
        qsort(cand, (size_t)nc, sizeof(uint64_t), cmp_u64);
        for (int64_t k = 0; k < need; ++k) {
            uint32_t s = (uint32_t)(cand[k] & 0xFFFFFFFFu);
            uint32_t id = id_of_slot[s];
            evicted_ids[nevict++] = id;
            slot_of_id[id] = NONE32;
            id_of_slot[s] = NONE32;
        }
        free(cand);
    }
    int64_t k = 0;
    for (int64_t s = 0; s < cap && k < misses; ++s) {
        if (id_of_slot[s] != NONE32) continue;
        id_of_slot[s] = miss_ids[k];
        slot_of_id[miss_ids[k]] = (uint32_t)s;
        ++k;
    }
    for (int64_t u = 0; u < nu; ++u) last_use[slot_of_id[uniq_out[u]]] = epoch;
    for (int64_t e = 0; e < n_entries; ++e) entry_slots[e] = slot_of_id[entry_ids[e]];
    stats[0] = hits; stats[1] = misses; stats[2] = nevict; stats[3] = nu;
    return ORC_OK;
}

/* Pack order of one list: positions 0..n-1 ordered by (slot, position),
 * built by inserting each position in turn into an already sorted array at
 * the place found by binary search (after all entries with slot <= its
 * slot), as in Section 3.2.  perm[k] = list position of the k-th staged
 * entry. */
void orc_pack_perm(int64_t n, const uint32_t *slots, uint32_t *perm)
{
    for (int64_t p = 0; p < n; ++p) {
        uint32_t s = slots[p];
        int64_t lo = 0, hi = p;           /* perm[0..p) is sorted */
        while (lo < hi) {
            int64_t mid = (lo + hi) / 2;
            if (slots[perm[mid]] <= s) lo = mid + 1; else hi = mid;
        }
        memmove(perm + lo + 1, perm + lo, sizeof(uint32_t) * (size_t)(p - lo));
        perm[lo] = (uint32_t)p;
    }
}

/* Pack permutation of a CSR batch of lists (loop of orc_pack_perm). */
void orc_pack_perm_batch(int64_t nlist, const uint64_t *off, const uint32_t *slots,
                         uint32_t *perm)
{
    for (int64_t t = 0; t < nlist; ++t)
        orc_pack_perm((int64_t)(off[t + 1] - off[t]), slots + off[t], perm + off[t]);
}

/* ------------------------------------------------------------------------ */
/* Cross-task reduction                                                      */
/* ------------------------------------------------------------------------ */

/* totals[4*id + c] += contrib[4*k + c] for k = 0..n-1 in order (admission
 * order of the contributions), FP64. */
void orc_reduce(int64_t n, const uint32_t *ids, const double *contrib, double *totals)
{
    for (int64_t k = 0; k < n; ++k)
        for (int c = 0; c < 4; ++c)
            totals[4 * (size_t)ids[k] + c] += contrib[4 * k + c];
}

/* ------------------------------------------------------------------------ */
/* Time integration (the step around the force computation, Section 4.1)    */
/* ------------------------------------------------------------------------ */

/*
 * Leapfrog with staggered velocities, one step of length dt:
 *   v' = v + a dt        (kick, a = acceleration at the current positions)
 *   x' = x + v' dt       (drift)
 * State in float32 (x, y, z, m and vx, vy, vz, 0 per particle), arithmetic
 * in FP64, each new value rounded once to float32: v' = fl(v + a*dt),
 * x' = fl(x + v'*dt) with v' the rounded velocity.  Masses unchanged.
 */
void orc_kick_drift(int64_t n, const double *acc, float *xyzm, float *vel, double dt)
{
    for (int64_t i = 0; i < n; ++i) {
        for (int c = 0; c < 3; ++c) {
            double v = (double)vel[4 * i + c] + acc[4 * i + c] * dt;
            float vf = (float)v;
            vel[4 * i + c] = vf;
            xyzm[4 * i + c] = (float)((double)xyzm[4 * i + c] + (double)vf * dt);
        }
    }
}

/* ------------------------------------------------------------------------ */
/* Periodic gravity: Ewald correction (the tree code's second combined      */
/* kernel, Section 4.1)                                                     */
/* ------------------------------------------------------------------------ */

/*
 * Ewald summation for a point mass in a periodic cube of side L with a
 * uniform neutralising background (G = 1, no softening).  For the
 * displacement r = x_target - x_source, the periodic Green's function is
 *   psi(r) = sum_n erfc(alpha |r + nL|) / |r + nL|
 *          + 1/(pi L) sum_{h != 0} exp(-pi^2 h^2 / (alpha L)^2) / h^2 cos(2 pi h.r / L)
 *          - pi / (alpha^2 L^3),
 * n over integer vectors with max |n_i| <= nrep, h over integer vectors with
 * 0 < |h|^2 <= hcut2.  The potential of mass M is -M psi and its
 * acceleration M grad psi.  The correction returned is the periodic
 * interaction minus the plain point-mass term of r itself:
 *   a_corr = M grad psi(r) + M r / |r|^3,   phi_corr = -M (psi(r) - 1/|r|),
 * finite at r = 0.  The n = 0 real-space term and the subtracted term are
 * combined (-erf(alpha s)/s, and its gradient) and, for alpha s < 1/2,
 * evaluated from the Taylor series of erf so that nothing cancels.
 */
#define ORC_PI 3.14159265358979323846

static void ewald_pair(const double r[3], double M, double L, double alpha, int nrep,
                       int hcut2, double out[4])
{
    const double sqpi = sqrt(ORC_PI);
    double ax = 0, ay = 0, az = 0, phi = 0;   /* of grad psi and psi - 1/|r| */
    for (int nx = -nrep; nx <= nrep; ++nx)
        for (int ny = -nrep; ny <= nrep; ++ny)
            for (int nz = -nrep; nz <= nrep; ++nz) {
                double d[3] = {r[0] + nx * L, r[1] + ny * L, r[2] + nz * L};
                double s2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                double s = sqrt(s2);
                double g, p;   /* grad term = -d * g; potential term p */
                if (nx == 0 && ny == 0 && nz == 0) {
                    /* erfc(alpha s)/s - 1/s = -erf(alpha s)/s: p = -alpha erf(x)/x,
                     * and its gradient -d g with g = alpha^3 f(x),
                     * f(x) = -erf(x)/x^3 + 2/sqrt(pi) exp(-x^2)/x^2 */
                    double x = alpha * s;
                    if (x < 0.5) {
                        /* erf(x)/x = 2/sqrt(pi) sum_{k>=0} (-1)^k x^(2k) / (k! (2k+1))
                         * f(x)     = 2/sqrt(pi) sum_{k>=1} (-1)^k x^(2k-2) 2k / (k! (2k+1)) */
                        double x2 = x * x, e = 0.0, fk = 0.0;
                        double t = 1.0;             /* (-1)^k x^(2k) / k!   at k = 0 */
                        for (int k = 0; k < 18; ++k) {
                            e += t / (2 * k + 1);
                            t *= -x2 / (k + 1);
                        }
                        double u = -1.0;            /* (-1)^k x^(2k-2) / k! at k = 1 */
                        for (int k = 1; k < 18; ++k) {
                            fk += u * (2.0 * k) / (2 * k + 1);
                            u *= -x2 / (k + 1);
                        }
                        g = alpha * alpha * alpha * (2.0 / sqpi) * fk;
                        p = -alpha * (2.0 / sqpi) * e;
                    } else {
                        g = -erf(x) / (s2 * s) + 2.0 * alpha / sqpi * exp(-x * x) / s2;
                        p = -erf(x) / s;
                    }
                } else {
                    double x = alpha * s;
                    g = erfc(x) / (s2 * s) + 2.0 * alpha / sqpi * exp(-x * x) / s2;
                    p = erfc(x) / s;
                }
                /* grad of the term is -d * g */
                ax -= d[0] * g; ay -= d[1] * g; az -= d[2] * g;
                phi += p;
            }
    const int hm = (int)ceil(sqrt((double)hcut2));
    for (int hx = -hm; hx <= hm; ++hx)
        for (int hy = -hm; hy <= hm; ++hy)
            for (int hz = -hm; hz <= hm; ++hz) {
                int h2 = hx * hx + hy * hy + hz * hz;
                if (h2 == 0 || h2 > hcut2) continue;
                double c = exp(-ORC_PI * ORC_PI * h2 / (alpha * alpha * L * L)) / h2;
                double arg = 2.0 * ORC_PI * (hx * r[0] + hy * r[1] + hz * r[2]) / L;
                phi += c * cos(arg) / (ORC_PI * L);
                double gs = -c * sin(arg) * 2.0 / (L * L);
                ax += gs * hx; ay += gs * hy; az += gs * hz;
            }
    phi -= ORC_PI / (alpha * alpha * L * L * L);
    out[0] += M * ax;
    out[1] += M * ay;
    out[2] += M * az;
    out[3] += -M * phi;
}

/* Ewald corrections of nt targets from the same ns sources (table rows
 * x, y, z, m), summed in source order: out[4t..4t+3] = (ax, ay, az, phi). */
void orc_ewald(const float *table, int64_t nt, const uint32_t *tgt, int64_t ns,
               const uint32_t *src, double L, double alpha, int nrep, int hcut2,
               double *out)
{
    for (int64_t t = 0; t < nt; ++t) {
        const float *xt = table + 4 * (size_t)tgt[t];
        double acc[4] = {0, 0, 0, 0};
        for (int64_t j = 0; j < ns; ++j) {
            const float *xs = table + 4 * (size_t)src[j];
            double r[3] = {(double)xt[0] - (double)xs[0], (double)xt[1] - (double)xs[1],
                           (double)xt[2] - (double)xs[2]};
            ewald_pair(r, (double)xs[3], L, alpha, nrep, hcut2, acc);
        }
        for (int c = 0; c < 4; ++c) out[4 * t + c] = acc[c];
    }
}
