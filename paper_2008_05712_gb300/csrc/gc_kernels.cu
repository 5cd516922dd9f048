// gc_kernels.cu -- the batched hot path after the chare-table step:
//   prepare : task records, result rows, work units (Section 3.1: many
//             requests combined into one launch; each request becomes one
//             or more warp-sized work units pulled from a device queue),
//   pack    : per list, entries ordered by (slot, list position) and
//             gathered from the pool into contiguous float4 staging
//             (Section 3.2, Fig. 1d: threads read data in sorted index order),
//   interact: FP32 pair loops with compensated (Kahan) accumulation --
//             Plummer-softened gravity (Section 4.1) and truncated
//             Lennard-Jones on cell pairs, both cells updated (Section 4.2),
//   scatter : per-id FP64 totals, each id's rows summed in admission order.
#include "gc_common.cuh"

namespace {

inline unsigned grid_for(uint64_t n, int threads, int max_blocks)
{
    uint64_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (uint64_t)max_blocks) b = max_blocks;
    return (unsigned)b;
}

#define GRID_STRIDE(i, n)                                                       \
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < (n); \
         i += (uint64_t)gridDim.x * blockDim.x)

// ---------------------------------------------------------------------------
// task records and preparation
// ---------------------------------------------------------------------------

__global__ void k_task_recs(uint64_t n, const uint64_t *task_ids, const uint32_t *kinds,
                            const int8_t *shifts, const uint64_t *tgt_off,
                            const uint64_t *src_off, uint64_t tgt_base, uint64_t src_base,
                            uint64_t id_base, TaskRec *out, unsigned long long *ctr)
{
    GRID_STRIDE(t, n) {
        TaskRec r;
        r.task_id = task_ids ? task_ids[t] : id_base + t;
        r.kind = kinds[t];
        r.tgt_off = tgt_base + tgt_off[t];
        r.src_off = src_base + src_off[t];
        r.nt = (uint32_t)(tgt_off[t + 1] - tgt_off[t]);
        r.ns = (uint32_t)(src_off[t + 1] - src_off[t]);
        r.row_off = 0;
        for (int a = 0; a < 3; ++a) r.shift[a] = shifts ? shifts[3 * t + a] : (int8_t)0;
        r.shift[3] = 0;
        if (r.kind > GC_LJ_SELF || (r.kind == GC_LJ_SELF && r.ns != 0))
            atomicOr(&ctr[CTR_FLAGS], (unsigned long long)GC_FLAG_BAD_TASK);
        out[t] = r;
    }
}

__global__ void k_prep_counts(const TaskRec *tasks, uint64_t n, uint64_t *rows,
                              uint32_t *wu_g, uint32_t *lj, unsigned long long *ctr)
{
    unsigned long long inter = 0;
    unsigned int mx = 0;
    GRID_STRIDE(t, n) {
        TaskRec r = tasks[t];
        uint64_t rw = r.nt + (r.kind == GC_LJ_PAIR ? r.ns : 0u);
        rows[t] = rw;
        wu_g[t] = (r.kind == GC_GRAVITY) ? (r.nt + 31u) / 32u : 0u;
        lj[t] = (r.kind != GC_GRAVITY) ? 1u : 0u;
        if (r.kind == GC_GRAVITY) inter += (unsigned long long)r.nt * r.ns;
        else if (r.kind == GC_LJ_PAIR) inter += (unsigned long long)r.nt * r.ns;
        else inter += (unsigned long long)r.nt * (r.nt ? r.nt - 1 : 0) / 2;
        mx = max(mx, max(r.nt, r.ns));
    }
    // warp-aggregate before the atomics
    for (int o = 16; o; o >>= 1) {
        inter += __shfl_xor_sync(0xffffffffu, inter, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (inter) atomicAdd(&ctr[CTR_INTER], inter);
        atomicMax(&ctr[CTR_MAXLIST], (unsigned long long)mx);
    }
}

__global__ void k_prep_fill(TaskRec *tasks, uint64_t n, const uint64_t *row_off,
                            const uint32_t *wu_off, const uint32_t *lj_off, GravWU *wu,
                            uint32_t *lj_list)
{
    GRID_STRIDE(t, n) {
        TaskRec &r = tasks[t];
        r.row_off = row_off[t];
        if (r.kind == GC_GRAVITY) {
            uint32_t nb = (r.nt + 31u) / 32u;
            for (uint32_t b = 0; b < nb; ++b) {
                GravWU w;
                w.task = (uint32_t)t;
                w.t0 = b * 32u;
                wu[wu_off[t] + b] = w;
            }
        } else {
            lj_list[lj_off[t]] = (uint32_t)t;
        }
    }
}

// ---------------------------------------------------------------------------
// pack: sort each list by (slot, position), gather into staging
// ---------------------------------------------------------------------------

constexpr int PACK_CAP = 4096;       // keys sorted in shared memory at once
constexpr int PACK_THREADS = 256;

struct PackArgs {
    const TaskRec *tasks;
    uint64_t t0, n_lists;
    const uint32_t *slot_t, *slot_s;     // batch-global entry index
    uint32_t *perm_t, *perm_s;           // batch-global entry index
    float4 *stg_t, *stg_s;               // wave-local entry index
    uint64_t tgt_base, src_base;
    const float4 *pool;
    uint64_t *ma, *mb;                   // merge scratch: targets at the wave-local
    uint64_t msrc;                       // target index, sources at msrc + local index
};

__device__ __forceinline__ void list_of(const PackArgs &a, uint64_t L, uint32_t &n,
                                        uint64_t &off, bool &src)
{
    const TaskRec *r = a.tasks + a.t0 + (L >> 1);
    src = (L & 1) != 0;
    n = src ? r->ns : r->nt;
    off = src ? r->src_off : r->tgt_off;
}

__device__ __forceinline__ void emit_sorted(const PackArgs &a, bool src, uint64_t off,
                                            uint32_t k, uint64_t key)
{
    uint32_t pos = (uint32_t)(key & 0xFFFFFFFFu);
    uint32_t slot = (uint32_t)(key >> 32);
    if (src) {
        a.perm_s[off + k] = pos;
        a.stg_s[off - a.src_base + k] = a.pool[slot];
    } else {
        a.perm_t[off + k] = pos;
        a.stg_t[off - a.tgt_base + k] = a.pool[slot];
    }
}

// Lists of at most 32 entries: one warp, bitonic sort in registers.
__global__ void k_pack_small(PackArgs a)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t L = warp; L < a.n_lists; L += nwarps) {
        uint32_t n;
        uint64_t off;
        bool src;
        list_of(a, L, n, off, src);
        if (n == 0 || n > 32) continue;
        const uint32_t *slots = src ? a.slot_s : a.slot_t;
        uint64_t key = ~0ull;
        if ((uint32_t)lane < n) key = ((uint64_t)slots[off + lane] << 32) | (uint64_t)lane;
#pragma unroll
        for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
            for (int j = k >> 1; j > 0; j >>= 1) {
                uint64_t other = __shfl_xor_sync(0xffffffffu, key, j);
                bool up = (lane & k) == 0;
                bool lower = (lane & j) == 0;
                uint64_t lo = key < other ? key : other;
                uint64_t hi = key < other ? other : key;
                key = (lower == up) ? lo : hi;
            }
        }
        if ((uint32_t)lane < n) emit_sorted(a, src, off, lane, key);
    }
}

__device__ void block_bitonic(uint64_t *s, int np)
{
    for (int k = 2; k <= np; k <<= 1) {
        for (int j = k >> 1; j > 0; j >>= 1) {
            for (int q = threadIdx.x; q < (np >> 1); q += blockDim.x) {
                int i = 2 * j * (q / j) + (q % j);
                int l = i + j;
                uint64_t x = s[i], y = s[l];
                bool up = (i & k) == 0;
                if ((x > y) == up) {
                    s[i] = y;
                    s[l] = x;
                }
            }
            __syncthreads();
        }
    }
}

// Lists of more than 32 entries: one block.  Up to PACK_CAP entries are
// sorted in shared memory; longer lists are sorted in chunks of PACK_CAP and
// merged pairwise in global scratch (keys are unique, so each element's
// output position is its rank in its own run plus its rank in the other).
__global__ void __launch_bounds__(PACK_THREADS) k_pack_large(PackArgs a)
{
    __shared__ uint64_t sk[PACK_CAP];
    for (uint64_t L = blockIdx.x; L < a.n_lists; L += gridDim.x) {
        uint32_t n;
        uint64_t off;
        bool src;
        list_of(a, L, n, off, src);
        if (n <= 32) continue;
        const uint32_t *slots = (src ? a.slot_s : a.slot_t) + off;
        if (n <= (uint32_t)PACK_CAP) {
            int np = 64;
            while (np < (int)n) np <<= 1;
            for (int k = threadIdx.x; k < np; k += blockDim.x)
                sk[k] = (k < (int)n) ? (((uint64_t)slots[k] << 32) | (uint64_t)k) : ~0ull;
            __syncthreads();
            block_bitonic(sk, np);
            for (int k = threadIdx.x; k < (int)n; k += blockDim.x)
                emit_sorted(a, src, off, (uint32_t)k, sk[k]);
            __syncthreads();
            continue;
        }
        uint64_t loc = src ? a.msrc + (off - a.src_base) : off - a.tgt_base;
        uint64_t *A = a.ma + loc;
        uint64_t *B = a.mb + loc;
        for (uint32_t c0 = 0; c0 < n; c0 += PACK_CAP) {
            uint32_t cn = min((uint32_t)PACK_CAP, n - c0);
            int np = 64;
            while (np < (int)cn) np <<= 1;
            for (int k = threadIdx.x; k < np; k += blockDim.x)
                sk[k] = (k < (int)cn) ? (((uint64_t)slots[c0 + k] << 32) | (uint64_t)(c0 + k))
                                      : ~0ull;
            __syncthreads();
            block_bitonic(sk, np);
            for (int k = threadIdx.x; k < (int)cn; k += blockDim.x) A[c0 + k] = sk[k];
            __syncthreads();
        }
        for (uint32_t w = PACK_CAP; w < n; w <<= 1) {
            for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
                uint32_t r = e / w;
                uint32_t ls = (r & ~1u) * w;            // left run start
                uint32_t rs = ls + w;                   // right run start
                uint64_t key = A[e];
                if (rs >= n) {
                    B[e] = key;
                    continue;
                }
                uint32_t re = min(rs + w, n);
                uint32_t lo, hi, rank_other, own;
                if (e < rs) {   // in the left run: count right-run keys < key
                    lo = rs; hi = re;
                    own = e - ls;
                } else {        // in the right run: count left-run keys < key
                    lo = ls; hi = rs;
                    own = e - rs;
                }
                uint32_t base = lo;
                while (lo < hi) {
                    uint32_t mid = (lo + hi) >> 1;
                    if (A[mid] < key) lo = mid + 1; else hi = mid;
                }
                rank_other = lo - base;
                B[ls + own + rank_other] = key;
            }
            __syncthreads();
            uint64_t *t = A; A = B; B = t;
        }
        for (uint32_t k = threadIdx.x; k < n; k += blockDim.x) emit_sorted(a, src, off, k, A[k]);
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// interaction: gravity
// ---------------------------------------------------------------------------

constexpr int GRAV_THREADS = 256;
constexpr int GRAV_WARPS = GRAV_THREADS / 32;
constexpr int KAHAN_BLOCK = 8;   // plain FP32 partial over <= 8 sources, then compensated add

struct InterArgs {
    const TaskRec *tasks;
    const GravWU *wu;
    uint64_t n_wu;
    const uint32_t *lj_list;
    uint64_t n_lj;
    const float4 *stg_t, *stg_s;
    uint64_t tgt_base, src_base;
    const uint32_t *perm_t, *perm_s;
    const uint32_t *tgt_ids, *src_ids;
    float eps2;
    float lj_eps24, lj_eps4, lj_sig2;
    int64_t rc2_grid;
    int32_t edge_grid;
    float4 *res;          // 2 float4 per row: sum, comp
    uint32_t *row_id;
    unsigned long long *queue;   // work-queue head
    unsigned long long *lj_in;
};

__device__ __forceinline__ void kahan_add(float &s, float &c, float v)
{
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Store the FP64 value v as the float pair (s, c) with s - c ~= v.
__device__ __forceinline__ void split_store(float4 *dst, double v0, double v1, double v2,
                                            double v3)
{
    float4 s, c;
    s.x = (float)v0; c.x = (float)((double)s.x - v0);
    s.y = (float)v1; c.y = (float)((double)s.y - v1);
    s.z = (float)v2; c.z = (float)((double)s.z - v2);
    s.w = (float)v3; c.w = (float)((double)s.w - v3);
    dst[0] = s;
    dst[1] = c;
}

// One warp per work unit (task, block of <= 32 targets).  With T targets in
// the block, the warp splits into S = 32 / T source lanes per target: lane
// (t, s) accumulates target t over sources s, s + S, ...; the S partial
// results of a target are combined in FP64 in lane order.  Work units are
// pulled from a device queue (persistent kernel).
__global__ void __launch_bounds__(GRAV_THREADS) k_gravity(InterArgs a)
{
    __shared__ double red[GRAV_WARPS][32][4];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t it = 0;; ++it) {
        unsigned long long w = gwarp + it * nwarps;
        if (a.queue) {
            if (lane == 0) w = atomicAdd(a.queue, 1ull);
            w = __shfl_sync(0xffffffffu, w, 0);
        }
        if (w >= a.n_wu) break;
        GravWU u = a.wu[w];
        const TaskRec r = a.tasks[u.task];
        const int T = (int)min(32u, r.nt - u.t0);
        const int S = 32 / T;
        const int t = lane % T;
        const int sl = lane / T;
        const bool active = sl < S;
        const float4 *src = a.stg_s + (r.src_off - a.src_base);
        const uint32_t ns = r.ns;
        float4 xi = a.stg_t[r.tgt_off - a.tgt_base + u.t0 + t];
        float sx = 0.f, sy = 0.f, sz = 0.f, sp = 0.f;
        float cx = 0.f, cy = 0.f, cz = 0.f, cp = 0.f;
        if (active) {
            uint32_t j = (uint32_t)sl;
            while (j < ns) {
                float bx = 0.f, by = 0.f, bz = 0.f, bp = 0.f;
#pragma unroll
                for (int q = 0; q < KAHAN_BLOCK; ++q) {
                    if (j < ns) {
                        float4 pj = __ldg(src + j);
                        float dx = pj.x - xi.x;
                        float dy = pj.y - xi.y;
                        float dz = pj.z - xi.z;
                        float r2 = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, a.eps2)));
                        float rinv = rsqrtf(r2);
                        float mr = pj.w * rinv;
                        float mr3 = mr * rinv * rinv;
                        bx = fmaf(mr3, dx, bx);
                        by = fmaf(mr3, dy, by);
                        bz = fmaf(mr3, dz, bz);
                        bp -= mr;
                    }
                    j += (uint32_t)S;
                }
                kahan_add(sx, cx, bx);
                kahan_add(sy, cy, by);
                kahan_add(sz, cz, bz);
                kahan_add(sp, cp, bp);
            }
        }
        red[wib][lane][0] = (double)sx - (double)cx;
        red[wib][lane][1] = (double)sy - (double)cy;
        red[wib][lane][2] = (double)sz - (double)cz;
        red[wib][lane][3] = (double)sp - (double)cp;
        __syncwarp();
        if (sl == 0) {
            double v0 = 0, v1 = 0, v2 = 0, v3 = 0;
            for (int q = 0; q < S; ++q) {
                int l = q * T + t;
                v0 += red[wib][l][0];
                v1 += red[wib][l][1];
                v2 += red[wib][l][2];
                v3 += red[wib][l][3];
            }
            uint64_t e = r.tgt_off + u.t0 + t;
            uint32_t pos = a.perm_t[e];
            uint64_t row = r.row_off + pos;
            split_store(a.res + 2 * row, v0, v1, v2, v3);
            a.row_id[row] = a.tgt_ids[r.tgt_off + pos];
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// interaction: Lennard-Jones cell pairs
// ---------------------------------------------------------------------------

// One warp per LJ task.  Every atom of the task is owned by one lane, which
// loops over all its partners: an A atom over cell B (or, in a self task,
// over the other A atoms), a B atom over cell A.  Each pair is therefore
// evaluated from both sides with the same operations, so F_j = -F_i exactly
// (Newton's third law, Section 4.2: interact() updates both patches).
__global__ void __launch_bounds__(GRAV_THREADS) k_lj(InterArgs a)
{
    const int lane = threadIdx.x & 31;
    const float inv_grid = 1.0f / 2097152.0f;
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t it = 0;; ++it) {
        unsigned long long w = gwarp + it * nwarps;
        if (a.queue) {
            if (lane == 0) w = atomicAdd(a.queue, 1ull);
            w = __shfl_sync(0xffffffffu, w, 0);
        }
        if (w >= a.n_lj) break;
        const uint32_t ti = a.lj_list[w];
        const TaskRec r = a.tasks[ti];
        const bool self = r.kind == GC_LJ_SELF;
        const uint32_t nA = r.nt, nB = self ? 0u : r.ns;
        const float4 *As = a.stg_t + (r.tgt_off - a.tgt_base);
        const float4 *Bs = a.stg_s + (r.src_off - a.src_base);
        const int32_t shx = (int32_t)r.shift[0] * a.edge_grid;
        const int32_t shy = (int32_t)r.shift[1] * a.edge_grid;
        const int32_t shz = (int32_t)r.shift[2] * a.edge_grid;
        unsigned long long inside = 0;
        for (uint32_t o = lane; o < nA + nB; o += 32) {
            const bool ownA = o < nA;
            float4 me = ownA ? As[o] : Bs[o - nA];
            // own integer grid position, with the B shift applied to B atoms
            int32_t mx = __float2int_rn(me.x * 2097152.0f);
            int32_t my = __float2int_rn(me.y * 2097152.0f);
            int32_t mz = __float2int_rn(me.z * 2097152.0f);
            if (!ownA) { mx += shx; my += shy; mz += shz; }
            const float4 *P = ownA ? (self ? As : Bs) : As;
            const uint32_t np = ownA ? (self ? nA : nB) : nA;
            const bool pshift = ownA && !self;   // partners are B atoms
            float sx = 0.f, sy = 0.f, sz = 0.f, su = 0.f;
            float cx = 0.f, cy = 0.f, cz = 0.f, cu = 0.f;
            for (uint32_t q = 0; q < np; ++q) {
                if (self && q == o) continue;
                float4 pq = P[q];
                int32_t px = __float2int_rn(pq.x * 2097152.0f);
                int32_t py = __float2int_rn(pq.y * 2097152.0f);
                int32_t pz = __float2int_rn(pq.z * 2097152.0f);
                if (pshift) { px += shx; py += shy; pz += shz; }
                // displacement partner - own, exact integers (|d| < 2^24)
                int32_t dx = px - mx, dy = py - my, dz = pz - mz;
                int64_t r2g = (int64_t)dx * dx + (int64_t)dy * dy + (int64_t)dz * dz;
                if (r2g >= a.rc2_grid) continue;
                if (ownA && (!self || q > o)) ++inside;
                float rx = (float)dx * inv_grid, ry = (float)dy * inv_grid,
                      rz = (float)dz * inv_grid;
                float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                float ir2 = 1.0f / r2;
                float s2 = a.lj_sig2 * ir2;
                float s6 = s2 * s2 * s2;
                float coef = a.lj_eps24 * fmaf(2.0f, s6 * s6, -s6) * ir2;
                float u = a.lj_eps4 * fmaf(s6, s6, -s6);
                // force on own atom: coef * (x_own - x_partner) = -coef * r
                kahan_add(sx, cx, -coef * rx);
                kahan_add(sy, cy, -coef * ry);
                kahan_add(sz, cz, -coef * rz);
                kahan_add(su, cu, 0.5f * u);
            }
            uint64_t row;
            uint32_t id;
            if (ownA) {
                uint32_t pos = a.perm_t[r.tgt_off + o];
                row = r.row_off + pos;
                id = a.tgt_ids[r.tgt_off + pos];
            } else {
                uint32_t pos = a.perm_s[r.src_off + (o - nA)];
                row = r.row_off + nA + pos;
                id = a.src_ids[r.src_off + pos];
            }
            split_store(a.res + 2 * row, (double)sx - (double)cx, (double)sy - (double)cy,
                        (double)sz - (double)cz, (double)su - (double)cu);
            a.row_id[row] = id;
        }
        for (int s = 16; s; s >>= 1) inside += __shfl_xor_sync(0xffffffffu, inside, s);
        if (lane == 0 && inside) atomicAdd(a.lj_in, inside);
    }
}

// ---------------------------------------------------------------------------
// scatter: per-id FP64 totals in admission order
// ---------------------------------------------------------------------------

__global__ void k_iota(uint32_t *v, uint64_t n)
{
    GRID_STRIDE(i, n) v[i] = (uint32_t)i;
}

__global__ void k_reduce_runs(const uint32_t *runs, const unsigned long long *n_runs_dev,
                              uint64_t n_rows, const uint32_t *rid, const uint32_t *row,
                              const float4 *res, gcd4 *totals)
{
    uint64_t nr = *n_runs_dev;
    GRID_STRIDE(k, nr) {
        uint32_t b = runs[k];
        uint32_t e = (k + 1 < nr) ? runs[k + 1] : (uint32_t)n_rows;
        uint32_t id = rid[b];
        gcd4 acc = totals[id];
        for (uint32_t q = b; q < e; ++q) {
            uint32_t rw = row[q];
            float4 s = res[2 * (uint64_t)rw], c = res[2 * (uint64_t)rw + 1];
            acc.x += (double)s.x - (double)c.x;
            acc.y += (double)s.y - (double)c.y;
            acc.z += (double)s.z - (double)c.z;
            acc.w += (double)s.w - (double)c.w;
        }
        totals[id] = acc;
    }
}

}  // namespace

// ---------------------------------------------------------------------------
// host entry points
// ---------------------------------------------------------------------------

int gc_make_task_recs(gc_pool *p, uint64_t n_tasks, const uint64_t *task_ids,
                      const uint32_t *kinds, const int8_t *shifts, const uint64_t *tgt_off,
                      const uint64_t *src_off, uint64_t tgt_base, uint64_t src_base,
                      uint64_t task_id_base, TaskRec *out)
{
    if (n_tasks == 0) return GC_OK;
    ++p->stats.kernel_launches;
    k_task_recs<<<grid_for(n_tasks, 256, p->num_sms * 16), 256, 0, p->s>>>(
        n_tasks, task_ids, kinds, shifts, tgt_off, src_off, tgt_base, src_base, task_id_base,
        out, p->d_ctr);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

// Result rows, work units and LJ task list of the whole batch.  Reads back
// {rows, gravity work units, LJ tasks, interactions, longest list}.
int gc_prepare(gc_pool *p, TaskRec *tasks, uint64_t n, uint64_t info[5])
{
    GC_TRY(p->rowcnt.reserve((n + 1) * sizeof(uint64_t) * 2));
    GC_TRY(p->wu_cnt.reserve((n + 1) * sizeof(uint32_t) * 2));
    GC_TRY(p->wu_off.reserve((n + 1) * sizeof(uint32_t) * 2));
    uint64_t *rows = p->rowcnt.as<uint64_t>();
    uint64_t *row_off = rows + (n + 1);
    uint32_t *wu_g = p->wu_cnt.as<uint32_t>();
    uint32_t *lj = wu_g + (n + 1);
    uint32_t *wu_off = p->wu_off.as<uint32_t>();
    uint32_t *lj_off = wu_off + (n + 1);
    GC_CUDA_TRY(cudaMemsetAsync(p->d_ctr + CTR_INTER, 0, sizeof(unsigned long long) * 5, p->s));
    GC_CUDA_TRY(cudaMemsetAsync(rows + n, 0, sizeof(uint64_t), p->s));
    GC_CUDA_TRY(cudaMemsetAsync(wu_g + n, 0, sizeof(uint32_t), p->s));
    GC_CUDA_TRY(cudaMemsetAsync(lj + n, 0, sizeof(uint32_t), p->s));
    ++p->stats.kernel_launches;
    k_prep_counts<<<grid_for(n, 256, p->num_sms * 16), 256, 0, p->s>>>(tasks, n, rows, wu_g, lj,
                                                                       p->d_ctr);
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u64(p->cub_tmp, rows, row_off, n + 1, p->s));
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u32(p->cub_tmp, wu_g, wu_off, n + 1, p->s));
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u32(p->cub_tmp, lj, lj_off, n + 1, p->s));
    // totals at index n
    uint64_t h_rows = 0;
    uint32_t h_wu = 0, h_lj = 0;
    GC_CUDA_TRY(cudaMemcpyAsync(&h_rows, row_off + n, sizeof(uint64_t), cudaMemcpyDeviceToHost, p->s));
    GC_CUDA_TRY(cudaMemcpyAsync(&h_wu, wu_off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, p->s));
    GC_CUDA_TRY(cudaMemcpyAsync(&h_lj, lj_off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, p->s));
    GC_CUDA_TRY(cudaMemcpyAsync(p->h_ctr + CTR_INTER, p->d_ctr + CTR_INTER,
                                sizeof(unsigned long long) * 5, cudaMemcpyDeviceToHost, p->s));
    GC_CUDA_TRY(cudaStreamSynchronize(p->s));
    GC_TRY(p->wu.reserve(((uint64_t)h_wu + 1) * sizeof(GravWU)));
    GC_TRY(p->small.reserve(((uint64_t)h_lj + 1) * sizeof(uint32_t)));
    ++p->stats.kernel_launches;
    k_prep_fill<<<grid_for(n, 256, p->num_sms * 16), 256, 0, p->s>>>(
        tasks, n, row_off, wu_off, lj_off, p->wu.as<GravWU>(), p->small.as<uint32_t>());
    GC_CUDA_TRY(cudaGetLastError());
    info[0] = h_rows;
    info[1] = h_wu;
    info[2] = h_lj;
    info[3] = p->h_ctr[CTR_INTER];
    info[4] = p->h_ctr[CTR_MAXLIST];
    return GC_OK;
}

// Host copies of the per-task work-unit offsets (for waves and per-task
// launches): wu_off[0..n], lj_off[0..n].
int gc_read_wu_offsets(gc_pool *p, uint64_t n, std::vector<uint32_t> &wu_off,
                       std::vector<uint32_t> &lj_off)
{
    wu_off.resize(n + 1);
    lj_off.resize(n + 1);
    uint32_t *d_wu_off = p->wu_off.as<uint32_t>();
    GC_CUDA_TRY(cudaMemcpyAsync(wu_off.data(), d_wu_off, (n + 1) * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, p->s));
    GC_CUDA_TRY(cudaMemcpyAsync(lj_off.data(), d_wu_off + (n + 1), (n + 1) * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, p->s));
    GC_CUDA_TRY(cudaStreamSynchronize(p->s));
    return GC_OK;
}

int gc_pack(gc_pool *p, const TaskRec *tasks, uint64_t t0, uint64_t t1, uint64_t tgt_base,
            uint64_t src_base, uint64_t msrc)
{
    if (t1 <= t0) return GC_OK;
    PackArgs a;
    a.tasks = tasks;
    a.t0 = t0;
    a.n_lists = 2 * (t1 - t0);
    a.slot_t = p->tgt_slot.as<uint32_t>();
    a.slot_s = p->src_slot.as<uint32_t>();
    a.perm_t = p->tgt_perm.as<uint32_t>();
    a.perm_s = p->src_perm.as<uint32_t>();
    a.stg_t = p->stg_tgt.as<float4>();
    a.stg_s = p->stg_src.as<float4>();
    a.tgt_base = tgt_base;
    a.src_base = src_base;
    a.pool = p->d_pool;
    a.ma = p->merge_a.as<uint64_t>();
    a.mb = p->merge_b.as<uint64_t>();
    a.msrc = msrc;
    ++p->stats.kernel_launches;
    k_pack_small<<<grid_for(a.n_lists * 32, 256, p->num_sms * 32), 256, 0, p->s>>>(a);
    ++p->stats.kernel_launches;
    k_pack_large<<<grid_for(a.n_lists, 1, p->num_sms * 8), PACK_THREADS, 0, p->s>>>(a);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

static int fill_inter_args(gc_pool *p, const TaskRec *tasks, uint64_t tgt_base,
                           uint64_t src_base, const uint32_t *tgt_ids, const uint32_t *src_ids,
                           InterArgs &a)
{
    a.tasks = tasks;
    a.stg_t = p->stg_tgt.as<float4>();
    a.stg_s = p->stg_src.as<float4>();
    a.tgt_base = tgt_base;
    a.src_base = src_base;
    a.perm_t = p->tgt_perm.as<uint32_t>();
    a.perm_s = p->src_perm.as<uint32_t>();
    a.tgt_ids = tgt_ids;
    a.src_ids = src_ids;
    a.eps2 = p->cfg.eps2;
    a.lj_eps24 = 24.0f * p->cfg.lj_eps;
    a.lj_eps4 = 4.0f * p->cfg.lj_eps;
    a.lj_sig2 = p->cfg.lj_sigma * p->cfg.lj_sigma;
    a.rc2_grid = p->rc2_grid;
    a.edge_grid = p->md_edge_grid;
    a.res = p->res.as<float4>();
    a.row_id = p->row_id.as<uint32_t>();
    a.queue = p->d_ctr + CTR_QUEUE;
    a.lj_in = p->d_ctr + CTR_LJ_IN;
    return GC_OK;
}

int gc_grav_blocks(gc_pool *p)
{
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_gravity, GRAV_THREADS, 0) !=
        cudaSuccess || per_sm < 1)
        per_sm = 1;
    return per_sm * p->num_sms;
}

// Launch the interaction kernels over gravity work units [w0, w1) and LJ
// tasks [l0, l1) of the prepared batch.
int gc_interact_range(gc_pool *p, const TaskRec *tasks, const uint32_t *tgt_ids,
                      const uint32_t *src_ids, uint64_t w0, uint64_t w1, uint64_t l0,
                      uint64_t l1, uint64_t tgt_base, uint64_t src_base)
{
    InterArgs a;
    fill_inter_args(p, tasks, tgt_base, src_base, tgt_ids, src_ids, a);
    int full = gc_grav_blocks(p);
    if (w1 > w0) {
        a.wu = p->wu.as<GravWU>() + w0;
        a.n_wu = w1 - w0;
        a.lj_list = nullptr;
        a.n_lj = 0;
        GC_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), p->s));
        uint64_t need = (a.n_wu + GRAV_WARPS - 1) / GRAV_WARPS;
        unsigned g = (unsigned)(need < (uint64_t)full ? need : (uint64_t)full);
        ++p->stats.kernel_launches;
        k_gravity<<<g, GRAV_THREADS, 0, p->s>>>(a);
    }
    if (l1 > l0) {
        a.wu = nullptr;
        a.n_wu = 0;
        a.lj_list = p->small.as<uint32_t>() + l0;
        a.n_lj = l1 - l0;
        GC_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), p->s));
        uint64_t need = (a.n_lj + GRAV_WARPS - 1) / GRAV_WARPS;
        unsigned g = (unsigned)(need < (uint64_t)full ? need : (uint64_t)full);
        ++p->stats.kernel_launches;
        k_lj<<<g, GRAV_THREADS, 0, p->s>>>(a);
    }
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

// One launch per task (the uncombined baseline): the same kernels, static
// work assignment, grid sized to the task.
int gc_interact_one_task(gc_pool *p, const TaskRec *tasks, const uint32_t *tgt_ids,
                         const uint32_t *src_ids, uint64_t w0, uint64_t w1, uint64_t l0,
                         uint64_t l1, uint64_t tgt_base, uint64_t src_base)
{
    InterArgs a;
    fill_inter_args(p, tasks, tgt_base, src_base, tgt_ids, src_ids, a);
    a.queue = nullptr;
    if (w1 > w0) {
        a.wu = p->wu.as<GravWU>() + w0;
        a.n_wu = w1 - w0;
        a.lj_list = nullptr;
        a.n_lj = 0;
        unsigned g = (unsigned)((a.n_wu + GRAV_WARPS - 1) / GRAV_WARPS);
        ++p->stats.kernel_launches;
        k_gravity<<<g, GRAV_THREADS, 0, p->s>>>(a);
    }
    if (l1 > l0) {
        a.wu = nullptr;
        a.n_wu = 0;
        a.lj_list = p->small.as<uint32_t>() + l0;
        a.n_lj = l1 - l0;
        ++p->stats.kernel_launches;
        k_lj<<<1, 32, 0, p->s>>>(a);
    }
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

int gc_scatter(gc_pool *p, uint64_t n_rows)
{
    if (n_rows == 0) return GC_OK;
    GC_TRY(p->rows_tmp.reserve(n_rows * sizeof(uint32_t)));
    GC_TRY(p->rid_sorted.reserve(n_rows * sizeof(uint32_t)));
    GC_TRY(p->row_sorted.reserve(n_rows * sizeof(uint32_t)));
    GC_TRY(p->runs.reserve((n_rows + 1) * sizeof(uint32_t)));
    const int maxb = p->num_sms * 16;
    ++p->stats.kernel_launches;
    k_iota<<<grid_for(n_rows, 256, maxb), 256, 0, p->s>>>(p->rows_tmp.as<uint32_t>(), n_rows);
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) < p->cfg.id_capacity) ++bits;
    ++p->stats.primitive_calls;
    GC_TRY(gc_sort_pairs_u32(p->cub_tmp, p->row_id.as<uint32_t>(), p->rid_sorted.as<uint32_t>(),
                             p->rows_tmp.as<uint32_t>(), p->row_sorted.as<uint32_t>(), n_rows,
                             bits, p->s));
    GC_TRY(gc_compact(p, CK_RUN_START, n_rows, nullptr, p->rid_sorted.as<uint32_t>(),
                      p->runs.as<uint32_t>(), p->d_ctr + CTR_RUNS));
    ++p->stats.kernel_launches;
    k_reduce_runs<<<grid_for(n_rows, 256, maxb), 256, 0, p->s>>>(
        p->runs.as<uint32_t>(), p->d_ctr + CTR_RUNS, n_rows, p->rid_sorted.as<uint32_t>(),
        p->row_sorted.as<uint32_t>(), p->res.as<float4>(), p->d_totals);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}
