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
#include "gc_ptx.cuh"

namespace {

// ---------------------------------------------------------------------------
// task records and preparation
// ---------------------------------------------------------------------------

__global__ void k_task_recs(uint64_t n, const uint64_t *task_ids, const uint32_t *kinds,
                            const int8_t *shifts, const uint64_t *tgt_off,
                            const uint64_t *src_off, uint64_t tgt_base, uint64_t src_base,
                            uint64_t id_base, TaskRec *out, unsigned long long *ctr,
                            int ewald_ok)
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
        if (r.kind > GC_EWALD || (r.kind == GC_LJ_SELF && r.ns != 0) ||
            (r.kind == GC_EWALD && !ewald_ok))
            atomicOr(&ctr[CTR_FLAGS], (unsigned long long)GC_FLAG_BAD_TASK);
        out[t] = r;
    }
}

__global__ void k_prep_counts(const TaskRec *tasks, uint64_t n, uint64_t *rows,
                              uint32_t *wu_g, uint32_t *lj, unsigned long long *ctr,
                              uint32_t wu_max)
{
    unsigned long long inter = 0;
    unsigned int mx = 0;
    GRID_STRIDE(t, n) {
        TaskRec r = tasks[t];
        uint64_t rw = r.nt + (r.kind == GC_LJ_PAIR ? r.ns : 0u);
        rows[t] = rw;
        wu_g[t] = (r.kind == GC_GRAVITY) ? (r.nt + wu_max - 1u) / wu_max : 0u;
        lj[t] = (r.kind != GC_GRAVITY) ? 1u : 0u;
        if (r.kind == GC_GRAVITY || r.kind == GC_LJ_PAIR || r.kind == GC_EWALD)
            inter += (unsigned long long)r.nt * r.ns;
        else inter += (unsigned long long)r.nt * (r.nt ? r.nt - 1 : 0) / 2;
        mx = max(mx, max(r.nt, r.ns));
    }
    // warp-aggregate before the atomics
    for (int o = 16; o; o >>= 1) {
        inter += __shfl_xor_sync(0xffffffffu, inter, o);
        mx = max(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (inter) atomicAdd(&ctr[FC_INTER], inter);
        atomicMax(&ctr[FC_MAXLIST], (unsigned long long)mx);
    }
}

__global__ void k_prep_fill(TaskRec *tasks, uint64_t n, const uint64_t *row_off,
                            const uint32_t *wu_off, const uint32_t *lj_off, GravWU *wu,
                            uint32_t *lj_list, uint32_t wu_max)
{
    GRID_STRIDE(t, n) {
        TaskRec &r = tasks[t];
        if (row_off) r.row_off = row_off[t];
        if (r.kind == GC_GRAVITY) {
            // blocks of at most wu_max targets, sizes as equal as possible
            uint32_t nb = (r.nt + wu_max - 1u) / wu_max;
            uint32_t bs = nb ? (r.nt + nb - 1u) / nb : 0u;
            for (uint32_t b = 0; b < nb; ++b) {
                GravWU w;
                w.task = (uint32_t)t;
                w.t0 = b * bs;
                w.tn = min(bs, r.nt - b * bs);
                w.pad = 0;
                wu[wu_off[t] + b] = w;
            }
        } else if (lj_list) {
            lj_list[lj_off[t]] = (uint32_t)t;
        }
    }
}

// Longest-first order of work units: sort key = (2^40 - 1) - targets x
// sources (a stable radix sort keeps admission order among equal costs).
__global__ void k_wu_cost(const GravWU *wu, uint64_t n, const TaskRec *tasks, uint64_t *key,
                          uint32_t *idx)
{
    GRID_STRIDE(i, n) {
        const GravWU w = wu[i];
        const uint64_t cost = (uint64_t)w.tn * tasks[w.task].ns;
        key[i] = ((1ull << 40) - 1ull) - cost;
        idx[i] = (uint32_t)i;
    }
}

__global__ void k_wu_gather(const GravWU *wu, const uint32_t *idx, uint64_t n, GravWU *out)
{
    GRID_STRIDE(i, n) out[i] = wu[idx[i]];
}

// ---------------------------------------------------------------------------
// pack: sort each list by (slot, position), gather into staging
// ---------------------------------------------------------------------------
//
// Staging layouts (wave-local, float4 units):
//   targets           : AoS, entry k of a list at (tgt_off - tgt_base) + k.
//   gravity sources   : paired SoA, for the list of task t starting at
//                       S_t = (src_off - src_base) + (t - task_base):
//                       float4 S_t + 2q     = (x_2q, x_2q+1, y_2q, y_2q+1)
//                       float4 S_t + 2q + 1 = (z_2q, z_2q+1, m_2q, m_2q+1)
//                       an odd list is padded with a zero-mass source;
//                       two sources then sit in register pairs ready for
//                       the paired FP32 instructions of the kernel.
//   LJ sources        : AoS at S_t + k.
// The extra float4 per task keeps every padded segment inside its own range.

constexpr int PK_CAP = 4096;          // entries sorted in shared memory at once
constexpr int PK_CAP_HUGE = 16384;    // the same, one block per SM (about 200 KB)

struct PackArgs {
    const TaskRec *tasks;
    uint64_t t0, n_lists;
    const uint32_t *tgt_ids, *src_ids;   // batch-global entry index
    const uint32_t *slot_of_id;
    const uint32_t *ent_t, *ent_s;       // entry slots (wave-local index; NONE: look up), or null
    uint32_t *perm_t, *perm_s;           // batch-global entry index
    float4 *stg_t, *stg_s;               // wave-local staging
    uint64_t tgt_base, src_base, task_base;
    const float4 *pool;
    uint64_t *ma, *mb;                   // merge scratch: targets at the wave-local
    uint64_t msrc;                       // target index, sources at msrc + local index
    int passes;                          // radix passes of 8 bits over the slot
    unsigned long long *work;            // list-claim counters, one per block kernel
};

struct PackList {
    uint32_t n;
    uint64_t off;     // batch-global first entry
    bool src;
    bool paired;      // gravity source list
    uint64_t stg;     // first staging float4 (wave-local)
    const uint32_t *es;   // entry slots of the list, or null
};

__device__ __forceinline__ PackList list_of(const PackArgs &a, uint64_t L)
{
    const uint64_t t = a.t0 + (L >> 1);
    const TaskRec *r = a.tasks + t;
    PackList l;
    l.src = (L & 1) != 0;
    l.n = l.src ? r->ns : r->nt;
    l.off = l.src ? r->src_off : r->tgt_off;
    l.paired = l.src && r->kind == GC_GRAVITY;
    l.stg = l.src ? (l.off - a.src_base) + (t - a.task_base) : l.off - a.tgt_base;
    l.es = !a.ent_t ? nullptr
                    : (l.src ? a.ent_s + (l.off - a.src_base) : a.ent_t + (l.off - a.tgt_base));
    return l;
}

__device__ __forceinline__ uint32_t list_n(const PackArgs &a, uint64_t L)
{
    const TaskRec *r = a.tasks + a.t0 + (L >> 1);
    return (L & 1) ? r->ns : r->nt;
}

// Slot of entry k of list l: the slot recorded by the chare-table step, or
// (a miss placed after it, or no record) a lookup.
__device__ __forceinline__ uint32_t entry_slot(const PackArgs &a, const PackList &l,
                                               const uint32_t *ids, uint32_t k)
{
    if (l.es) {
        const uint32_t s = __ldg(l.es + k);
        if (s != GC_NONE) return s;
    }
    return __ldg(a.slot_of_id + __ldg(ids + k));
}

// The block-per-list kernels claim lists dynamically, PK_CHUNK at a time
// from a device counter, and keep those of their size class: every block
// stays busy whatever the mix of list sizes (a static stride over lists
// 2t, 2t+1 would hand all target lists to half of the blocks).
constexpr int PK_CHUNK = 16;

struct ListClaim {
    uint64_t base;
    uint32_t cnt;
    uint8_t off[PK_CHUNK];
};

// Claim the next PK_CHUNK lists; keep those with lo < n <= hi.  Block-wide
// (barriers before and after: every thread is done reading the previous
// claim); false once the lists are exhausted.
__device__ __forceinline__ bool claim_lists(const PackArgs &a, unsigned long long *ctr,
                                            uint32_t lo, uint32_t hi, ListClaim &cl)
{
    __syncthreads();
    if (threadIdx.x < 32) {
        const int lane = threadIdx.x;
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(ctr, (unsigned long long)PK_CHUNK);
        base = __shfl_sync(0xffffffffu, base, 0);
        const uint64_t L = base + (uint64_t)lane;
        bool q = false;
        if (lane < PK_CHUNK && L < a.n_lists) {
            const uint32_t n = list_n(a, L);
            q = n > lo && n <= hi;
        }
        const uint32_t bal = __ballot_sync(0xffffffffu, q);
        if (q) cl.off[__popc(bal & ((1u << lane) - 1u))] = (uint8_t)lane;
        if (lane == 0) {
            cl.base = base;
            cl.cnt = (uint32_t)__popc(bal);
        }
    }
    __syncthreads();
    return cl.base < a.n_lists;
}

// write staged entry k (list position pos, pool slot) of list l
__device__ __forceinline__ void emit(const PackArgs &a, const PackList &l, uint32_t k,
                                     uint32_t slot, uint32_t pos)
{
    float4 v = a.pool[slot];
    if (!l.src) {
        a.perm_t[l.off + k] = pos;
        a.stg_t[l.stg + k] = v;
        return;
    }
    a.perm_s[l.off + k] = pos;
    if (!l.paired) {
        a.stg_s[l.stg + k] = v;
        return;
    }
    float *f = reinterpret_cast<float *>(a.stg_s + l.stg + 2 * (k >> 1));
    const uint32_t h = k & 1u;
    f[h] = v.x;
    f[2 + h] = v.y;
    f[4 + h] = v.z;
    f[6 + h] = v.w;
    if (h == 0 && k + 1 == l.n) {   // odd list: zero-mass pad source
        f[1] = 0.f;
        f[3] = 0.f;
        f[5] = 0.f;
        f[7] = 0.f;
    }
}

// Bitonic sort of one (slot << 32 | pos) key per lane over groups of G
// lanes (G = 16 or 32; xor partners stay inside the group), ascending.
template <int G>
__device__ __forceinline__ uint64_t bitonic_lanes(uint64_t key, int gl)
{
#pragma unroll
    for (int k = 2; k <= G; k <<= 1) {
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            const uint64_t other = __shfl_xor_sync(0xffffffffu, key, j);
            const bool up = (gl & k) == 0;
            const bool lower = (gl & j) == 0;
            const uint64_t lo = key < other ? key : other;
            const uint64_t hi = key < other ? other : key;
            key = (lower == up) ? lo : hi;
        }
    }
    return key;
}

// Lists of at most 32 entries: bitonic sort of (slot, pos) keys in
// registers.  A warp takes the two lists of one task; when both hold at most
// 16 entries (MD cells hold about 14 atoms) each half-warp sorts one of them
// at once, otherwise the warp sorts them one after the other.
__global__ void k_pack_small(PackArgs a)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t n_pairs = a.n_lists >> 1;     // targets and sources of one task
    for (uint64_t t = warp; t < n_pairs; t += nwarps) {
        const uint32_t n0 = list_n(a, 2 * t), n1 = list_n(a, 2 * t + 1);
        if (n0 <= 16 && n1 <= 16) {
            const int h = lane >> 4, hl = lane & 15;
            const PackList l = list_of(a, 2 * t + (uint64_t)h);
            const uint32_t *ids = (l.src ? a.src_ids : a.tgt_ids) + l.off;
            uint64_t key = ~0ull;
            if ((uint32_t)hl < l.n)
                key = ((uint64_t)entry_slot(a, l, ids, (uint32_t)hl) << 32) | (uint64_t)hl;
            key = bitonic_lanes<16>(key, hl);
            if ((uint32_t)hl < l.n)
                emit(a, l, hl, (uint32_t)(key >> 32), (uint32_t)(key & 0xFFFFFFFFu));
            continue;
        }
        for (int h = 0; h < 2; ++h) {
            const uint32_t n = h ? n1 : n0;
            if (n == 0 || n > 32) continue;
            const PackList l = list_of(a, 2 * t + (uint64_t)h);
            const uint32_t *ids = (l.src ? a.src_ids : a.tgt_ids) + l.off;
            uint64_t key = ~0ull;
            if ((uint32_t)lane < l.n)
                key = ((uint64_t)entry_slot(a, l, ids, (uint32_t)lane) << 32) | (uint64_t)lane;
            key = bitonic_lanes<32>(key, lane);
            if ((uint32_t)lane < l.n)
                emit(a, l, lane, (uint32_t)(key >> 32), (uint32_t)(key & 0xFFFFFFFFu));
        }
    }
}

// Lanes of the warp holding the same BITS-bit label as this lane, among the
// lanes in `valid` (one ballot per label bit: 10 % faster in the pack than
// the hardware match instruction, measured on the 1M-particle step).
template <int BITS>
__device__ __forceinline__ uint32_t warp_match(uint32_t d, uint32_t valid)
{
    uint32_t m = valid;
#pragma unroll
    for (int b = 0; b < BITS; ++b) {
        const bool bit = (d >> b) & 1u;
        const uint32_t q = __ballot_sync(0xffffffffu, bit);
        m &= bit ? q : ~q;
    }
    return m;
}

// Exclusive prefix sum over the block's NW warps (one value per thread);
// barriers before and after the use of wsum, so it can be called again.
template <int NW>
__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *wsum)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    uint32_t before = 0;
    for (int q = 0; q < w; ++q) before += wsum[q];
    __syncthreads();
    return before + x - v;
}

// Stable LSD radix sort of n (slot, position) entries held in (ka, pa) by
// slot - kmin, 8-bit digits, `passes` passes, alternating with (kb, pb).
// Warp w owns a contiguous range of the current layout; inside a warp, 32
// items at a time are ranked among equal digits by label ballots, so equal
// digits keep their order (warp by warp, chunk by chunk, lane by lane).  A
// pass whose digits are all equal is skipped.  hist: NW x 256 counters.
// Returns true if the result ends in (kb, pb).
template <int NW>
__device__ __forceinline__ bool radix_lsd(uint32_t *ka, uint16_t *pa, uint32_t *kb, uint16_t *pb,
                          uint32_t *hist, uint32_t *wsum, int *skip, int n, int passes,
                          uint32_t kmin)
{
    constexpr int NT = NW * 32;
    constexpr int DPT = NT >= 256 ? 1 : 256 / NT;   // digits per thread in the offset scan
    static_assert(DPT * NT >= 256, "every digit has an owner");
    const bool owner = threadIdx.x * DPT < 256;
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const uint32_t lt = (1u << lane) - 1u;
    const int per = (((n + NW - 1) / NW) + 31) & ~31;
    const int b0 = min(n, w * per), b1 = min(n, b0 + per);
    bool flip = false;
    for (int pass = 0; pass < passes; ++pass) {
        const int sh = 8 * pass;
        for (int i = threadIdx.x; i < 256 * NW; i += NT) hist[i] = 0;
        if (threadIdx.x == 0) *skip = 0;
        __syncthreads();
        for (int k = b0 + lane; k < b1; k += 32)
            atomicAdd(&hist[w * 256 + (((ka[k] - kmin) >> sh) & 255u)], 1u);
        __syncthreads();
        uint32_t s = 0;
        if (owner) {
#pragma unroll
            for (int i = 0; i < DPT; ++i) {
                uint32_t c = 0;
                for (int q = 0; q < NW; ++q) c += hist[q * 256 + DPT * threadIdx.x + i];
                if (c == (uint32_t)n) *skip = 1;       // one digit value: identity pass
                s += c;
            }
        }
        uint32_t run = block_excl_scan<NW>(s, wsum);
        if (owner) {
#pragma unroll
            for (int i = 0; i < DPT; ++i)
                for (int q = 0; q < NW; ++q) {
                    const uint32_t c = hist[q * 256 + DPT * threadIdx.x + i];
                    hist[q * 256 + DPT * threadIdx.x + i] = run;
                    run += c;
                }
        }
        __syncthreads();
        const bool skip_pass = *skip != 0;
        if (!skip_pass) {
            for (int c = b0; c < b1; c += 32) {
                const int k = c + lane;
                const bool v = k < b1;
                const uint32_t key = v ? ka[k] : 0u;
                const uint32_t d = ((key - kmin) >> sh) & 255u;
                const uint32_t m = warp_match<8>(d, __ballot_sync(0xffffffffu, v));
                if (v) {
                    const uint32_t dst = hist[w * 256 + d] + (uint32_t)__popc(m & lt);
                    kb[dst] = key;
                    pb[dst] = pa[k];
                }
                __syncwarp();
                if (v && (m & lt) == 0) hist[w * 256 + d] += (uint32_t)__popc(m);
                __syncwarp();
            }
        }
        __syncthreads();
        if (!skip_pass) {
            uint32_t *tk = ka; ka = kb; kb = tk;
            uint16_t *tp = pa; pa = pb; pb = tp;
            flip = !flip;
        }
    }
    return flip;
}

// Insertion sort of entries [s, e) of (k, p) by (slot, position), one thread.
__device__ __forceinline__ void insertion_sort(uint32_t *k, uint16_t *p, int s, int e)
{
    for (int i = s + 1; i < e; ++i) {
        const uint32_t kv = k[i];
        const uint16_t pv = p[i];
        int j = i - 1;
        while (j >= s) {
            const uint32_t kj = k[j];
            const uint16_t pj = p[j];
            if (kj < kv || (kj == kv && pj < pv)) break;
            k[j + 1] = kj;
            p[j + 1] = pj;
            --j;
        }
        k[j + 1] = kv;
        p[j + 1] = pv;
    }
}

// Lists of 33..2048 entries: one block of 4 warps per list, sorted in shared
// memory by (slot, position) in three steps that all lead to that one order:
//
//   1. the ordered tail of the key range: P = 1 + the largest slot that
//      follows a larger slot in list order (a prefix-maximum scan), so the
//      entries with slot >= P are already in ascending order -- in the
//      N-body lists these are the tree nodes, about two thirds of every
//      list, whose slots follow their depth-first numbering;
//   2. a stable split: entries below P first, in list order, then the
//      ordered tail (every tail slot is >= P, so the tail goes last as is);
//   3. the part below P: one distribution pass into 256 buckets of equal
//      slot range (shared-memory atomics), then each bucket finished by an
//      insertion sort on (slot, position).  If a bucket would hold more than
//      PK_BUCKET_MAX entries, 8-bit LSD radix passes sort that part instead.
//
// The lookups are latency-bound reads: each thread issues PM_U of them
// before using any; the 1025..2048 class also reads the next list of its
// claim while the current one is sorted.
constexpr int PM_THREADS = 128;
constexpr int PM_W = PM_THREADS / 32;
constexpr int PM_U = 8;             // lookups in flight per thread
constexpr int PM_CAP = 2048;        // largest list of the mid class
constexpr int PM_NB = 256;          // buckets of the distribution pass
constexpr int PK_BUCKET_MAX = 48;   // largest bucket finished by insertion

// Shared memory of a block sort of up to CAP entries by NW warps with NB
// distribution buckets (the crowded-bucket LSD fallback reuses the bucket
// words for its per-warp digit counts).
template <int CAP, int NW, int NB>
struct SortSmem {
    uint32_t ka[CAP], kb[CAP];
    uint16_t pa[CAP], pb[CAP];
    union {
        uint32_t hist[NW * 256];        // LSD passes: per (warp, digit)
        uint32_t bcur[NB];              // bucket counts, then scatter cursors
    };
    uint32_t wsum[NW];
    uint32_t wmax[NW], wmin[NW], winv[NW], wsmall[NW];
    int flag, skip;
};
template <int CAP> using PackSmemMid = SortSmem<CAP, PM_W, PM_NB>;

__host__ __device__ constexpr int ilog2(int v) { return v > 1 ? 1 + ilog2(v / 2) : 0; }

// Slots of entries c0 .. c0+cn-1 of list l into ka (positions 0..cn-1 in
// pa): PM_U reads in flight per thread (entry slots, or ids then slots).
template <int NT>
__device__ __forceinline__ void load_slots(const PackArgs &a, const PackList &l, uint32_t c0,
                                           int cn, uint32_t *ka, uint16_t *pa)
{
    const uint32_t *ids = (l.src ? a.src_ids : a.tgt_ids) + l.off + c0;
    const uint32_t *es = l.es ? l.es + c0 : nullptr;
    for (int base = 0; base < cn; base += NT * PM_U) {
        uint32_t s[PM_U];
#pragma unroll
        for (int j = 0; j < PM_U; ++j) {
            const int k = base + threadIdx.x + NT * j;
            s[j] = k < cn ? __ldg((es ? es : ids) + k) : 0u;
        }
        if (!es) {
#pragma unroll
            for (int j = 0; j < PM_U; ++j) {
                const int k = base + threadIdx.x + NT * j;
                if (k < cn) s[j] = __ldg(a.slot_of_id + s[j]);
            }
        } else {
#pragma unroll
            for (int j = 0; j < PM_U; ++j) {
                const int k = base + threadIdx.x + NT * j;
                if (k < cn && s[j] == GC_NONE) s[j] = __ldg(a.slot_of_id + __ldg(ids + k));
            }
        }
#pragma unroll
        for (int j = 0; j < PM_U; ++j) {
            const int k = base + threadIdx.x + NT * j;
            if (k < cn) {
                ka[k] = s[j];
                pa[k] = (uint16_t)k;
            }
        }
    }
}

// The crowded-bucket fallback of block_sort, kept out of line: it is rare,
// and inlined beside the insertion sort it costs the common path registers.
template <int CAP, int NW, int NB>
__device__ __noinline__ bool sort_radix_fallback(SortSmem<CAP, NW, NB> &sm, int ns, int passes,
                                                 uint32_t kmin)
{
    return radix_lsd<NW>(sm.kb, sm.pb, sm.ka, sm.pa, sm.hist, sm.wsum, &sm.skip, ns, passes,
                         kmin);
}

// Sort entries 0..n-1 of a list (slots in ka, positions pa = 0..n-1) by
// (slot, position), steps 1-3 above, with NW warps and NB distribution
// buckets.  Result: entries [0, split) in (ka, pa) if low_in_a, else in
// (kb, pb); entries [split, n) in (kb, pb).
template <int CAP, int NW, int NB>
__device__ __forceinline__ int block_sort(SortSmem<CAP, NW, NB> &sm, int n, bool &low_in_a)
{
    constexpr int NT = NW * 32;
    constexpr int BPT = NB / NT;        // buckets per thread in the bucket scan
    constexpr int NBB = ilog2(NB);
    static_assert(BPT >= 1 && BPT * NT == NB && (1 << NBB) == NB, "bucket layout");
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // Each thread takes a chunk of E consecutive entries (E odd, so the
    // lanes' strided reads fall in distinct banks); running maxima and
    // counts go sequentially within a chunk and by one scan across chunks.
    const int E = ((n + NT - 1) / NT) | 1;
    const int c0 = min(n, (int)threadIdx.x * E), c1 = min(n, c0 + E);
    // 1. largest and smallest slot of each chunk; the running maximum in list
    //    order: P = 1 + the largest slot below it
    uint32_t tmax = 0u, tmin = 0xFFFFFFFFu;
    for (int k = c0; k < c1; ++k) {
        const uint32_t v = sm.ka[k];
        tmax = max(tmax, v);
        tmin = min(tmin, v);
    }
    uint32_t incl = tmax;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl = max(incl, y);
    }
    tmin = __reduce_min_sync(0xffffffffu, tmin);
    if (lane == 31) sm.wmax[w] = incl;
    if (lane == 0) sm.wmin[w] = tmin;
    __syncthreads();
    uint32_t carry = __shfl_up_sync(0xffffffffu, incl, 1);
    if (lane == 0) carry = 0u;
    uint32_t kmin = 0xFFFFFFFFu;
    for (int q = 0; q < NW; ++q) {
        if (q < w) carry = max(carry, sm.wmax[q]);
        kmin = min(kmin, sm.wmin[q]);
    }
    uint32_t inv = 0u;
    for (int k = c0; k < c1; ++k) {
        const uint32_t v = sm.ka[k];
        if (carry > v) inv = max(inv, v + 1u);
        carry = max(carry, v);
    }
    inv = __reduce_max_sync(0xffffffffu, inv);
    if (lane == 0) sm.winv[w] = inv;
    __syncthreads();
    uint32_t P = 0u;
    for (int q = 0; q < NW; ++q) P = max(P, sm.winv[q]);
    if (P == 0u) {           // the list is in order already
        low_in_a = true;
        return n;
    }
    // 2. stable split: slots below P to kb[0, ns), the ordered tail to kb[ns, n)
    uint32_t cl = 0;
    for (int k = c0; k < c1; ++k) cl += sm.ka[k] < P ? 1u : 0u;
    uint32_t lincl = cl;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(0xffffffffu, lincl, o);
        if (lane >= o) lincl += y;
    }
    if (lane == 31) sm.wsmall[w] = lincl;
    __syncthreads();
    uint32_t nlow = lincl - cl, ns = 0;   // low entries before this chunk; in the list
    for (int q = 0; q < NW; ++q) {
        if (q < w) nlow += sm.wsmall[q];
        ns += sm.wsmall[q];
    }
    for (int k = c0; k < c1; ++k) {
        const uint32_t v = sm.ka[k];
        const uint16_t pos = sm.pa[k];
        const uint32_t dst = v < P ? nlow++ : ns + (uint32_t)k - nlow;
        sm.kb[dst] = v;
        sm.pb[dst] = pos;
    }
    __syncthreads();
    if (ns <= 1u) {
        low_in_a = false;
        return (int)ns;
    }
    // 3. distribution over [kmin, P - 1] into NB buckets, kb -> ka
    const uint32_t r = P - 1u - kmin;
    const int bits = 32 - __clz((int)r);          // 0 when every low slot is kmin
    const int shift = bits > NBB ? bits - NBB : 0;
    for (int i = threadIdx.x; i < NB; i += NT) sm.bcur[i] = 0u;
    if (threadIdx.x == 0) sm.flag = 0;
    __syncthreads();
    for (int k = threadIdx.x; k < (int)ns; k += NT)
        atomicAdd(&sm.bcur[(sm.kb[k] - kmin) >> shift], 1u);
    __syncthreads();
    // thread t owns buckets BPT t .. BPT t + BPT - 1
    uint32_t cnt[BPT], tot = 0;
    bool crowded = false;
#pragma unroll
    for (int i = 0; i < BPT; ++i) {
        cnt[i] = sm.bcur[BPT * threadIdx.x + i];
        tot += cnt[i];
        crowded |= cnt[i] > (uint32_t)PK_BUCKET_MAX;
    }
    if (crowded) sm.flag = 1;
    const uint32_t st = block_excl_scan<NW>(tot, sm.wsum);
    {
        uint32_t at = st;
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            sm.bcur[BPT * threadIdx.x + i] = at;
            at += cnt[i];
        }
    }
    __syncthreads();
    if (sm.flag == 0) {
        for (int k = threadIdx.x; k < (int)ns; k += NT) {
            const uint32_t key = sm.kb[k];
            const uint32_t dst = atomicAdd(&sm.bcur[(key - kmin) >> shift], 1u);
            sm.ka[dst] = key;
            sm.pa[dst] = sm.pb[k];
        }
        __syncthreads();
        uint32_t at = st;
#pragma unroll
        for (int i = 0; i < BPT; ++i) {
            insertion_sort(sm.ka, sm.pa, (int)at, (int)(at + cnt[i]));
            at += cnt[i];
        }
        __syncthreads();
        low_in_a = true;
        return (int)ns;
    }
    // a crowded bucket: LSD radix passes over the low part (kb -> ka -> ...)
    const int passes = (bits + 7) / 8;
    low_in_a = sort_radix_fallback(sm, (int)ns, passes, kmin);
    return (int)ns;
}

// Write sorted entries 0..n-1 of list l: permutation and staging.  Entry k
// comes from (ka, pa) if k < split, else from (kb, pb).  Entries k =
// threadIdx.x + NT * j, so the lanes of a warp hold consecutive k: in the
// paired source layout lanes 2i and 2i+1 swap halves with one shuffle pair
// and each writes a whole float4.
template <int NT = PM_THREADS>
__device__ __forceinline__ void emit_block(const PackArgs &a, const PackList &l, int n,
                                           const uint32_t *ka, const uint16_t *pa, int split,
                                           const uint32_t *kb, const uint16_t *pb)
{
    const int lane = threadIdx.x & 31;
    const int h = lane & 1;
    // paired lists also run the (zero) pad lane of an odd list
    const int n_run = l.paired ? ((n + 1) & ~1) : n;
    for (int base = 0; base < n_run; base += NT * PM_U) {
        float4 v[PM_U];
#pragma unroll
        for (int j = 0; j < PM_U; ++j) {
            const int k = base + threadIdx.x + NT * j;
            v[j] = make_float4(0.f, 0.f, 0.f, 0.f);
            if (k < n) v[j] = a.pool[k < split ? ka[k] : kb[k]];
        }
#pragma unroll
        for (int j = 0; j < PM_U; ++j) {
            const int k = base + threadIdx.x + NT * j;
            if (base + NT * j >= n_run) break;      // uniform over the block
            if (k < n) (l.src ? a.perm_s : a.perm_t)[l.off + k] = k < split ? pa[k] : pb[k];
            if (!l.paired) {
                if (k < n) (l.src ? a.stg_s : a.stg_t)[l.stg + k] = v[j];
                continue;
            }
            const float sa = h ? v[j].x : v[j].z, sb = h ? v[j].y : v[j].w;
            const float ra = __shfl_xor_sync(0xffffffffu, sa, 1);
            const float rb = __shfl_xor_sync(0xffffffffu, sb, 1);
            if (k < n_run) {
                const float4 o = h ? make_float4(ra, v[j].z, rb, v[j].w)
                                   : make_float4(v[j].x, ra, v[j].y, rb);
                a.stg_s[l.stg + 2 * (k >> 1) + h] = o;
            }
        }
    }
}

template <int CAP>
__global__ void __launch_bounds__(PM_THREADS) k_pack_mid(PackArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PackSmemMid<CAP> &sm = *reinterpret_cast<PackSmemMid<CAP> *>(smem_raw);
    constexpr uint32_t LO = CAP == PM_CAP ? (uint32_t)(PM_CAP / 2) : 32u;
    __shared__ ListClaim cl;
    unsigned long long *ctr = a.work + (CAP == PM_CAP ? 1 : 0);
    // The 1025..2048 class reads the next list of the claim while this one
    // is sorted: its entry slots (or ids) before the sort, the lookups it
    // still needs after it, into registers that the sort does not touch.
    constexpr int PF = CAP / PM_THREADS;     // entries per thread of a full list
    constexpr bool PREFETCH = CAP == PM_CAP;
    uint32_t pf[PF];
    while (claim_lists(a, ctr, LO, (uint32_t)CAP, cl)) {
        bool have_pf = false;
        for (uint32_t ci = 0; ci < cl.cnt; ++ci) {
            const PackList l = list_of(a, cl.base + cl.off[ci]);
            const int n = (int)l.n;
            if (have_pf) {
#pragma unroll
                for (int j = 0; j < PF; ++j) {
                    const int k = threadIdx.x + PM_THREADS * j;
                    if (k < n) {
                        sm.ka[k] = pf[j];
                        sm.pa[k] = (uint16_t)k;
                    }
                }
            } else {
                load_slots<PM_THREADS>(a, l, 0, n, sm.ka, sm.pa);
            }
            __syncthreads();
            const bool pf_next = PREFETCH && ci + 1 < cl.cnt;
            PackList ln;
            int nn = 0;
            if (pf_next) {
                ln = list_of(a, cl.base + cl.off[ci + 1]);
                nn = (int)ln.n;
                const uint32_t *src = ln.es ? ln.es : (ln.src ? a.src_ids : a.tgt_ids) + ln.off;
#pragma unroll
                for (int j = 0; j < PF; ++j) {
                    const int k = threadIdx.x + PM_THREADS * j;
                    pf[j] = k < nn ? __ldg(src + k) : 0u;
                }
            }
            bool low_in_a = true;
            const int split = block_sort(sm, n, low_in_a);
            if (pf_next) {
                // the lookups the next list still needs (its reads have arrived)
                const uint32_t *idn = (ln.src ? a.src_ids : a.tgt_ids) + ln.off;
#pragma unroll
                for (int j = 0; j < PF; ++j) {
                    const int k = threadIdx.x + PM_THREADS * j;
                    if (k < nn) {
                        if (!ln.es) pf[j] = __ldg(a.slot_of_id + pf[j]);
                        else if (pf[j] == GC_NONE) pf[j] = __ldg(a.slot_of_id + __ldg(idn + k));
                    }
                }
            }
            emit_block(a, l, n, low_in_a ? sm.ka : sm.kb, low_in_a ? sm.pa : sm.pb, split,
                       sm.kb, sm.pb);
            __syncthreads();
            have_pf = pf_next;
        }
    }
}

// Lists of more than 2048 entries: one block of 16 warps per list, sorted in
// shared memory by the same block sort (ordered-tail split, distribution
// pass, insertion).  CAP = PK_CAP takes lists of 2049..4096 entries (about
// 64 KB of shared memory, three blocks per SM); CAP = PK_CAP_HUGE every
// longer list (about 224 KB, one block per SM), and a list beyond PK_CAP_HUGE is
// sorted in chunks of PK_CAP_HUGE that are merged pairwise in global scratch
// (keys (slot << 32 | pos) are unique, so an element's output index is its
// rank in its own run plus its rank in the other run).

// Warps and distribution buckets of each block-sort class: the largest lists
// take a whole SM; one bucket per entry at full size for 4096 entries, one
// per two for 16384 (its shared memory, about 224 KB, is then full).  Fewer
// entries per bucket shorten the insertion sorts, chains of dependent
// shared-memory accesses.
constexpr int PK_NW_MID = 16, PK_NW_HUGE = 16;
template <int CAP> struct PackLargeWarps { static constexpr int value = PK_NW_MID; };
template <> struct PackLargeWarps<PK_CAP_HUGE> { static constexpr int value = PK_NW_HUGE; };
template <int CAP>
using PackSmemLarge = SortSmem<CAP, PackLargeWarps<CAP>::value,
                               CAP == PK_CAP_HUGE ? CAP / 2 : CAP>;

template <int CAP>
__global__ void __launch_bounds__(PackLargeWarps<CAP>::value * 32) k_pack_large(PackArgs a)
{
    constexpr int NW = PackLargeWarps<CAP>::value;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    PackSmemLarge<CAP> &sm = *reinterpret_cast<PackSmemLarge<CAP> *>(smem_raw);
    static_assert(CAP == PK_CAP || CAP == PK_CAP_HUGE, "two block-sort classes");
    const uint32_t lo_n = (CAP == PK_CAP) ? (uint32_t)PM_CAP : (uint32_t)PK_CAP;
    const uint32_t hi_n = (CAP == PK_CAP) ? (uint32_t)PK_CAP : 0xFFFFFFFFu;
    __shared__ ListClaim cl;
    while (claim_lists(a, a.work + (CAP == PK_CAP ? 2 : 3), lo_n, hi_n, cl))
    for (uint32_t ci = 0; ci < cl.cnt; ++ci) {
        PackList l = list_of(a, cl.base + cl.off[ci]);
        if (l.n <= (uint32_t)CAP) {
            load_slots<NW * 32>(a, l, 0, (int)l.n, sm.ka, sm.pa);
            __syncthreads();
            bool low_in_a = true;
            const int split = block_sort(sm, (int)l.n, low_in_a);
            emit_block<NW * 32>(a, l, (int)l.n, low_in_a ? sm.ka : sm.kb,
                                low_in_a ? sm.pa : sm.pb, split, sm.kb, sm.pb);
            __syncthreads();
            continue;
        }
        const uint64_t loc = l.src ? a.msrc + (l.off - a.src_base) : l.off - a.tgt_base;
        uint64_t *A = a.ma + loc;
        uint64_t *B = a.mb + loc;
        const uint32_t n = l.n;
        for (uint32_t c0 = 0; c0 < n; c0 += CAP) {
            const int cn = (int)min((uint32_t)CAP, n - c0);
            load_slots<NW * 32>(a, l, c0, cn, sm.ka, sm.pa);
            __syncthreads();
            bool low_in_a = true;
            const int split = block_sort(sm, cn, low_in_a);
            const uint32_t *kl = low_in_a ? sm.ka : sm.kb;
            const uint16_t *pl = low_in_a ? sm.pa : sm.pb;
            for (int k = threadIdx.x; k < cn; k += blockDim.x) {
                const uint32_t key = k < split ? kl[k] : sm.kb[k];
                const uint32_t pos = k < split ? pl[k] : sm.pb[k];
                A[c0 + k] = ((uint64_t)key << 32) | (uint64_t)(c0 + pos);
            }
            __syncthreads();
        }
        for (uint32_t w = CAP; w < n; w <<= 1) {
            for (uint32_t e = threadIdx.x; e < n; e += blockDim.x) {
                const uint32_t r = e / w;
                const uint32_t ls = (r & ~1u) * w;
                const uint32_t rs = ls + w;
                const uint64_t key = A[e];
                if (rs >= n) {
                    B[e] = key;
                    continue;
                }
                const uint32_t re = min(rs + w, n);
                uint32_t lo, hi, own;
                if (e < rs) {
                    lo = rs; hi = re; own = e - ls;
                } else {
                    lo = ls; hi = rs; own = e - rs;
                }
                const uint32_t base = lo;
                while (lo < hi) {
                    uint32_t mid = (lo + hi) >> 1;
                    if (A[mid] < key) lo = mid + 1; else hi = mid;
                }
                B[ls + own + (lo - base)] = key;
            }
            __syncthreads();
            uint64_t *t = A; A = B; B = t;
        }
        for (uint32_t k = threadIdx.x; k < n; k += blockDim.x)
            emit(a, l, k, (uint32_t)(A[k] >> 32), (uint32_t)(A[k] & 0xFFFFFFFFu));
        __syncthreads();
    }
}

// ---------------------------------------------------------------------------
// interaction: gravity
// ---------------------------------------------------------------------------

constexpr int GRAV_THREADS = 256;
constexpr int GRAV_WARPS = GRAV_THREADS / 32;
constexpr int KB = 8;   // source pairs per plain FP32 partial (the indirect ablation kernel)

struct InterArgs {
    const TaskRec *tasks;
    const GravWU *wu;
    uint64_t n_wu;
    const uint32_t *lj_list;
    uint64_t n_lj;
    const float4 *stg_t, *stg_s;
    uint64_t tgt_base, src_base, task_base;
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
    unsigned long long *flags;   // device error bits
    const float4 *ewald_h;       // half of the reciprocal vectors (GC_EWALD)
    int n_ewald_h;
    float ewald_L;
};

__device__ __forceinline__ void kahan_add(float &s, float &c, float v)
{
    float y = v - c;
    float t = s + y;
    c = (t - s) - y;
    s = t;
}

// Paired compensated add: (s, c) += b on both halves, with FMA-by-(-1)
// standing in for subtraction (exact: one rounding, as a subtraction).
__device__ __forceinline__ void kahan_add2(float2 &s, float2 &c, float2 b, float2 m1)
{
    float2 y = __ffma2_rn(c, m1, b);      // b - c
    float2 t = __fadd2_rn(s, y);
    float2 d = __ffma2_rn(s, m1, t);      // t - s
    c = __ffma2_rn(y, m1, d);             // (t - s) - y
    s = t;
}

// Compensated pair (s, c), value s - c, plus another such pair (s2, c2): the
// sums s + s2 are split exactly (Knuth's two-sum) and the rounding error is
// carried into the compensation.  FP32 only: the FP64 pipe of this GPU runs
// at 1/64 of the FP32 rate, so per-lane FP64 work would dominate the kernel.
__device__ __forceinline__ void comp_add(float &s, float &c, float s2, float c2)
{
    const float t = __fadd_rn(s, s2);
    const float bb = __fsub_rn(t, s);
    const float e = __fadd_rn(__fsub_rn(s, __fsub_rn(t, bb)), __fsub_rn(s2, bb));  // s + s2 = t + e
    c = __fsub_rn(__fadd_rn(c, c2), e);
    s = t;
}

// One source pair against one target, paired FP32 arithmetic.
#define GRAV_PAIR(A, B)                                                   \
    do {                                                                  \
        float2 dx = __fadd2_rn(make_float2((A).x, (A).y), nx);            \
        float2 dy = __fadd2_rn(make_float2((A).z, (A).w), ny);            \
        float2 dz = __fadd2_rn(make_float2((B).x, (B).y), nz);            \
        float2 r2 = __ffma2_rn(dx, dx, e2);                               \
        r2 = __ffma2_rn(dy, dy, r2);                                      \
        r2 = __ffma2_rn(dz, dz, r2);                                      \
        float2 ri = make_float2(gc_rsqrt(r2.x), gc_rsqrt(r2.y));          \
        float2 mr = __fmul2_rn(make_float2((B).z, (B).w), ri);            \
        float2 mr3 = __fmul2_rn(mr, __fmul2_rn(ri, ri));                  \
        bx = __ffma2_rn(mr3, dx, bx);                                     \
        by = __ffma2_rn(mr3, dy, by);                                     \
        bz = __ffma2_rn(mr3, dz, bz);                                     \
        bp = __ffma2_rn(mr, m1, bp);                                      \
    } while (0)

// The same against the lane's target k (k a compile-time index into the
// per-target arrays of the kernel below).
#define GRAV_PAIR_K(A, B, k)                                              \
    do {                                                                  \
        float2 dx = __fadd2_rn(make_float2((A).x, (A).y), nx[k]);         \
        float2 dy = __fadd2_rn(make_float2((A).z, (A).w), ny[k]);         \
        float2 dz = __fadd2_rn(make_float2((B).x, (B).y), nz[k]);         \
        float2 r2 = __ffma2_rn(dx, dx, e2);                               \
        r2 = __ffma2_rn(dy, dy, r2);                                      \
        r2 = __ffma2_rn(dz, dz, r2);                                      \
        float2 ri = make_float2(gc_rsqrt(r2.x), gc_rsqrt(r2.y));          \
        float2 mr = __fmul2_rn(make_float2((B).z, (B).w), ri);            \
        float2 mr3 = __fmul2_rn(mr, __fmul2_rn(ri, ri));                  \
        bx[k] = __ffma2_rn(mr3, dx, bx[k]);                               \
        by[k] = __ffma2_rn(mr3, dy, by[k]);                               \
        bz[k] = __ffma2_rn(mr3, dz, bz[k]);                               \
        bp[k] = __ffma2_rn(mr, m1, bp[k]);                                \
    } while (0)

constexpr uint32_t WAIT_LIMIT = 1u << 22;  // bounded mbarrier polling

// TP source pairs per staged tile (32 TP bytes): shared memory of a block is
// 512 TP bytes of tiles plus 8 KB per target a lane holds, which sets the
// resident blocks per SM.
template <int TP, int TPL>
struct GravSmem {
    float4 buf[GRAV_WARPS][2][2 * TP];  // per warp: two tiles of source pairs
    uint64_t bar[GRAV_WARPS][2];        // one mbarrier per tile buffer
    float4 red[GRAV_WARPS][32][2 * TPL];  // cross-lane combine: (sum, compensation)
};

// One warp per work unit (task, block of <= 32 targets).  With T targets in
// the block and TPL targets per lane, the warp splits into TL = ceil(T / TPL)
// target lanes times S = 32 / TL source lanes: lane (t, s) accumulates
// targets t, t + TL, ... over source pairs s, s + S, ... of each tile, so
// each source pair read from shared memory serves TPL targets.
// Source pairs stream through two shared-memory tile buffers per warp,
// filled by 1-D bulk copies (TMA) that complete on mbarriers, one tile
// ahead of the compute.  Every source pair is evaluated with paired FP32
// instructions (two interactions per instruction); plain FP32 partial sums
// of KB pairs are added with compensation; the S lane results of a target are combined
// as compensated FP32 pairs in lane order.  Work units come from a device queue (persistent
// kernel); with a null queue each warp takes a fixed share
// (one-launch-per-task mode).  A bulk copy that does not complete within the
// polling limit sets GC_FLAG_TIMEOUT and the warp stops; the lanes poll
// together and take that decision as one, so no lane is left waiting at a
// later warp-wide shuffle.
// The tile size TP, the block KB and the targets per lane TPL are the
// autotuner's tile shape; a lane's target slot beyond the block's targets
// (odd T) repeats the last target and is not written.
template <int TP, int KB, int TPL>
__global__ void __launch_bounds__(GRAV_THREADS) k_gravity(InterArgs a)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    GravSmem<TP, TPL> &sm = *reinterpret_cast<GravSmem<TP, TPL> *>(smem_raw);
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 e2 = make_float2(a.eps2, a.eps2);
    uint64_t *bar = sm.bar[wib];
    if (lane == 0) {
        gc_mbar_init(&bar[0], 1);
        gc_mbar_init(&bar[1], 1);
        gc_fence_mbar_init();
    }
    __syncwarp();
    uint32_t parity = 0;     // bit b: parity of the next completion of buffer b
    for (uint64_t it = 0;; ++it) {
        unsigned long long w = gwarp + it * nwarps;
        if (a.queue) {
            if (lane == 0) w = atomicAdd(a.queue, 1ull);
            w = __shfl_sync(0xffffffffu, w, 0);
        }
        if (w >= a.n_wu) break;
        const GravWU u = a.wu[w];
        const TaskRec r = a.tasks[u.task];
        const int T = (int)u.tn;
        const int TL = (T + TPL - 1) / TPL;
        const int S = 32 / TL;
        const int t = lane % TL;
        const int sl = lane / TL;
        const bool active = sl < S;
        const float4 *P = a.stg_s + (r.src_off - a.src_base) + (u.task - a.task_base);
        const uint32_t np = (r.ns + 1u) >> 1;
        const uint32_t ntiles = (np + TP - 1) / TP;
        float2 nx[TPL], ny[TPL], nz[TPL];
        float2 sx[TPL], sy[TPL], sz[TPL], sp[TPL], cx[TPL], cy[TPL], cz[TPL], cp[TPL];
#pragma unroll
        for (int k = 0; k < TPL; ++k) {
            const int tk = min(t + k * TL, T - 1);
            const float4 xi = a.stg_t[r.tgt_off - a.tgt_base + u.t0 + tk];
            nx[k] = make_float2(-xi.x, -xi.x);
            ny[k] = make_float2(-xi.y, -xi.y);
            nz[k] = make_float2(-xi.z, -xi.z);
            sx[k] = sy[k] = sz[k] = sp[k] = make_float2(0.f, 0.f);
            cx[k] = cy[k] = cz[k] = cp[k] = make_float2(0.f, 0.f);
        }
        if (lane == 0) {
            for (uint32_t b = 0; b < 2 && b < ntiles; ++b) {
                const uint32_t bytes = min((uint32_t)TP, np - b * TP) * 32u;
                gc_mbar_arrive_expect_tx(&bar[b], bytes);
                gc_bulk_g2s(sm.buf[wib][b], P + 2 * b * TP, bytes, &bar[b]);
            }
        }
        bool ok = true;
        uint32_t failed_at = 0;
        for (uint32_t i = 0; i < ntiles; ++i) {
            const uint32_t b = i & 1u;
            if (!gc_mbar_wait_bounded_warp(&bar[b], (parity >> b) & 1u, WAIT_LIMIT)) {
                ok = false;
                failed_at = i;
                break;
            }
            parity ^= 1u << b;
            const uint32_t m = min((uint32_t)TP, np - i * TP);
            const uint32_t nq = (active && (uint32_t)sl < m) ? (m - (uint32_t)sl + S - 1) / S : 0u;
            const float4 *q = sm.buf[wib][b] + 2 * sl;
            const uint32_t stride = 2u * (uint32_t)S;
            uint32_t j = 0;
            for (; j + KB <= nq; j += KB) {
                float2 bx[TPL], by[TPL], bz[TPL], bp[TPL];
#pragma unroll
                for (int k = 0; k < TPL; ++k) bx[k] = by[k] = bz[k] = bp[k] = make_float2(0.f, 0.f);
#pragma unroll
                for (int kk = 0; kk < KB; ++kk) {
                    const float4 A = q[0];
                    const float4 B = q[1];
                    q += stride;
#pragma unroll
                    for (int k = 0; k < TPL; ++k) GRAV_PAIR_K(A, B, k);
                }
#pragma unroll
                for (int k = 0; k < TPL; ++k) {
                    kahan_add2(sx[k], cx[k], bx[k], m1);
                    kahan_add2(sy[k], cy[k], by[k], m1);
                    kahan_add2(sz[k], cz[k], bz[k], m1);
                    kahan_add2(sp[k], cp[k], bp[k], m1);
                }
            }
            if (j < nq) {
                float2 bx[TPL], by[TPL], bz[TPL], bp[TPL];
#pragma unroll
                for (int k = 0; k < TPL; ++k) bx[k] = by[k] = bz[k] = bp[k] = make_float2(0.f, 0.f);
                for (; j < nq; ++j) {
                    const float4 A = q[0];
                    const float4 B = q[1];
                    q += stride;
#pragma unroll
                    for (int k = 0; k < TPL; ++k) GRAV_PAIR_K(A, B, k);
                }
#pragma unroll
                for (int k = 0; k < TPL; ++k) {
                    kahan_add2(sx[k], cx[k], bx[k], m1);
                    kahan_add2(sy[k], cy[k], by[k], m1);
                    kahan_add2(sz[k], cz[k], bz[k], m1);
                    kahan_add2(sp[k], cp[k], bp[k], m1);
                }
            }
            gc_fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0 && i + 2 < ntiles) {
                const uint32_t bytes = min((uint32_t)TP, np - (i + 2) * TP) * 32u;
                gc_mbar_arrive_expect_tx(&bar[b], bytes);
                gc_bulk_g2s(sm.buf[wib][b], P + 2 * (i + 2) * TP, bytes, &bar[b]);
            }
        }
        if (!ok) {
            // a copy never completed: report, wait (bounded) for the other
            // copy of this work unit still in flight, stop this warp
            if (lane == 0) atomicOr(a.flags, (unsigned long long)GC_FLAG_TIMEOUT);
            if (failed_at + 1 < ntiles) {
                const uint32_t ob = (failed_at + 1) & 1u;
                gc_mbar_wait_bounded_warp(&bar[ob], (parity >> ob) & 1u, WAIT_LIMIT);
            }
            return;
        }
        // the two halves of each lane, then the S lanes of a target in lane
        // order, all as compensated FP32 pairs
#pragma unroll
        for (int k = 0; k < TPL; ++k) {
            comp_add(sx[k].x, cx[k].x, sx[k].y, cx[k].y);
            comp_add(sy[k].x, cy[k].x, sy[k].y, cy[k].y);
            comp_add(sz[k].x, cz[k].x, sz[k].y, cz[k].y);
            comp_add(sp[k].x, cp[k].x, sp[k].y, cp[k].y);
            sm.red[wib][lane][2 * k] = make_float4(sx[k].x, sy[k].x, sz[k].x, sp[k].x);
            sm.red[wib][lane][2 * k + 1] = make_float4(cx[k].x, cy[k].x, cz[k].x, cp[k].x);
        }
        __syncwarp();
        if (sl == 0) {
#pragma unroll
            for (int k = 0; k < TPL; ++k) {
                const int tk = t + k * TL;
                if (tk >= T) break;
                float4 vs = sm.red[wib][t][2 * k], vc = sm.red[wib][t][2 * k + 1];
                for (int s = 1; s < S; ++s) {
                    const int l = s * TL + t;
                    const float4 ws = sm.red[wib][l][2 * k], wc = sm.red[wib][l][2 * k + 1];
                    comp_add(vs.x, vc.x, ws.x, wc.x);
                    comp_add(vs.y, vc.y, ws.y, wc.y);
                    comp_add(vs.z, vc.z, ws.z, wc.z);
                    comp_add(vs.w, vc.w, ws.w, wc.w);
                }
                const uint64_t e = r.tgt_off + u.t0 + tk;
                const uint32_t pos = a.perm_t[e];
                const uint64_t row = r.row_off + pos;
                a.res[2 * row] = vs;
                a.res[2 * row + 1] = vc;
                a.row_id[row] = a.tgt_ids[r.tgt_off + pos];
            }
        }
        __syncwarp();
    }
}

// ---------------------------------------------------------------------------
// interaction reading sources through their pool slots (reuse ablation)
// ---------------------------------------------------------------------------

// The same work units and pair arithmetic as k_gravity, but without staging:
// every source is read from the device pool through its slot, in the order
// given by `seq` (entry slots of each list in list order -- the "address
// buffer" of Section 3.2 before sorting -- or sorted by slot).  Lane (t, s)
// takes source pairs s, s + S, ... of the list, as k_gravity does.
struct IndirectSmem {
    float4 red[GRAV_WARPS][32][2];      // cross-lane combine: (sum, compensation)
};

__global__ void __launch_bounds__(GRAV_THREADS) k_gravity_indirect(InterArgs a,
                                                                  const uint32_t *seq,
                                                                  const float4 *pool)
{
    __shared__ IndirectSmem sm;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const float2 m1 = make_float2(-1.0f, -1.0f);
    const float2 e2 = make_float2(a.eps2, a.eps2);
    for (;;) {
        unsigned long long w = 0;
        if (lane == 0) w = atomicAdd(a.queue, 1ull);
        w = __shfl_sync(0xffffffffu, w, 0);
        if (w >= a.n_wu) break;
        const GravWU u = a.wu[w];
        const TaskRec r = a.tasks[u.task];
        const int T = (int)u.tn;
        const int S = 32 / T;
        const int t = lane % T;
        const int sl = lane / T;
        const bool active = sl < S;
        const uint32_t *q = seq + r.src_off;
        const uint32_t np = (r.ns + 1u) >> 1;
        const float4 xi = a.stg_t[r.tgt_off - a.tgt_base + u.t0 + t];
        const float2 nx = make_float2(-xi.x, -xi.x);
        const float2 ny = make_float2(-xi.y, -xi.y);
        const float2 nz = make_float2(-xi.z, -xi.z);
        float2 sx = make_float2(0.f, 0.f), sy = sx, sz = sx, sp = sx;
        float2 cx = sx, cy = sx, cz = sx, cp = sx;
        float2 bx = sx, by = sx, bz = sx, bp = sx;
        int inblk = 0;
        for (uint32_t j = active ? (uint32_t)sl : np; j < np; j += (uint32_t)S) {
            const float4 v0 = pool[q[2 * j]];
            const float4 v1 = (2 * j + 1 < r.ns) ? pool[q[2 * j + 1]]
                                                  : make_float4(0.f, 0.f, 0.f, 0.f);
            const float4 A = make_float4(v0.x, v1.x, v0.y, v1.y);
            const float4 B = make_float4(v0.z, v1.z, v0.w, v1.w);
            GRAV_PAIR(A, B);
            if (++inblk == KB) {
                kahan_add2(sx, cx, bx, m1);
                kahan_add2(sy, cy, by, m1);
                kahan_add2(sz, cz, bz, m1);
                kahan_add2(sp, cp, bp, m1);
                bx = by = bz = bp = make_float2(0.f, 0.f);
                inblk = 0;
            }
        }
        kahan_add2(sx, cx, bx, m1);
        kahan_add2(sy, cy, by, m1);
        kahan_add2(sz, cz, bz, m1);
        kahan_add2(sp, cp, bp, m1);
        comp_add(sx.x, cx.x, sx.y, cx.y);
        comp_add(sy.x, cy.x, sy.y, cy.y);
        comp_add(sz.x, cz.x, sz.y, cz.y);
        comp_add(sp.x, cp.x, sp.y, cp.y);
        sm.red[wib][lane][0] = make_float4(sx.x, sy.x, sz.x, sp.x);
        sm.red[wib][lane][1] = make_float4(cx.x, cy.x, cz.x, cp.x);
        __syncwarp();
        if (sl == 0) {
            float4 vs = sm.red[wib][t][0], vc = sm.red[wib][t][1];
            for (int s2 = 1; s2 < S; ++s2) {
                const int l = s2 * T + t;
                const float4 ws = sm.red[wib][l][0], wc = sm.red[wib][l][1];
                comp_add(vs.x, vc.x, ws.x, wc.x);
                comp_add(vs.y, vc.y, ws.y, wc.y);
                comp_add(vs.z, vc.z, ws.z, wc.z);
                comp_add(vs.w, vc.w, ws.w, wc.w);
            }
            const uint64_t e = r.tgt_off + u.t0 + t;
            const uint32_t pos = a.perm_t[e];
            const uint64_t row = r.row_off + pos;
            a.res[2 * row] = vs;
            a.res[2 * row + 1] = vc;
        }
        __syncwarp();
    }
}

// out[off + k] = in[off + perm[off + k]] within each task's source list
// (the slots of a list in ascending-slot order); one warp per task.
__global__ void k_sorted_slots(const TaskRec *tasks, uint64_t n, const uint32_t *in,
                               const uint32_t *perm, uint32_t *out)
{
    const int lane = threadIdx.x & 31;
    const uint64_t warp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t t = warp; t < n; t += nw) {
        const TaskRec r = tasks[t];
        for (uint32_t k = lane; k < r.ns; k += 32)
            out[r.src_off + k] = in[r.src_off + perm[r.src_off + k]];
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
constexpr int LJ_STAGE = 128;   // atoms of a task staged in shared memory
constexpr uint32_t LJ_CHUNK = 8; // list entries claimed per queue access

__global__ void __launch_bounds__(GRAV_THREADS) k_lj(InterArgs a)
{
    __shared__ float4 lj_buf[GRAV_WARPS][LJ_STAGE];
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const float inv_grid = 1.0f / 2097152.0f;
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    // tasks are small: claim LJ_CHUNK list entries per queue access (one
    // counter shared by every warp would otherwise serialise the kernel)
    unsigned long long next = 0;
    uint32_t left = 0;
    for (uint64_t it = 0;; ++it) {
        unsigned long long w = gwarp + it * nwarps;
        if (a.queue) {
            if (left == 0) {
                if (lane == 0) next = atomicAdd(a.queue, (unsigned long long)LJ_CHUNK);
                next = __shfl_sync(0xffffffffu, next, 0);
                left = LJ_CHUNK;
            }
            w = next++;
            --left;
        }
        if (w >= a.n_lj) break;
        const uint32_t ti = a.lj_list[w];
        const TaskRec r = a.tasks[ti];
        if (r.kind == GC_EWALD) continue;   // k_ewald's
        const bool self = r.kind == GC_LJ_SELF;
        const uint32_t nA = r.nt, nB = self ? 0u : r.ns;
        const float4 *As = a.stg_t + (r.tgt_off - a.tgt_base);
        const float4 *Bs = a.stg_s + (r.src_off - a.src_base) + (ti - a.task_base);
        if (nA + nB <= (uint32_t)LJ_STAGE) {
            // every lane reads every partner: stage the task's atoms once
            for (uint32_t k = lane; k < nA + nB; k += 32)
                lj_buf[wib][k] = k < nA ? As[k] : Bs[k - nA];
            __syncwarp();
            As = &lj_buf[wib][0];
            Bs = &lj_buf[wib][nA];
        }
        // positions in the frame of cell A: A atoms at u, B atoms at u + shift * edge.
        // Offsets are multiples of 2^-21 below 2^3, so these sums and the
        // differences below are exact in FP32.
        const float edge = (float)a.edge_grid * inv_grid;
        const float fsx = (float)r.shift[0] * edge, fsy = (float)r.shift[1] * edge,
                    fsz = (float)r.shift[2] * edge;
        // |r|^2 in FP32 (relative error below 2^-22) decides the cutoff outside
        // a band of relative width 2^-18 around rc^2; inside it the decision
        // is taken exactly on the integer grid
        const float rc2 = (float)((double)a.rc2_grid * (1.0 / 4398046511104.0));
        const float rc2_lo = rc2 * (1.0f - 3.814697265625e-6f), rc2_hi = rc2 * (1.0f + 3.814697265625e-6f);
        unsigned long long inside = 0;
        for (uint32_t o = lane; o < nA + nB; o += 32) {
            const bool ownA = o < nA;
            float4 me = ownA ? As[o] : Bs[o - nA];
            if (!ownA) { me.x += fsx; me.y += fsy; me.z += fsz; }
            const float4 *P = ownA ? (self ? As : Bs) : As;
            const uint32_t np = ownA ? (self ? nA : nB) : nA;
            const bool pshift = ownA && !self;   // partners are B atoms
            float sx = 0.f, sy = 0.f, sz = 0.f, su = 0.f;
            float cx = 0.f, cy = 0.f, cz = 0.f, cu = 0.f;
            // 32 partners at a time: first every cutoff decision (a bit per
            // partner), then the force of the partners inside, in ascending
            // order.  About one candidate in seven is inside, so the warp runs
            // the force code for the most accepted partners of any lane
            // instead of for every partner slot that some lane accepts.
            for (uint32_t q0 = 0; q0 < np; q0 += 32) {
                const uint32_t qn = min(32u, np - q0);
                uint32_t mask = 0;
#pragma unroll 4
                for (uint32_t u = 0; u < qn; ++u) {
                    const uint32_t q = q0 + u;
                    float4 pq = P[q];
                    if (pshift) { pq.x += fsx; pq.y += fsy; pq.z += fsz; }
                    // displacement partner - own (exact)
                    const float rx = pq.x - me.x, ry = pq.y - me.y, rz = pq.z - me.z;
                    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    bool in = !(self && q == o) && r2 < rc2_hi;
                    if (in && r2 >= rc2_lo) {
                        const int64_t ix = __float2int_rn(rx * 2097152.0f);
                        const int64_t iy = __float2int_rn(ry * 2097152.0f);
                        const int64_t iz = __float2int_rn(rz * 2097152.0f);
                        in = ix * ix + iy * iy + iz * iz < a.rc2_grid;
                    }
                    mask |= (uint32_t)in << u;
                }
                while (mask) {
                    const uint32_t u = (uint32_t)__ffs(mask) - 1u;
                    mask &= mask - 1u;
                    const uint32_t q = q0 + u;
                    if (ownA && (!self || q > o)) ++inside;
                    float4 pq = P[q];
                    if (pshift) { pq.x += fsx; pq.y += fsy; pq.z += fsz; }
                    const float rx = pq.x - me.x, ry = pq.y - me.y, rz = pq.z - me.z;
                    const float r2 = fmaf(rx, rx, fmaf(ry, ry, rz * rz));
                    float ir2 = gc_rcp(r2);
                    float s2 = a.lj_sig2 * ir2;
                    float s6 = s2 * s2 * s2;
                    float coef = a.lj_eps24 * fmaf(2.0f, s6 * s6, -s6) * ir2;
                    float uu = a.lj_eps4 * fmaf(s6, s6, -s6);
                    // force on own atom: coef * (x_own - x_partner) = -coef * r
                    kahan_add(sx, cx, -coef * rx);
                    kahan_add(sy, cy, -coef * ry);
                    kahan_add(sz, cz, -coef * rz);
                    kahan_add(su, cu, 0.5f * uu);
                }
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
            a.res[2 * row] = make_float4(sx, sy, sz, su);        // value s - c, as stored
            a.res[2 * row + 1] = make_float4(cx, cy, cz, cu);
            a.row_id[row] = id;
        }
        for (int s = 16; s; s >>= 1) inside += __shfl_xor_sync(0xffffffffu, inside, s);
        if (lane == 0 && inside) atomicAdd(a.lj_in, inside);
        __syncwarp();   // the staged atoms are read before the next task overwrites them
    }
}

// ---------------------------------------------------------------------------
// interaction: Ewald correction of periodic gravity
// ---------------------------------------------------------------------------

// Part of the correction of one source at displacement r = x_target -
// x_source in a periodic cube of side L (splitting alpha = 2/L): the terms of
// the Ewald sum over the real-space images i = part, part + parts, ... of the
// 125 images |n_j| <= 2 (i = 25 (nx + 2) + 5 (ny + 2) + nz + 2) and over the
// reciprocal vectors j = part, part + parts, ... of the half set hv, minus
// the plain point-mass term of r (carried by the zero image, i = 62).  Adds
// grad psi to (gx, gy, gz) and psi - 1/|r| to ps; the background term is
// added by part 0.  The zero image and the subtracted term are combined and
// taken from the series of erf below alpha |r| = 1/2.
__device__ __forceinline__ void ewald_part(float rx, float ry, float rz, float L,
                                           const float4 *hv, int nh, int part, int parts,
                                           float &gx, float &gy, float &gz, float &ps)
{
    const float alpha = 2.0f / L;
    const float c2 = 1.1283791670955126f;    // 2 / sqrt(pi)
    for (int i = part; i < 125; i += parts) {
        const int nx = i / 25 - 2, ny = (i / 5) % 5 - 2, nz = i % 5 - 2;
        const float dx = rx + (float)nx * L, dy = ry + (float)ny * L, dz = rz + (float)nz * L;
        const float s2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
        const float s = sqrtf(s2);
        const float x = alpha * s;
        float g, p;
        if (i == 62) {
            if (x < 0.5f) {
                // erf(x)/x and -erf(x)/x^3 + c2 exp(-x^2)/x^2 as series in x^2
                const float x2 = x * x;
                float e = 0.f, fk = 0.f, t = 1.f, u = -1.f;
                for (int k = 0; k < 9; ++k) {
                    e += t / (float)(2 * k + 1);
                    t *= -x2 / (float)(k + 1);
                }
                for (int k = 1; k < 10; ++k) {
                    fk += u * (float)(2 * k) / (float)(2 * k + 1);
                    u *= -x2 / (float)(k + 1);
                }
                g = alpha * alpha * alpha * c2 * fk;
                p = -alpha * c2 * e;
            } else {
                const float er = erff(x);
                g = -er / (s2 * s) + alpha * c2 * expf(-x * x) / s2;
                p = -er / s;
            }
        } else {
            const float ec = erfcf(x);
            g = ec / (s2 * s) + alpha * c2 * expf(-x * x) / s2;
            p = ec / s;
        }
        gx = fmaf(-dx, g, gx);
        gy = fmaf(-dy, g, gy);
        gz = fmaf(-dz, g, gz);
        ps += p;
    }
    const float inv_l = 1.0f / L;
    const float kphi = inv_l * 0.3183098861837907f;     // 1 / (pi L)
    const float kacc = -2.0f * inv_l * inv_l;
    for (int j = part; j < nh; j += parts) {
        const float4 h = hv[j];
        float sn, cs;
        sincospif(2.0f * (h.x * rx + h.y * ry + h.z * rz) * inv_l, &sn, &cs);
        ps = fmaf(h.w * kphi, cs, ps);
        const float gs = kacc * h.w * sn;
        gx = fmaf(gs, h.x, gx);
        gy = fmaf(gs, h.y, gy);
        gz = fmaf(gs, h.z, gz);
    }
    if (part == 0) ps -= 3.14159265358979f / (alpha * alpha * L * L * L);
}

struct EwaldSmem {
    float4 red[GRAV_WARPS][32][2];      // cross-lane combine: (sum, compensation)
};

// One warp per GC_EWALD task of the task list.  Targets are taken 32 at a
// time; with T targets in a pass the warp splits into S = 32 / T lanes per
// target, lane (t, s) summing the image and reciprocal-vector parts s, s + S,
// ... of every source with compensation; the S partial sums of a target are
// combined as compensated pairs in lane order.
__global__ void __launch_bounds__(GRAV_THREADS) k_ewald(InterArgs a)
{
    __shared__ EwaldSmem sm;
    const int lane = threadIdx.x & 31;
    const int wib = threadIdx.x >> 5;
    const uint64_t gwarp = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nwarps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t it = 0;; ++it) {
        unsigned long long w = gwarp + it * nwarps;   // fixed share without a queue
        if (a.queue) {
            if (lane == 0) w = atomicAdd(a.queue, 1ull);
            w = __shfl_sync(0xffffffffu, w, 0);
        }
        if (w >= a.n_lj) break;
        const uint32_t ti = a.lj_list[w];
        const TaskRec r = a.tasks[ti];
        if (r.kind != GC_EWALD) continue;
        const float4 *As = a.stg_t + (r.tgt_off - a.tgt_base);
        const float4 *Bs = a.stg_s + (r.src_off - a.src_base) + (ti - a.task_base);
        for (uint32_t o0 = 0; o0 < r.nt; o0 += 32) {
            const int T = (int)min(32u, r.nt - o0);
            const int S = 32 / T;
            const int t = lane % T, sl = lane / T;
            float sx = 0.f, sy = 0.f, sz = 0.f, su = 0.f;
            float cx = 0.f, cy = 0.f, cz = 0.f, cu = 0.f;
            if (sl < S) {
                const float4 me = As[o0 + t];
                for (uint32_t q = 0; q < r.ns; ++q) {
                    const float4 src = Bs[q];
                    float gx = 0.f, gy = 0.f, gz = 0.f, ps = 0.f;
                    ewald_part(me.x - src.x, me.y - src.y, me.z - src.z, a.ewald_L, a.ewald_h,
                               a.n_ewald_h, sl, S, gx, gy, gz, ps);
                    kahan_add(sx, cx, src.w * gx);
                    kahan_add(sy, cy, src.w * gy);
                    kahan_add(sz, cz, src.w * gz);
                    kahan_add(su, cu, -src.w * ps);
                }
            }
            sm.red[wib][lane][0] = make_float4(sx, sy, sz, su);
            sm.red[wib][lane][1] = make_float4(cx, cy, cz, cu);
            __syncwarp();
            if (sl == 0) {
                float4 vs = sm.red[wib][t][0], vc = sm.red[wib][t][1];
                for (int s2 = 1; s2 < S; ++s2) {
                    const int l = s2 * T + t;
                    const float4 ws = sm.red[wib][l][0], wc = sm.red[wib][l][1];
                    comp_add(vs.x, vc.x, ws.x, wc.x);
                    comp_add(vs.y, vc.y, ws.y, wc.y);
                    comp_add(vs.z, vc.z, ws.z, wc.z);
                    comp_add(vs.w, vc.w, ws.w, wc.w);
                }
                const uint32_t pos = a.perm_t[r.tgt_off + o0 + t];
                const uint64_t row = r.row_off + pos;
                a.res[2 * row] = vs;
                a.res[2 * row + 1] = vc;
                a.row_id[row] = a.tgt_ids[r.tgt_off + pos];
            }
            __syncwarp();
        }
    }
}

// ---------------------------------------------------------------------------
// scatter: per-id FP64 totals in admission order
// ---------------------------------------------------------------------------

__global__ void k_iota(uint32_t *v, uint64_t n)
{
    GRID_STRIDE(i, n) v[i] = (uint32_t)i;
}

// Rows whose ids are distinct: each row is its id's only contribution, so
// the sorted path's result is one FP64 add per component, done in place.
__global__ void k_reduce_unique(uint64_t n_rows, const uint32_t *row_id, const float4 *res,
                                gcd4 *totals)
{
    GRID_STRIDE(r, n_rows) {
        const uint32_t id = row_id[r];
        const float4 sv = res[2 * r], cv = res[2 * r + 1];
        gcd4 acc = totals[id];
        acc.x += gc_f2d(sv.x) - gc_f2d(cv.x);
        acc.y += gc_f2d(sv.y) - gc_f2d(cv.y);
        acc.z += gc_f2d(sv.z) - gc_f2d(cv.z);
        acc.w += gc_f2d(sv.w) - gc_f2d(cv.w);
        totals[id] = acc;
    }
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
        uint32_t q = b;
        // four rows' loads in flight at a time; the sums keep the row order
        for (; q + 4 <= e; q += 4) {
            uint32_t rw[4];
            float4 sv[4], cv[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) rw[u] = row[q + u];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                sv[u] = res[2 * (uint64_t)rw[u]];
                cv[u] = res[2 * (uint64_t)rw[u] + 1];
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
                acc.x += gc_f2d(sv[u].x) - gc_f2d(cv[u].x);
                acc.y += gc_f2d(sv[u].y) - gc_f2d(cv[u].y);
                acc.z += gc_f2d(sv[u].z) - gc_f2d(cv[u].z);
                acc.w += gc_f2d(sv[u].w) - gc_f2d(cv[u].w);
            }
        }
        for (; q < e; ++q) {
            uint32_t rw = row[q];
            float4 s = res[2 * (uint64_t)rw], c = res[2 * (uint64_t)rw + 1];
            acc.x += gc_f2d(s.x) - gc_f2d(c.x);
            acc.y += gc_f2d(s.y) - gc_f2d(c.y);
            acc.z += gc_f2d(s.z) - gc_f2d(c.z);
            acc.w += gc_f2d(s.w) - gc_f2d(c.w);
        }
        totals[id] = acc;
    }
}

// Small batches (at most SCATTER_SMALL rows): the per-id accumulation in
// one block.  The (id, row) keys -- distinct, one per row -- are sorted in
// shared memory by a bitonic network, which orders rows by id and, within
// an id, by row (the order of the stable sort of the general path); each
// id's rows are then added to its total in that order with the same
// arithmetic as k_reduce_runs, so both paths give the same totals.
constexpr int SCATTER_SMALL = 2048;

__global__ void __launch_bounds__(1024) k_scatter_small(uint32_t n_rows, const uint32_t *row_id,
                                                        const float4 *res, gcd4 *totals)
{
    __shared__ unsigned long long sorted[SCATTER_SMALL];
    uint32_t n2 = 1;
    while (n2 < n_rows) n2 <<= 1;
    for (uint32_t r = threadIdx.x; r < n2; r += blockDim.x)
        sorted[r] = r < n_rows ? ((unsigned long long)row_id[r] << 32) | r : ~0ull;
    __syncthreads();
    for (uint32_t k = 2; k <= n2; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = threadIdx.x; i < n2; i += blockDim.x) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const unsigned long long a = sorted[i], b = sorted[l];
                    if ((a > b) == ((i & k) == 0)) {
                        sorted[i] = b;
                        sorted[l] = a;
                    }
                }
            }
            __syncthreads();
        }
    for (uint32_t q = threadIdx.x; q < n_rows; q += blockDim.x) {
        const uint32_t id = (uint32_t)(sorted[q] >> 32);
        if (q > 0 && (uint32_t)(sorted[q - 1] >> 32) == id) continue;   // not a run start
        gcd4 acc = totals[id];
        for (uint32_t e = q; e < n_rows && (uint32_t)(sorted[e] >> 32) == id; ++e) {
            const uint32_t rw = (uint32_t)sorted[e];
            const float4 sv = res[2 * (uint64_t)rw], cv = res[2 * (uint64_t)rw + 1];
            acc.x += gc_f2d(sv.x) - gc_f2d(cv.x);
            acc.y += gc_f2d(sv.y) - gc_f2d(cv.y);
            acc.z += gc_f2d(sv.z) - gc_f2d(cv.z);
            acc.w += gc_f2d(sv.w) - gc_f2d(cv.w);
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
                      uint64_t task_id_base, TaskRec *out, cudaStream_t s)
{
    if (n_tasks == 0) return GC_OK;
    ++p->stats.kernel_launches;
    k_task_recs<<<grid_for(n_tasks, 256, p->num_sms * 16), 256, 0, s>>>(
        n_tasks, task_ids, kinds, shifts, tgt_off, src_off, tgt_base, src_base, task_id_base,
        out, p->d_ctr, p->n_ewald_h > 0 ? 1 : 0);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

// Result rows, work units and LJ task list of the batch in context c.  Reads
// back {rows, gravity work units, LJ tasks, interactions, longest list}.
int gc_prepare_issue(gc_pool *p, FlushCtx &c)
{
    const uint64_t n = c.n_tasks;
    TaskRec *tasks = c.tasks.as<TaskRec>();
    GC_TRY(c.rowcnt.reserve((n + 1) * sizeof(uint64_t) * 2));
    GC_TRY(c.wu_cnt.reserve((n + 1) * sizeof(uint32_t) * 2));
    GC_TRY(c.wu_off.reserve((n + 1) * sizeof(uint32_t) * 2));
    uint64_t *rows = c.rowcnt.as<uint64_t>();
    uint64_t *row_off = rows + (n + 1);
    uint32_t *wu_g = c.wu_cnt.as<uint32_t>();
    uint32_t *lj = wu_g + (n + 1);
    uint32_t *wu_off = c.wu_off.as<uint32_t>();
    uint32_t *lj_off = wu_off + (n + 1);
    GC_CUDA_TRY(cudaMemsetAsync(c.d_ctr, 0, sizeof(unsigned long long) * FC_COUNT, c.s));
    GC_CUDA_TRY(cudaMemsetAsync(rows + n, 0, sizeof(uint64_t), c.s));
    GC_CUDA_TRY(cudaMemsetAsync(wu_g + n, 0, sizeof(uint32_t), c.s));
    GC_CUDA_TRY(cudaMemsetAsync(lj + n, 0, sizeof(uint32_t), c.s));
    ++p->stats.kernel_launches;
    k_prep_counts<<<grid_for(n, 256, p->num_sms * 16), 256, 0, c.s>>>(tasks, n, rows, wu_g, lj,
                                                                       c.d_ctr,
                                                                       p->wu_max_targets);
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u64(c.cub_tmp, rows, row_off, n + 1, c.s));
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u32(c.cub_tmp, wu_g, wu_off, n + 1, c.s));
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u32(c.cub_tmp, lj, lj_off, n + 1, c.s));
    // sizes into the context's pinned words (the copies do not block)
    c.h_ctr[FH_ROWS] = c.h_ctr[FH_WU] = c.h_ctr[FH_LJ] = 0;
    GC_CUDA_TRY(cudaMemcpyAsync(c.h_ctr + FH_ROWS, row_off + n, sizeof(uint64_t),
                                cudaMemcpyDeviceToHost, c.s));
    GC_CUDA_TRY(cudaMemcpyAsync(c.h_ctr + FH_WU, wu_off + n, sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, c.s));
    GC_CUDA_TRY(cudaMemcpyAsync(c.h_ctr + FH_LJ, lj_off + n, sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, c.s));
    GC_CUDA_TRY(cudaMemcpyAsync(c.h_ctr, c.d_ctr, sizeof(unsigned long long) * FC_COUNT,
                                cudaMemcpyDeviceToHost, c.s));
    return GC_OK;
}

int gc_prepare_finish(gc_pool *p, FlushCtx &c, uint64_t info[5])
{
    const uint64_t n = c.n_tasks;
    TaskRec *tasks = c.tasks.as<TaskRec>();
    uint64_t *row_off = c.rowcnt.as<uint64_t>() + (n + 1);
    uint32_t *wu_off = c.wu_off.as<uint32_t>();
    uint32_t *lj_off = wu_off + (n + 1);
    const uint64_t h_rows = c.h_ctr[FH_ROWS];
    const uint32_t h_wu = (uint32_t)c.h_ctr[FH_WU], h_lj = (uint32_t)c.h_ctr[FH_LJ];
    GC_TRY(c.wu.reserve(((uint64_t)h_wu + 1) * sizeof(GravWU)));
    GC_TRY(c.lj_list.reserve(((uint64_t)h_lj + 1) * sizeof(uint32_t)));
    ++p->stats.kernel_launches;
    k_prep_fill<<<grid_for(n, 256, p->num_sms * 16), 256, 0, c.s>>>(
        tasks, n, row_off, wu_off, lj_off, c.wu.as<GravWU>(), c.lj_list.as<uint32_t>(),
        p->wu_max_targets);
    GC_CUDA_TRY(cudaGetLastError());
    info[0] = h_rows;
    info[1] = h_wu;
    info[2] = h_lj;
    info[3] = c.h_ctr[FC_INTER];
    info[4] = c.h_ctr[FC_MAXLIST];
    return GC_OK;
}

int gc_prepare(gc_pool *p, FlushCtx &c, uint64_t info[5])
{
    GC_TRY(gc_prepare_issue(p, c));
    GC_CUDA_TRY(cudaStreamSynchronize(c.s));
    return gc_prepare_finish(p, c, info);
}

// Host copies of the per-task work-unit offsets (for waves and per-task
// launches): wu_off[0..n], lj_off[0..n].
int gc_read_wu_offsets(gc_pool *p, FlushCtx &c, std::vector<uint32_t> &wu_off,
                       std::vector<uint32_t> &lj_off)
{
    (void)p;
    const uint64_t n = c.n_tasks;
    wu_off.resize(n + 1);
    lj_off.resize(n + 1);
    uint32_t *d_wu_off = c.wu_off.as<uint32_t>();
    GC_CUDA_TRY(cudaMemcpyAsync(wu_off.data(), d_wu_off, (n + 1) * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, c.s));
    GC_CUDA_TRY(cudaMemcpyAsync(lj_off.data(), d_wu_off + (n + 1), (n + 1) * sizeof(uint32_t),
                                cudaMemcpyDeviceToHost, c.s));
    GC_CUDA_TRY(cudaStreamSynchronize(c.s));
    return GC_OK;
}

int gc_pack(gc_pool *p, FlushCtx &c, uint64_t t0, uint64_t t1, uint64_t tgt_base,
            uint64_t src_base, uint64_t msrc, const uint32_t *ent, uint64_t ent_nt)
{
    if (t1 <= t0) return GC_OK;
    static bool attr_set = false;
    if (!attr_set) {
        GC_CUDA_TRY(cudaFuncSetAttribute(
            k_pack_large<PK_CAP>, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)sizeof(PackSmemLarge<PK_CAP>)));
        GC_CUDA_TRY(cudaFuncSetAttribute(
            k_pack_large<PK_CAP_HUGE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
            (int)sizeof(PackSmemLarge<PK_CAP_HUGE>)));
        GC_CUDA_TRY(cudaFuncSetAttribute(k_pack_mid<PM_CAP>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(PackSmemMid<PM_CAP>)));
        GC_CUDA_TRY(cudaFuncSetAttribute(k_pack_mid<PM_CAP / 2>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)sizeof(PackSmemMid<PM_CAP / 2>)));
        attr_set = true;
    }
    PackArgs a;
    a.tasks = c.tasks.as<TaskRec>();
    a.t0 = t0;
    a.n_lists = 2 * (t1 - t0);
    a.tgt_ids = c.tgt_ids.as<uint32_t>();
    a.src_ids = c.src_ids.as<uint32_t>();
    a.slot_of_id = p->d_slot_of_id;
    a.ent_t = ent;
    a.ent_s = ent ? ent + ent_nt : nullptr;
    a.task_base = t0;
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) < p->cfg.pool_capacity) ++bits;
    a.passes = (bits + 7) / 8;
    a.perm_t = c.tgt_perm.as<uint32_t>();
    a.perm_s = c.src_perm.as<uint32_t>();
    a.stg_t = c.stg_tgt.as<float4>();
    a.stg_s = c.stg_src.as<float4>();
    a.tgt_base = tgt_base;
    a.src_base = src_base;
    a.pool = p->d_pool;
    a.ma = c.merge_a.as<uint64_t>();
    a.mb = c.merge_b.as<uint64_t>();
    a.msrc = msrc;
    ++p->stats.kernel_launches;
    a.work = c.d_ctr + FC_PACK_WORK;
    GC_CUDA_TRY(cudaMemsetAsync(a.work, 0, 4 * sizeof(unsigned long long), c.s));
    // The size classes pack disjoint lists, each with a claim counter of its
    // own.  The block-per-list classes of more than 1024 entries a batch
    // needs run on side streams beside the context's stream (longest lists
    // first), so that a small batch's pack takes about its longest class's
    // time instead of the sum over its classes; the context's stream joins
    // them before the interaction.
    int forked = 0;
    cudaError_t ferr = cudaSuccess;
    auto side = [&](int i) -> cudaStream_t {
        if (!forked++ && ferr == cudaSuccess) ferr = cudaEventRecord(c.pev[3], c.s);
        if (ferr == cudaSuccess) ferr = cudaStreamWaitEvent(c.ps[i], c.pev[3], 0);
        return c.ps[i];
    };
    bool joined[3] = {false, false, false};
    if (c.max_list > PK_CAP) {
        ++p->stats.kernel_launches;
        constexpr int nw = PackLargeWarps<PK_CAP_HUGE>::value;
        k_pack_large<PK_CAP_HUGE><<<grid_for(a.n_lists, 1, p->num_sms), nw * 32,
                                    sizeof(PackSmemLarge<PK_CAP_HUGE>), side(0)>>>(a);
        joined[0] = true;
    }
    if (c.max_list > PM_CAP) {
        ++p->stats.kernel_launches;
        constexpr int nw = PackLargeWarps<PK_CAP>::value;
        k_pack_large<PK_CAP><<<grid_for(a.n_lists, 1, p->num_sms * 3), nw * 32,
                               sizeof(PackSmemLarge<PK_CAP>), side(1)>>>(a);
        joined[1] = true;
    }
    if (c.max_list > PM_CAP / 2) {
        ++p->stats.kernel_launches;
        k_pack_mid<PM_CAP><<<grid_for(a.n_lists, 1, p->num_sms * 6), PM_THREADS,
                             sizeof(PackSmemMid<PM_CAP>), side(2)>>>(a);
        joined[2] = true;
    }
    // the block-per-list classes only when the batch has lists of their sizes
    if (c.max_list > 32) {
        ++p->stats.kernel_launches;
        k_pack_mid<PM_CAP / 2><<<grid_for(a.n_lists, 1, p->num_sms * 9), PM_THREADS,
                                 sizeof(PackSmemMid<PM_CAP / 2>), c.s>>>(a);
    }
    k_pack_small<<<grid_for(a.n_lists * 32, 256, p->num_sms * 32), 256, 0, c.s>>>(a);
    GC_CUDA_TRY(ferr);
    GC_CUDA_TRY(cudaGetLastError());
    for (int i = 0; i < 3; ++i)
        if (joined[i]) {
            GC_CUDA_TRY(cudaEventRecord(c.pev[i], c.ps[i]));
            GC_CUDA_TRY(cudaStreamWaitEvent(c.s, c.pev[i], 0));
        }
    return GC_OK;
}

static void fill_inter_args(gc_pool *p, FlushCtx &c, uint64_t tgt_base, uint64_t src_base,
                            uint64_t task_base, InterArgs &a)
{
    a.tasks = c.tasks.as<TaskRec>();
    a.task_base = task_base;
    a.stg_t = c.stg_tgt.as<float4>();
    a.stg_s = c.stg_src.as<float4>();
    a.tgt_base = tgt_base;
    a.src_base = src_base;
    a.perm_t = c.tgt_perm.as<uint32_t>();
    a.perm_s = c.src_perm.as<uint32_t>();
    a.tgt_ids = c.tgt_ids.as<uint32_t>();
    a.src_ids = c.src_ids.as<uint32_t>();
    a.eps2 = p->cfg.eps2;
    a.lj_eps24 = 24.0f * p->cfg.lj_eps;
    a.lj_eps4 = 4.0f * p->cfg.lj_eps;
    a.lj_sig2 = p->cfg.lj_sigma * p->cfg.lj_sigma;
    a.rc2_grid = p->rc2_grid;
    a.edge_grid = p->md_edge_grid;
    a.res = c.res.as<float4>();
    a.row_id = c.row_id.as<uint32_t>();
    a.queue = c.d_ctr + FC_QUEUE;
    a.lj_in = c.d_ctr + FC_LJ_IN;
    a.ewald_h = p->d_ewald_h;
    a.n_ewald_h = p->n_ewald_h;
    a.ewald_L = p->cfg.ewald_box;
    a.flags = p->d_ctr + CTR_FLAGS;
}

// Tile shapes of the gravity kernel: TP in {64, 128, 256} source pairs per
// staged tile, KB in {8, 16, 32} pairs per plain partial sum, TPL in {1, 2}
// targets per lane.
struct GravVariant {
    void (*fn)(InterArgs);
    uint32_t tp, kb, tpl;
    size_t smem;
    int ready;    // shared-memory limit raised
    int per_sm;   // resident blocks per SM (0: not yet asked)
};

#define GRAV_V(tp, kb, tpl) {k_gravity<tp, kb, tpl>, tp, kb, tpl, sizeof(GravSmem<tp, tpl>), 0, 0}
static GravVariant g_grav[18] = {
    GRAV_V(64, 8, 1),  GRAV_V(64, 16, 1),  GRAV_V(64, 32, 1),
    GRAV_V(128, 8, 1), GRAV_V(128, 16, 1), GRAV_V(128, 32, 1),
    GRAV_V(256, 8, 1), GRAV_V(256, 16, 1), GRAV_V(256, 32, 1),
    GRAV_V(64, 8, 2),  GRAV_V(64, 16, 2),  GRAV_V(64, 32, 2),
    GRAV_V(128, 8, 2), GRAV_V(128, 16, 2), GRAV_V(128, 32, 2),
    GRAV_V(256, 8, 2), GRAV_V(256, 16, 2), GRAV_V(256, 32, 2)};
#undef GRAV_V

static GravVariant *grav_variant(uint32_t tp, uint32_t kb, uint32_t tpl)
{
    for (GravVariant &v : g_grav)
        if (v.tp == tp && v.kb == kb && v.tpl == tpl) return &v;
    return nullptr;
}

static bool grav_shape_ok(uint32_t tp, uint32_t kb, uint32_t tpl)
{
    return grav_variant(tp, kb, tpl) != nullptr;
}

// The pool's variant, its shared-memory limit raised.
static int grav_setup(gc_pool *p, GravVariant **out)
{
    GravVariant *v = grav_variant(p->wu_tile, p->wu_kb, p->wu_tpl);
    if (!v) return GC_ERR_STATE;
    if (!v->ready) {
        if (cudaFuncSetAttribute(v->fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)v->smem) != cudaSuccess)
            return GC_ERR_CUDA;
        v->ready = 1;
    }
    *out = v;
    return GC_OK;
}

// Persistent grid of the gravity kernel: resident blocks per SM (occupancy
// API) x SMs -- the number of work units one launch runs at once.
// Resident blocks of a kernel on the whole GPU (occupancy API), cached.
template <class K>
static int resident_blocks(gc_pool *p, K kernel, int &cache)
{
    if (cache == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kernel, GRAV_THREADS, 0) !=
                cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        cache = per_sm;
    }
    return cache * p->num_sms;
}

static int lj_blocks(gc_pool *p)
{
    static int per_sm = 0;
    return resident_blocks(p, k_lj, per_sm);
}

static int ewald_blocks(gc_pool *p)
{
    static int per_sm = 0;
    return resident_blocks(p, k_ewald, per_sm);
}

int gc_grav_blocks(gc_pool *p)
{
    GravVariant *v = nullptr;
    if (grav_setup(p, &v) != GC_OK) {
        cudaGetLastError();
        return p->num_sms;
    }
    if (v->per_sm == 0) {
        int per_sm = 0;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, v->fn, GRAV_THREADS,
                                                          v->smem) != cudaSuccess ||
            per_sm < 1) {
            cudaGetLastError();
            per_sm = 1;
        }
        v->per_sm = per_sm;
    }
    return v->per_sm * p->num_sms;
}

extern "C" int gc_max_combine_size(gc_pool_t *p, uint64_t *out)
{
    if (!p || !out) return GC_ERR_ARG;
    *out = (uint64_t)gc_grav_blocks(p) * (uint64_t)GRAV_WARPS;
    return GC_OK;
}

// Launch the interaction kernels over gravity work units [w0, w1) and LJ
// tasks [l0, l1) of the prepared batch.
int gc_interact_range(gc_pool *p, FlushCtx &c, uint64_t w0, uint64_t w1, uint64_t l0,
                      uint64_t l1, uint64_t tgt_base, uint64_t src_base, uint64_t task_base)
{
    InterArgs a;
    fill_inter_args(p, c, tgt_base, src_base, task_base, a);
    const int full = gc_grav_blocks(p);
    if (w1 > w0) {
        a.wu = c.wu.as<GravWU>() + w0;
        a.n_wu = w1 - w0;
        a.lj_list = nullptr;
        a.n_lj = 0;
        if (p->wu_schedule == GC_SCHED_LPT && a.n_wu > 1) {
            // reorder this wave's work units longest first, in place
            const uint64_t m = a.n_wu;
            GC_TRY(c.lpt.reserve(m * (2 * sizeof(uint64_t) + 2 * sizeof(uint32_t) +
                                      sizeof(GravWU)) + 64));
            char *b = (char *)c.lpt.p;
            GravWU *tmp = (GravWU *)b;
            uint64_t *k0 = (uint64_t *)(b + m * sizeof(GravWU));
            uint64_t *k1 = k0 + m;
            uint32_t *i0 = (uint32_t *)(k1 + m);
            uint32_t *i1 = i0 + m;
            GravWU *w = c.wu.as<GravWU>() + w0;
            p->stats.kernel_launches += 2;
            k_wu_cost<<<grid_for(m, 256, p->num_sms * 16), 256, 0, c.s>>>(w, m, a.tasks, k0, i0);
            ++p->stats.primitive_calls;
            GC_TRY(gc_sort_pairs_u64(c.cub_tmp, k0, k1, i0, i1, m, 40, c.s));
            k_wu_gather<<<grid_for(m, 256, p->num_sms * 16), 256, 0, c.s>>>(w, i1, m, tmp);
            GC_CUDA_TRY(cudaMemcpyAsync(w, tmp, m * sizeof(GravWU), cudaMemcpyDeviceToDevice,
                                        c.s));
        }
        GC_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), c.s));
        const uint64_t need = (a.n_wu + GRAV_WARPS - 1) / GRAV_WARPS;
        const unsigned g = (unsigned)(need < (uint64_t)full ? need : (uint64_t)full);
        GravVariant *v = nullptr;
        GC_TRY(grav_setup(p, &v));
        ++p->stats.kernel_launches;
        v->fn<<<g, GRAV_THREADS, v->smem, c.s>>>(a);
    }
    if (l1 > l0) {
        a.wu = nullptr;
        a.n_wu = 0;
        a.lj_list = c.lj_list.as<uint32_t>() + l0;
        a.n_lj = l1 - l0;
        GC_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), c.s));
        const uint64_t need = (a.n_lj + GRAV_WARPS - 1) / GRAV_WARPS;
        const unsigned g = (unsigned)std::min<uint64_t>(need, (uint64_t)lj_blocks(p));
        ++p->stats.kernel_launches;
        k_lj<<<g, GRAV_THREADS, 0, c.s>>>(a);
        if (p->n_ewald_h > 0) {
            GC_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), c.s));
            const unsigned ge = (unsigned)std::min<uint64_t>(need, (uint64_t)ewald_blocks(p));
            ++p->stats.kernel_launches;
            k_ewald<<<ge, GRAV_THREADS, 0, c.s>>>(a);
        }
    }
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

// One launch per task (the uncombined baseline): the same kernels, static
// work assignment, grid sized to the task.
int gc_interact_one_task(gc_pool *p, FlushCtx &c, uint64_t w0, uint64_t w1, uint64_t l0,
                         uint64_t l1, uint64_t tgt_base, uint64_t src_base, uint64_t task_base)
{
    InterArgs a;
    fill_inter_args(p, c, tgt_base, src_base, task_base, a);
    a.queue = nullptr;
    if (w1 > w0) {
        a.wu = c.wu.as<GravWU>() + w0;
        a.n_wu = w1 - w0;
        a.lj_list = nullptr;
        a.n_lj = 0;
        const unsigned g = (unsigned)((a.n_wu + GRAV_WARPS - 1) / GRAV_WARPS);
        GravVariant *v = nullptr;
        GC_TRY(grav_setup(p, &v));
        ++p->stats.kernel_launches;
        v->fn<<<g, GRAV_THREADS, v->smem, c.s>>>(a);
    }
    if (l1 > l0) {
        a.wu = nullptr;
        a.n_wu = 0;
        a.lj_list = c.lj_list.as<uint32_t>() + l0;
        a.n_lj = l1 - l0;
        ++p->stats.kernel_launches;
        k_lj<<<1, 32, 0, c.s>>>(a);
        if (p->n_ewald_h > 0) {
            ++p->stats.kernel_launches;
            k_ewald<<<1, 32, 0, c.s>>>(a);
        }
    }
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

int gc_scatter(gc_pool *p, FlushCtx &c)
{
    const uint64_t n_rows = c.n_rows;
    if (n_rows == 0) return GC_OK;
    if (c.md_struct) return gc_md_reduce(p, c);
    if (c.unique_rows) {
        ++p->stats.kernel_launches;
        k_reduce_unique<<<grid_for(n_rows, 256, p->num_sms * 16), 256, 0, c.s>>>(
            n_rows, c.row_id.as<uint32_t>(), c.res.as<float4>(), p->d_totals);
        GC_CUDA_TRY(cudaGetLastError());
        return GC_OK;
    }
    if (n_rows <= (uint64_t)SCATTER_SMALL) {   // one block (no sorted state kept)
        ++p->stats.kernel_launches;
        k_scatter_small<<<1, 1024, 0, c.s>>>((uint32_t)n_rows, c.row_id.as<uint32_t>(),
                                             c.res.as<float4>(), p->d_totals);
        GC_CUDA_TRY(cudaGetLastError());
        return GC_OK;
    }
    GC_TRY(c.rows_tmp.reserve(n_rows * sizeof(uint32_t)));
    GC_TRY(c.rid_sorted.reserve(n_rows * sizeof(uint32_t)));
    GC_TRY(c.row_sorted.reserve(n_rows * sizeof(uint32_t)));
    GC_TRY(c.runs.reserve((n_rows + 1) * sizeof(uint32_t)));
    const int maxb = p->num_sms * 16;
    ++p->stats.kernel_launches;
    k_iota<<<grid_for(n_rows, 256, maxb), 256, 0, c.s>>>(c.rows_tmp.as<uint32_t>(), n_rows);
    int bits = 1;
    while (bits < 32 && ((uint64_t)1 << bits) < p->cfg.id_capacity) ++bits;
    ++p->stats.primitive_calls;
    GC_TRY(gc_sort_pairs_u32(c.cub_tmp, c.row_id.as<uint32_t>(), c.rid_sorted.as<uint32_t>(),
                             c.rows_tmp.as<uint32_t>(), c.row_sorted.as<uint32_t>(), n_rows,
                             bits, c.s));
    GC_TRY(gc_compact(p, c.tiles, c.s, CK_RUN_START, n_rows, nullptr,
                      c.rid_sorted.as<uint32_t>(), c.runs.as<uint32_t>(), c.d_ctr + FC_RUNS));
    ++p->stats.kernel_launches;
    k_reduce_runs<<<grid_for(n_rows, 256, maxb), 256, 0, c.s>>>(
        c.runs.as<uint32_t>(), c.d_ctr + FC_RUNS, n_rows, c.rid_sorted.as<uint32_t>(),
        c.row_sorted.as<uint32_t>(), c.res.as<float4>(), p->d_totals);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

// The accumulation step of a batch whose rows were sorted by id before (the
// run boundaries and row order are kept in the context): rows summed into
// the per-id totals in the same order.
int gc_scatter_replay(gc_pool *p, FlushCtx &c)
{
    if (c.n_rows == 0) return GC_OK;
    if (c.md_struct) return gc_md_reduce(p, c);
    if (c.unique_rows) return gc_scatter(p, c);   // no sorted state to replay
    if (c.n_rows <= (uint64_t)SCATTER_SMALL) return gc_scatter(p, c);   // the one-block path
    ++p->stats.kernel_launches;
    k_reduce_runs<<<grid_for(c.n_rows, 256, p->num_sms * 16), 256, 0, c.s>>>(
        c.runs.as<uint32_t>(), c.d_ctr + FC_RUNS, c.n_rows, c.rid_sorted.as<uint32_t>(),
        c.row_sorted.as<uint32_t>(), c.res.as<float4>(), p->d_totals);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

// ---------------------------------------------------------------------------
// interaction schedule: set / get / autotune
// ---------------------------------------------------------------------------

extern "C" int gc_set_tuning(gc_pool_t *p, const gc_tuning *t)
{
    if (!p || !t) return GC_ERR_ARG;
    if (t->wu_max_targets != 8 && t->wu_max_targets != 16 && t->wu_max_targets != 32)
        return GC_ERR_ARG;
    if (t->schedule != GC_SCHED_FIFO && t->schedule != GC_SCHED_LPT) return GC_ERR_ARG;
    if (!grav_shape_ok(t->tile_pairs, t->comp_block, t->targets_per_lane)) return GC_ERR_ARG;
    p->wu_max_targets = t->wu_max_targets;
    p->wu_schedule = t->schedule;
    p->wu_tile = t->tile_pairs;
    p->wu_kb = t->comp_block;
    p->wu_tpl = t->targets_per_lane;
    return GC_OK;
}

extern "C" int gc_get_tuning(gc_pool_t *p, gc_tuning *t)
{
    if (!p || !t) return GC_ERR_ARG;
    t->wu_max_targets = p->wu_max_targets;
    t->schedule = p->wu_schedule;
    t->tile_pairs = p->wu_tile;
    t->comp_block = p->wu_kb;
    t->targets_per_lane = p->wu_tpl;
    return GC_OK;
}

// Rebuild the gravity work units of a context's batch for work units of at
// most wu_max targets; *n_wu_out = their number.
static int rebuild_wus(gc_pool *p, FlushCtx &c, uint32_t wu_max, uint64_t *n_wu_out)
{
    const uint64_t n = c.n_tasks;
    TaskRec *tasks = c.tasks.as<TaskRec>();
    uint64_t *rows = c.rowcnt.as<uint64_t>();
    uint32_t *wu_g = c.wu_cnt.as<uint32_t>();
    uint32_t *lj = wu_g + (n + 1);
    uint32_t *wu_off = c.wu_off.as<uint32_t>();
    GC_CUDA_TRY(cudaMemsetAsync(wu_g + n, 0, sizeof(uint32_t), c.s));
    p->stats.kernel_launches += 1;
    // counters of the batch are recounted into a scratch copy
    GC_TRY(c.lpt.reserve(sizeof(unsigned long long) * FC_COUNT + 64));
    unsigned long long *scratch_ctr = c.lpt.as<unsigned long long>();
    GC_CUDA_TRY(cudaMemsetAsync(scratch_ctr, 0, sizeof(unsigned long long) * FC_COUNT, c.s));
    k_prep_counts<<<grid_for(n, 256, p->num_sms * 16), 256, 0, c.s>>>(tasks, n, rows, wu_g, lj,
                                                                       scratch_ctr, wu_max);
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u32(c.cub_tmp, wu_g, wu_off, n + 1, c.s));
    uint32_t h_wu = 0;
    GC_CUDA_TRY(cudaMemcpyAsync(&h_wu, wu_off + n, sizeof(uint32_t), cudaMemcpyDeviceToHost, c.s));
    GC_CUDA_TRY(cudaStreamSynchronize(c.s));
    GC_TRY(c.wu.reserve(((uint64_t)h_wu + 1) * sizeof(GravWU)));
    ++p->stats.kernel_launches;
    k_prep_fill<<<grid_for(n, 256, p->num_sms * 16), 256, 0, c.s>>>(
        tasks, n, nullptr, wu_off, nullptr, c.wu.as<GravWU>(), nullptr, wu_max);
    GC_CUDA_TRY(cudaGetLastError());
    *n_wu_out = h_wu;
    return GC_OK;
}

extern "C" int gc_autotune(gc_pool_t *p, int reps, gc_tuning *best_out,
                           float ms_out[GC_TUNE_COUNT])
{
    if (!p || reps < 1) return GC_ERR_ARG;
    if (p->last < 0 || !p->ctx[p->last].valid) return GC_ERR_NOT_READY;
    FlushCtx &c = p->ctx[p->last];
    GC_CUDA_TRY(cudaEventSynchronize(c.ev_done));
    if (c.n_waves != 1) return GC_ERR_STATE;
    const gc_tuning saved{p->wu_max_targets, p->wu_schedule, p->wu_tile, p->wu_kb, p->wu_tpl};
    const uint32_t wus[3] = {8, 16, 32}, tps[3] = {64, 128, 256}, kbs[3] = {8, 16, 32};
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        if (e0) cudaEventDestroy(e0);
        return GC_ERR_CUDA;
    }
    float best = 1e30f, best1 = 1e30f;
    gc_tuning choice = saved, choice1 = saved;
    int rc = GC_OK;
    // index = (((wu * 2 + schedule) * 3 + tile) * 3 + block) * 2 + targets per lane - 1
    for (int idx = 0; idx < GC_TUNE_COUNT && rc == GC_OK; ++idx) {
        const gc_tuning t{wus[idx / 36], (uint32_t)((idx / 18) % 2), tps[(idx / 6) % 3],
                          kbs[(idx / 2) % 3], (uint32_t)(idx % 2) + 1u};
        p->wu_max_targets = t.wu_max_targets;
        p->wu_schedule = t.schedule;
        p->wu_tile = t.tile_pairs;
        p->wu_kb = t.comp_block;
        p->wu_tpl = t.targets_per_lane;
        float tbest = 1e30f;
        for (int r = 0; r < reps && rc == GC_OK; ++r) {
            uint64_t W = 0;
            rc = rebuild_wus(p, c, t.wu_max_targets, &W);
            if (rc != GC_OK) break;
            if (W == 0) {
                rc = GC_ERR_STATE;
                break;
            }
            // the ordering pass (LPT) is part of the schedule's cost
            cudaEventRecord(e0, c.s);
            rc = gc_interact_range(p, c, 0, W, 0, 0, 0, 0, 0);
            cudaEventRecord(e1, c.s);
            if (rc != GC_OK) break;
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                rc = GC_ERR_CUDA;
                break;
            }
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < tbest) tbest = ms;
        }
        if (rc != GC_OK) break;
        if (ms_out) ms_out[idx] = tbest;
        if (tbest < best) {
            best = tbest;
            choice = t;
        }
        if (t.targets_per_lane == 1 && tbest < best1) {
            best1 = tbest;
            choice1 = t;
        }
    }
    // Two targets per lane hold fewer warps per SM, which lowers the
    // combine size (resident warps) and slows small batches: taken only
    // when more than 3 % faster than the best one-target shape
    if (choice.targets_per_lane != 1 && best1 <= best * 1.03f) {
        best = best1;
        choice = choice1;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    const gc_tuning keep = rc == GC_OK ? choice : saved;
    p->wu_max_targets = keep.wu_max_targets;
    p->wu_schedule = keep.schedule;
    p->wu_tile = keep.tile_pairs;
    p->wu_kb = keep.comp_block;
    p->wu_tpl = keep.targets_per_lane;
    if (rc != GC_OK) return rc;
    uint64_t W = 0;
    GC_TRY(rebuild_wus(p, c, choice.wu_max_targets, &W));   // context matches the choice
    GC_CUDA_TRY(cudaStreamSynchronize(c.s));
    if (best_out) *best_out = choice;
    return GC_OK;
}

// ---------------------------------------------------------------------------
// reuse ablation (Section 3.2, Fig. 3): ways of feeding the sources
// ---------------------------------------------------------------------------

extern "C" int gc_reuse_ablation(gc_pool_t *p, int reps, double out[7])
{
    if (!p || !out || reps < 1) return GC_ERR_ARG;
    if (p->last < 0 || !p->ctx[p->last].valid) return GC_ERR_NOT_READY;
    FlushCtx &c = p->ctx[p->last];
    GC_CUDA_TRY(cudaEventSynchronize(c.ev_done));
    if (c.n_waves != 1 || c.waves.size() != 1) return GC_ERR_STATE;
    const WaveRange &wv = c.waves[0];
    if (wv.w1 <= wv.w0 || wv.l1 > wv.l0) return GC_ERR_STATE;   // gravity only
    const uint64_t T = c.n_tasks, NS = c.n_src;
    const int maxb = p->num_sms * 16;
    DBuf seq_list, seq_sorted;
    int rc = GC_OK;
    if ((rc = seq_list.reserve((NS + 1) * 4)) != GC_OK ||
        (rc = seq_sorted.reserve((NS + 1) * 4)) != GC_OK) {
        seq_list.release();
        return rc;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaEventCreate(&e0);
    cudaEventCreate(&e1);
    const uint32_t saved_sched = p->wu_schedule;
    p->wu_schedule = GC_SCHED_FIFO;
    auto timed = [&](auto &&launch, double *ms_out) {
        float best = 1e30f;
        for (int r = 0; r < reps && rc == GC_OK; ++r) {
            GC_CUDA_TRY(cudaEventRecord(e0, c.s));
            rc = launch();
            GC_CUDA_TRY(cudaEventRecord(e1, c.s));
            if (rc != GC_OK) break;
            GC_CUDA_TRY(cudaEventSynchronize(e1));
            float ms = 0.f;
            cudaEventElapsedTime(&ms, e0, e1);
            if (ms < best) best = ms;
        }
        *ms_out = best;
        return rc;
    };
    // the three device modes share the work units of the batch
    InterArgs a;
    fill_inter_args(p, c, 0, 0, 0, a);
    a.wu = c.wu.as<GravWU>() + wv.w0;
    a.n_wu = wv.w1 - wv.w0;
    a.lj_list = nullptr;
    a.n_lj = 0;
    const int full = gc_grav_blocks(p);
    const unsigned g = (unsigned)std::min<uint64_t>((a.n_wu + GRAV_WARPS - 1) / GRAV_WARPS,
                                                     (uint64_t)full);
    // entry slots in list order (the address buffer) and sorted per list
    GC_TRY(gc_entry_slots(p, c.s, c.src_ids.as<uint32_t>(), NS, seq_list.as<uint32_t>()));
    k_sorted_slots<<<grid_for(T * 32, 256, maxb), 256, 0, c.s>>>(
        c.tasks.as<TaskRec>(), T, seq_list.as<uint32_t>(), c.src_perm.as<uint32_t>(),
        seq_sorted.as<uint32_t>());
    auto indirect = [&](const uint32_t *seq) {
        return [&, seq]() -> int {
            GC_CUDA_TRY(cudaMemsetAsync(a.queue, 0, sizeof(unsigned long long), c.s));
            k_gravity_indirect<<<g, GRAV_THREADS, 0, c.s>>>(a, seq, p->d_pool);
            GC_CUDA_TRY(cudaGetLastError());
            return GC_OK;
        };
    };
    timed([&]() { return gc_interact_range(p, c, wv.w0, wv.w1, 0, 0, 0, 0, 0); }, &out[0]);
    if (rc == GC_OK) timed(indirect(seq_list.as<uint32_t>()), &out[1]);
    if (rc == GC_OK) timed(indirect(seq_sorted.as<uint32_t>()), &out[2]);
    // the batch's rows end as the sorted-indirect run left them (same values
    // up to summation order)
    // redundant transfer: every list's sources gathered on the host from the
    // authoritative mirror into contiguous staging, then copied to the device
    if (rc == GC_OK) {
        std::vector<uint32_t> ids(NS);
        std::vector<TaskRec> h(T);
        if (cudaMemcpy(ids.data(), c.src_ids.p, NS * 4, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(h.data(), c.tasks.p, T * sizeof(TaskRec), cudaMemcpyDeviceToHost) !=
                cudaSuccess)
            rc = GC_ERR_CUDA;
        const uint64_t slots = NS + T;   // paired layout, one pad per task
        float4 *hst = nullptr;
        if (rc == GC_OK && cudaHostAlloc((void **)&hst, slots * sizeof(float4),
                                         cudaHostAllocDefault) != cudaSuccess)
            rc = GC_ERR_OOM;
        if (rc == GC_OK) {
            double best_g = 1e30, best_c = 1e30;
            for (int r = 0; r < reps && rc == GC_OK; ++r) {
                struct timespec t0, t1;
                clock_gettime(CLOCK_MONOTONIC, &t0);
                for (uint64_t t = 0; t < T; ++t) {
                    const TaskRec &tr = h[t];
                    float *f = reinterpret_cast<float *>(hst + tr.src_off + t);
                    for (uint32_t k = 0; k < tr.ns; ++k) {
                        const float4 v = p->h_mirror[ids[tr.src_off + k]];
                        float *d = f + 8 * (k >> 1);
                        const uint32_t hh = k & 1u;
                        d[hh] = v.x; d[2 + hh] = v.y; d[4 + hh] = v.z; d[6 + hh] = v.w;
                    }
                    if (tr.ns & 1u) {
                        float *d = f + 8 * (tr.ns >> 1);
                        d[1] = d[3] = d[5] = d[7] = 0.f;
                    }
                }
                clock_gettime(CLOCK_MONOTONIC, &t1);
                const double gms = (t1.tv_sec - t0.tv_sec) * 1e3 + (t1.tv_nsec - t0.tv_nsec) * 1e-6;
                if (gms < best_g) best_g = gms;
                cudaEventRecord(e0, c.s);
                if (cudaMemcpyAsync(c.stg_src.p, hst, slots * sizeof(float4),
                                    cudaMemcpyHostToDevice, c.s) != cudaSuccess)
                    rc = GC_ERR_CUDA;
                cudaEventRecord(e1, c.s);
                if (cudaEventSynchronize(e1) != cudaSuccess) rc = GC_ERR_CUDA;
                float cms = 0.f;
                cudaEventElapsedTime(&cms, e0, e1);
                if (cms < best_c) best_c = cms;
            }
            out[3] = best_g;
            out[4] = best_c;
            out[5] = (double)slots * sizeof(float4);
        }
        if (hst) cudaFreeHost(hst);
    }
    out[6] = (double)p->stats.last_misses * sizeof(float4);
    p->wu_schedule = saved_sched;
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    seq_list.release();
    seq_sorted.release();
    return rc;
}
