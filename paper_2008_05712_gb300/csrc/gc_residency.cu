// gc_residency.cu -- the chare table (Section 3.2 of Rengasamy & Vadhiyar,
// arXiv 2008.05712): maps data ids to device slots so that data already on
// the device is reused and only missing data crosses the host link.
//
// Per flush wave (all steps on the device, one small counter read-back):
//   1. mark every referenced id with the wave's epoch and count references,
//   2. list the distinct ids: for a wave of many entries, in ascending order
//      by an order-preserving compaction over the id space; for a wave of
//      few entries (fewer than a sixteenth of the id range), as the marking
//      finds them, so the wave costs its entries and not the id range,
//   3. split them into hits (resident) and misses (read back with the
//      counters: one host round trip), misses then in ascending id order,
//   4. if misses exceed the free slots (counted on the host), evict the
//      resident ids not referenced now in ascending (last use, slot) order,
//      writing their values back to the host mirror; list the free slots in
//      ascending order,
//   5. give the i-th smallest missing id the i-th smallest free slot and
//      fetch its value from the pinned host mirror (mapped memory, read by
//      the kernel over the CPU-GPU link),
//   6. stamp last use.
#include <algorithm>

#include "gc_common.cuh"

namespace {

constexpr int CT_THREADS = 256;
constexpr int CT_ITEMS = 16;
constexpr int CT_TILE = CT_THREADS * CT_ITEMS;

struct CompactArgs {
    int kind;
    uint64_t n;                   // host bound
    const unsigned long long *count_dev;   // optional device bound
    const uint32_t *arr;
    const uint32_t *ref_epoch;
    const uint32_t *slot_of_id;
    const uint32_t *id_of_slot;
    uint32_t epoch;
};

__device__ __forceinline__ uint64_t ca_limit(const CompactArgs &a)
{
    uint64_t lim = a.n;
    if (a.count_dev) {
        uint64_t c = *a.count_dev;
        if (c < lim) lim = c;
    }
    return lim;
}

__device__ __forceinline__ bool ca_pred(const CompactArgs &a, uint64_t i, uint32_t &val)
{
    switch (a.kind) {
    case CK_REF_EPOCH:
        val = (uint32_t)i;
        return a.ref_epoch[i] == a.epoch;
    case CK_MISS: {
        uint32_t id = a.arr[i];
        val = id;
        return a.slot_of_id[id] == GC_NONE;
    }
    case CK_FREE:
        val = (uint32_t)i;
        return a.id_of_slot[i] == GC_NONE;
    default:  // CK_RUN_START
        val = (uint32_t)i;
        return i == 0 || a.arr[i] != a.arr[i - 1];
    }
}

__device__ __forceinline__ uint32_t block_excl_scan(uint32_t v, uint32_t *total)
{
    __shared__ uint32_t warp_sums[CT_THREADS / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[w] = x;
    __syncthreads();
    if (w == 0) {
        uint32_t s = (lane < CT_THREADS / 32) ? warp_sums[lane] : 0;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        if (lane < CT_THREADS / 32) warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t before = (w > 0 ? warp_sums[w - 1] : 0) + x - v;
    if (total) *total = warp_sums[CT_THREADS / 32 - 1];
    __syncthreads();
    return before;
}

__global__ void k_compact_count(CompactArgs a, uint32_t *tile_cnt)
{
    uint64_t lim = ca_limit(a);
    uint64_t base = (uint64_t)blockIdx.x * CT_TILE + (uint64_t)threadIdx.x * CT_ITEMS;
    uint32_t c = 0, v;
    for (int j = 0; j < CT_ITEMS; ++j) {
        uint64_t i = base + j;
        if (i < lim && ca_pred(a, i, v)) ++c;
    }
    uint32_t tot;
    block_excl_scan(c, &tot);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = tot;
}

// Single-block exclusive scan of the tile counts; total to *count_out.
__global__ void k_compact_scan(uint32_t *tile_cnt, uint64_t n_tiles,
                               unsigned long long *count_out)
{
    uint32_t carry = 0;
    for (uint64_t b = 0; b < n_tiles; b += CT_THREADS) {
        uint64_t i = b + threadIdx.x;
        uint32_t v = (i < n_tiles) ? tile_cnt[i] : 0;
        uint32_t tot;
        uint32_t ex = block_excl_scan(v, &tot);
        if (i < n_tiles) tile_cnt[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0) *count_out = carry;
}

__global__ void k_compact_write(CompactArgs a, const uint32_t *tile_off, uint32_t *out)
{
    uint64_t lim = ca_limit(a);
    uint64_t base = (uint64_t)blockIdx.x * CT_TILE + (uint64_t)threadIdx.x * CT_ITEMS;
    uint32_t flags = 0, v;
    for (int j = 0; j < CT_ITEMS; ++j) {
        uint64_t i = base + j;
        if (i < lim && ca_pred(a, i, v)) flags |= 1u << j;
    }
    uint32_t pos = tile_off[blockIdx.x] + block_excl_scan(__popc(flags), nullptr);
    for (int j = 0; j < CT_ITEMS; ++j) {
        if (flags & (1u << j)) {
            ca_pred(a, base + j, v);
            out[pos++] = v;
        }
    }
}

// ---- residency kernels ------------------------------------------------------

// Reference marking and counting.  Each block takes a contiguous chunk of
// entries (neighbouring tasks share many ids: the far tree nodes appear in
// almost every list), aggregates reference counts in a small shared-memory
// hash table and adds them to the global counters once per block; ids that
// do not find a table slot fall back to global atomics.  Only the thread
// that enters an id into the table (or finds no place for it) reads and
// moves the id's reference word: a chunk of 8192 N-body entries holds about
// 1900 distinct ids.  With `ent` set, the
// entry's current slot is recorded too (wave-local entry order: targets,
// then sources; NONE for an id not resident yet): the slot is read beside
// the reference word, in parallel with it, so the pack that follows reads
// the slots of its entries in order instead of looking each one up.  A hit
// keeps its slot through the rest of the chare-table step (only ids not
// referenced now are evicted); a miss is looked up again by the pack.  With
// `first` set, the thread that moves an id's reference word to the wave's
// epoch appends the id to `first` (the distinct ids of the wave, in no
// particular order, counted in ctr[CTR_UNIQUE]).
constexpr int MARK_HASH_BITS = 12;
constexpr int MARK_HASH = 1 << MARK_HASH_BITS;   // about twice the distinct ids of a chunk

__global__ void k_mark(const uint32_t *tgt, uint64_t nt, const uint32_t *src, uint64_t ns,
                       uint64_t id_cap, uint32_t *ref_epoch,
                       uint32_t *ref_count, uint32_t epoch, unsigned long long *ctr,
                       uint64_t chunk, const uint32_t *slot_of_id, uint32_t *ent,
                       uint32_t *first)
{
    __shared__ uint32_t hkey[MARK_HASH];
    __shared__ uint32_t hcnt[MARK_HASH];
    for (int i = threadIdx.x; i < MARK_HASH; i += blockDim.x) {
        hkey[i] = GC_NONE;
        hcnt[i] = 0;
    }
    __syncthreads();
    const uint64_t n = nt + ns;
    const uint64_t b0 = (uint64_t)blockIdx.x * chunk;
    const uint64_t b1 = min(n, b0 + chunk);
    bool bad = false;
    for (uint64_t e = b0 + threadIdx.x; e < b1; e += blockDim.x) {
        const uint32_t id = e < nt ? tgt[e] : src[e - nt];
        if ((uint64_t)id >= id_cap) {
            bad = true;
            continue;
        }
        if (ent) ent[e] = slot_of_id[id];
        // count the reference in the block's table; the thread that puts the
        // id there (or finds no place for it) marks it, the others skip it
        uint32_t h = (id * 2654435761u) >> (32 - MARK_HASH_BITS);   // top bits of the product
        bool counted = false, inserted = false;
        for (int probe = 0; probe < 8; ++probe) {
            uint32_t k = hkey[h];
            if (k == GC_NONE) {
                k = atomicCAS(&hkey[h], GC_NONE, id);
                inserted = k == GC_NONE;
            }
            if (k == GC_NONE || k == id) {
                atomicAdd(&hcnt[h], 1u);
                counted = true;
                break;
            }
            h = (h + 1) & (MARK_HASH - 1);
        }
        bool is_first = false;
        bool known = true;
        if (inserted || !counted) {
            const uint32_t e0 = ref_epoch[id];   // one word: uploaded? referenced this wave?
            if (e0 == GC_EPOCH_UNKNOWN) {
                bad = true;
                known = false;
                if (counted) atomicOr(&hcnt[h], 0x80000000u);   // never uploaded: not counted
            } else if (e0 != epoch) {
                if (first) is_first = atomicExch(&ref_epoch[id], epoch) != epoch;
                else ref_epoch[id] = epoch;
            }
        }
        if (first) {
            // one counter add per warp for the ids it sees first
            const unsigned am = __activemask();
            const unsigned fm = __ballot_sync(am, is_first);
            if (fm) {
                const int lane = threadIdx.x & 31, leader = __ffs((int)fm) - 1;
                unsigned long long at = 0;
                if (lane == leader) at = atomicAdd(&ctr[CTR_UNIQUE], (unsigned long long)__popc(fm));
                at = __shfl_sync(am, at, leader);
                if (is_first) first[at + __popc(fm & ((1u << lane) - 1u))] = id;
            }
        }
        if (!counted && known) atomicAdd(&ref_count[id], 1u);
    }
    if (bad) atomicOr(&ctr[CTR_FLAGS], (unsigned long long)GC_FLAG_UNKNOWN_ID);
    __syncthreads();
    for (int i = threadIdx.x; i < MARK_HASH; i += blockDim.x)
        if (hkey[i] != GC_NONE && !(hcnt[i] & 0x80000000u)) atomicAdd(&ref_count[hkey[i]], hcnt[i]);
}

__device__ __forceinline__ int hist_bin(uint32_t c)
{
    if (c <= 1) return 0;
    if (c == 2) return 1;
    int b = 32 - __clz(c - 1);   // ceil(log2 c)
    return b > 7 ? 7 : b;        // 3-4 -> 2, 5-8 -> 3, ..., >64 -> 7
}

__global__ void k_classify(const uint32_t *uniq, const unsigned long long *count_dev,
                           const uint32_t *slot_of_id, uint32_t *ref_count,
                           unsigned long long *ctr)
{
    __shared__ unsigned int hist[8];
    __shared__ unsigned int hits;
    if (threadIdx.x < 8) hist[threadIdx.x] = 0;
    if (threadIdx.x == 0) hits = 0;
    __syncthreads();
    // counts kept per thread and summed per warp at the end: one shared-
    // memory add per id made every thread of a block wait on the same few
    // words
    uint32_t h[8] = {0u, 0u, 0u, 0u, 0u, 0u, 0u, 0u};
    uint32_t nh = 0;
    uint64_t U = *count_dev;
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < U;
         k += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t id = uniq[k];
        uint32_t c = ref_count[id];
        ref_count[id] = 0;
        const int bin = hist_bin(c);
#pragma unroll
        for (int q = 0; q < 8; ++q) h[q] += bin == q ? 1u : 0u;
        nh += slot_of_id[id] != GC_NONE ? 1u : 0u;
    }
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
        uint32_t v = q < 8 ? h[q] : nh;
        for (int o = 16; o; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && v) atomicAdd(q < 8 ? &hist[q] : &hits, v);
    }
    __syncthreads();
    if (threadIdx.x < 8 && hist[threadIdx.x])
        atomicAdd(&ctr[CTR_HIST0 + threadIdx.x], (unsigned long long)hist[threadIdx.x]);
    if (threadIdx.x == 0 && hits) atomicAdd(&ctr[CTR_HITS], (unsigned long long)hits);
}

__global__ void k_evict_keys(uint64_t cap, const uint32_t *id_of_slot,
                             const uint32_t *ref_epoch, const uint32_t *last_use,
                             uint32_t epoch, uint64_t *keys)
{
    for (uint64_t s = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; s < cap;
         s += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t id = id_of_slot[s];
        uint64_t k = ~0ull;
        if (id != GC_NONE && ref_epoch[id] != epoch)
            k = ((uint64_t)last_use[s] << 32) | (uint64_t)s;
        keys[s] = k;
    }
}

__global__ void k_evict_apply(const uint64_t *sorted, uint64_t need, uint32_t *id_of_slot,
                              uint32_t *slot_of_id, const float4 *pool, float4 *mirror,
                              uint32_t *evicted)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < need;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t s = (uint32_t)(sorted[i] & 0xFFFFFFFFu);
        uint32_t id = id_of_slot[s];
        mirror[id] = pool[s];          // write back: the slot held the current value
        slot_of_id[id] = GC_NONE;
        id_of_slot[s] = GC_NONE;
        evicted[i] = id;
    }
}

__global__ void k_assign(const uint32_t *miss, uint64_t M, const uint32_t *freel,
                         uint32_t *slot_of_id, uint32_t *id_of_slot, float4 *pool,
                         const float4 *mirror)
{
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < M;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t id = miss[i], s = freel[i];
        slot_of_id[id] = s;
        id_of_slot[s] = id;
        pool[s] = mirror[id];          // fetch over the host link (mapped memory)
    }
}

__global__ void k_touch(const uint32_t *uniq, uint64_t U, const uint32_t *slot_of_id,
                        uint32_t *last_use, uint32_t epoch)
{
    for (uint64_t k = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; k < U;
         k += (uint64_t)gridDim.x * blockDim.x)
        last_use[slot_of_id[uniq[k]]] = epoch;
}

__global__ void k_entry_slots(const uint32_t *ids, uint64_t n, const uint32_t *slot_of_id,
                              uint32_t *out)
{
    for (uint64_t e = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; e < n;
         e += (uint64_t)gridDim.x * blockDim.x)
        out[e] = slot_of_id[ids[e]];
}

__global__ void k_upload(const uint32_t *ids, uint32_t id_base, const float4 *vals, uint64_t n,
                         uint64_t id_cap,
                         const uint32_t *slot_of_id, float4 *pool, float4 *mirror,
                         uint32_t *ref_epoch, int write_mirror, unsigned long long *ctr)
{
    __shared__ unsigned int upd;
    if (threadIdx.x == 0) upd = 0;
    __syncthreads();
    for (uint64_t i = blockIdx.x * (uint64_t)blockDim.x + threadIdx.x; i < n;
         i += (uint64_t)gridDim.x * blockDim.x) {
        uint32_t id = ids ? ids[i] : id_base + (uint32_t)i;
        if ((uint64_t)id >= id_cap) {
            atomicOr(&ctr[CTR_FLAGS], (unsigned long long)GC_FLAG_ID_RANGE);
            continue;
        }
        float4 v = vals[i];
        if (ref_epoch[id] == GC_EPOCH_UNKNOWN) ref_epoch[id] = 0;   // known, never referenced
        uint32_t s = slot_of_id[id];
        if (s != GC_NONE) {
            pool[s] = v;
            atomicAdd(&upd, 1u);
        } else if (write_mirror) {
            mirror[id] = v;
        }
    }
    __syncthreads();
    if (threadIdx.x == 0 && upd) atomicAdd(&ctr[CTR_UPDATES], (unsigned long long)upd);
}

}  // namespace

// Slots of the given ids (introspection of the chare table).
int gc_entry_slots(gc_pool *p, cudaStream_t s, const uint32_t *ids, uint64_t n, uint32_t *out)
{
    if (n == 0) return GC_OK;
    ++p->stats.kernel_launches;
    k_entry_slots<<<grid_for(n, 256, p->num_sms * 16), 256, 0, s>>>(ids, n, p->d_slot_of_id,
                                                                    out);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

int gc_compact(gc_pool *p, DBuf &tiles, cudaStream_t s, int kind, uint64_t n_bound,
               const uint64_t *count_dev, const uint32_t *arr, uint32_t *out,
               unsigned long long *count_out)
{
    uint64_t n_tiles = (n_bound + CT_TILE - 1) / CT_TILE;
    if (n_tiles == 0) {
        GC_CUDA_TRY(cudaMemsetAsync(count_out, 0, sizeof(unsigned long long), s));
        return GC_OK;
    }
    GC_TRY(tiles.reserve(n_tiles * sizeof(uint32_t)));
    CompactArgs a;
    a.kind = kind;
    a.n = n_bound;
    a.count_dev = reinterpret_cast<const unsigned long long *>(count_dev);
    a.arr = arr;
    a.ref_epoch = p->d_ref_epoch;
    a.slot_of_id = p->d_slot_of_id;
    a.id_of_slot = p->d_id_of_slot;
    a.epoch = p->epoch;
    ++p->stats.kernel_launches;
    k_compact_count<<<(unsigned)n_tiles, CT_THREADS, 0, s>>>(a, tiles.as<uint32_t>());
    ++p->stats.kernel_launches;
    k_compact_scan<<<1, CT_THREADS, 0, s>>>(tiles.as<uint32_t>(), n_tiles, count_out);
    ++p->stats.kernel_launches;
    k_compact_write<<<(unsigned)n_tiles, CT_THREADS, 0, s>>>(a, tiles.as<uint32_t>(), out);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

int gc_launch_upload(gc_pool *p, const uint32_t *ids, const float4 *vals, uint64_t n,
                     int write_mirror)
{
    if (n == 0) return GC_OK;
    ++p->stats.kernel_launches;
    k_upload<<<grid_for(n, 256, p->num_sms * 16), 256, 0, p->s>>>(
        ids, 0, vals, n, p->cfg.id_capacity, p->d_slot_of_id, p->d_pool, p->d_mirror,
        p->d_ref_epoch, write_mirror, p->d_ctr);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

// Device upload of ids id_base .. id_base + n - 1 (values written through to
// the host mirror for non-resident ids).
int gc_launch_upload_seq(gc_pool *p, uint32_t id_base, const float4 *vals, uint64_t n)
{
    if (n == 0) return GC_OK;
    ++p->stats.kernel_launches;
    k_upload<<<grid_for(n, 256, p->num_sms * 16), 256, 0, p->s>>>(
        nullptr, id_base, vals, n, p->cfg.id_capacity, p->d_slot_of_id, p->d_pool,
        p->d_mirror, p->d_ref_epoch, 1, p->d_ctr);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

// Steps 1-3 on the device and the counters' copy to the host (no wait).
int gc_residency_issue(gc_pool *p, const uint32_t *tgt, uint64_t nt, const uint32_t *src,
                       uint64_t ns, uint32_t *ent)
{
    const uint64_t id_cap = p->cfg.id_capacity;
    const uint64_t n = nt + ns;
    unsigned long long *ctr = p->d_ctr;
    p->epoch += 1;
    if (p->epoch == 0 || p->epoch == GC_EPOCH_UNKNOWN) p->epoch = 1;   // reserved values
    const int maxb = p->num_sms * 16;

    GC_CUDA_TRY(cudaMemsetAsync(ctr + CTR_UNIQUE, 0,
                                sizeof(unsigned long long) * (CTR_COUNT - CTR_UNIQUE), p->s));
    // a wave of few entries lists its distinct ids while marking them
    const bool few = n * 16 < id_cap;
    uint64_t ubound = n < id_cap ? n : id_cap;
    GC_TRY(p->uniq.reserve((ubound + 1) * sizeof(uint32_t)));
    GC_TRY(p->miss.reserve((ubound + 1) * sizeof(uint32_t)));
    if (n > 0) {
        // chunks of 8192 entries (neighbouring lists share ids, so a block's
        // table aggregates well); a small wave in chunks of at least 1024
        // spread over more SMs
        uint64_t chunk = (n + (uint64_t)p->num_sms * 4 - 1) / ((uint64_t)p->num_sms * 4);
        chunk = std::min<uint64_t>(8192, std::max<uint64_t>(1024, (chunk + 511) / 512 * 512));
        ++p->stats.kernel_launches;
        k_mark<<<(unsigned)((n + chunk - 1) / chunk), 512, 0, p->s>>>(
            tgt, nt, src, ns, id_cap, p->d_ref_epoch, p->d_ref_count, p->epoch, ctr,
            chunk, p->d_slot_of_id, ent, few ? p->uniq.as<uint32_t>() : nullptr);
    }
    if (!few)
        GC_TRY(gc_compact(p, p->tiles, p->s, CK_REF_EPOCH, id_cap, nullptr, nullptr,
                          p->uniq.as<uint32_t>(), ctr + CTR_UNIQUE));
    ++p->stats.kernel_launches;
    k_classify<<<grid_for(ubound, 256, maxb), 256, 0, p->s>>>(
        p->uniq.as<uint32_t>(), ctr + CTR_UNIQUE, p->d_slot_of_id, p->d_ref_count, ctr);
    GC_TRY(gc_compact(p, p->tiles, p->s, CK_MISS, ubound, (const uint64_t *)(ctr + CTR_UNIQUE),
                      p->uniq.as<uint32_t>(), p->miss.as<uint32_t>(), ctr + CTR_MISSES));
    GC_CUDA_TRY(cudaMemcpyAsync(p->h_ctr, ctr, sizeof(unsigned long long) * CTR_COUNT,
                                cudaMemcpyDeviceToHost, p->s));
    p->res_n = n;
    p->res_few = few;
    return GC_OK;
}

// Steps 3-6 once the counters issued by gc_residency_issue have reached the
// host (the caller has waited for the stream).
int gc_residency_finish(gc_pool *p)
{
    const uint64_t id_cap = p->cfg.id_capacity, cap = p->cfg.pool_capacity;
    const uint64_t n = p->res_n;
    const bool few = p->res_few;
    unsigned long long *ctr = p->d_ctr;
    const int maxb = p->num_sms * 16;
    GC_CUDA_TRY(cudaGetLastError());

    // this step's own status bits; a timeout of an earlier batch stays for
    // gc_wait to report
    const unsigned long long flags = p->h_ctr[CTR_FLAGS] & (GC_FLAG_UNKNOWN_ID | GC_FLAG_ID_RANGE);
    if (flags) {
        GC_TRY(gc_clear_flags(p, p->s, GC_FLAG_UNKNOWN_ID | GC_FLAG_ID_RANGE));
        return GC_ERR_UNKNOWN_ID;
    }
    const uint64_t U = p->h_ctr[CTR_UNIQUE], H = p->h_ctr[CTR_HITS];
    const uint64_t M = p->h_ctr[CTR_MISSES], F = p->free_slots;
    uint64_t need = M > F ? M - F : 0;
    p->n_evicted_last = 0;
    const uint32_t *miss = p->miss.as<uint32_t>();
    if (few && M > 1) {
        // misses take free slots in ascending id order
        GC_TRY(p->miss_sorted.reserve((M + 1) * sizeof(uint32_t)));
        int bits = 1;
        while (bits < 32 && ((uint64_t)1 << bits) < id_cap) ++bits;
        ++p->stats.primitive_calls;
        GC_TRY(gc_sort_keys_u32(p->cub_tmp, miss, p->miss_sorted.as<uint32_t>(), M, bits, p->s));
        miss = p->miss_sorted.as<uint32_t>();
    }
    if (M) GC_TRY(p->freel.reserve((cap + 1) * sizeof(uint32_t)));
    if (need) {
        uint64_t resident = cap - F;
        uint64_t candidates = resident - H;
        if (candidates < need) return GC_ERR_POOL_FULL;
        GC_TRY(p->ekeys.reserve(cap * sizeof(uint64_t)));
        GC_TRY(p->ekeys2.reserve(cap * sizeof(uint64_t)));
        GC_TRY(p->evicted.reserve(need * sizeof(uint32_t)));
        ++p->stats.kernel_launches;
        k_evict_keys<<<grid_for(cap, 256, maxb), 256, 0, p->s>>>(
            cap, p->d_id_of_slot, p->d_ref_epoch, p->d_last_use, p->epoch,
            p->ekeys.as<uint64_t>());
        ++p->stats.primitive_calls;
        GC_TRY(gc_sort_keys_u64(p->cub_tmp, p->ekeys.as<uint64_t>(), p->ekeys2.as<uint64_t>(),
                                cap, p->s));
        ++p->stats.kernel_launches;
        k_evict_apply<<<grid_for(need, 256, maxb), 256, 0, p->s>>>(
            p->ekeys2.as<uint64_t>(), need, p->d_id_of_slot, p->d_slot_of_id, p->d_pool,
            p->d_mirror, p->evicted.as<uint32_t>());
        p->n_evicted_last = need;
    }
    if (M || need) ++p->table_version;   // slots assigned or freed: captured graphs stale
    if (M) {
        GC_TRY(gc_compact(p, p->tiles, p->s, CK_FREE, cap, nullptr, nullptr,
                          p->freel.as<uint32_t>(), ctr + CTR_FREE));
        ++p->stats.kernel_launches;
        k_assign<<<grid_for(M, 256, maxb), 256, 0, p->s>>>(
            miss, M, p->freel.as<uint32_t>(), p->d_slot_of_id, p->d_id_of_slot, p->d_pool,
            p->d_mirror);
    }
    p->free_slots = F + need - M;
    if (U) {
        ++p->stats.kernel_launches;
        k_touch<<<grid_for(U, 256, maxb), 256, 0, p->s>>>(p->uniq.as<uint32_t>(), U,
                                                          p->d_slot_of_id, p->d_last_use,
                                                          p->epoch);
    }
    GC_CUDA_TRY(cudaGetLastError());

    gc_stats_t &st = p->stats;
    st.entries += n;
    st.unique += U;
    st.hits += H;
    st.misses += M;
    st.evictions += need;
    st.h2d_bytes += M * sizeof(float4);
    st.last_unique += U;
    st.last_hits += H;
    st.last_misses += M;
    st.last_evictions += need;
    for (int b = 0; b < 8; ++b) st.reuse_hist[b] += p->h_ctr[CTR_HIST0 + b];
    return GC_OK;
}

int gc_residency(gc_pool *p, const uint32_t *tgt, uint64_t nt, const uint32_t *src,
                 uint64_t ns, uint32_t *ent)
{
    GC_TRY(gc_residency_issue(p, tgt, nt, src, ns, ent));
    GC_CUDA_TRY(cudaStreamSynchronize(p->s));
    return gc_residency_finish(p);
}
