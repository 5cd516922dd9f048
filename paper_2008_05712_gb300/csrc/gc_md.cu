// gc_md.cu -- MD task builder on the device (Section 4.2: the space is
// split into patches (here cubic periodic cells of edge >= cutoff) that own
// their atoms; a compute object per pair of neighbouring patches calls
// interact() on the two atom vectors and updates the forces of both).
//
// Cells: a stable sort of the atoms by cell index gives each cell's atoms in
// ascending atom id; cell_start comes from the sorted keys.  Tasks: for
// every cell in ascending index, its self task, then one task per
// neighbour offset in the upper half-shell (13 offsets lexicographically
// above (0,0,0), dx most significant), so every pair of neighbouring cells
// is visited exactly once.
#include "gc_common.cuh"
#include "gc_ptx.cuh"

namespace {

// task slot o = 1..13 -> neighbour offset; slot 0 is the self task
__constant__ int8_t c_half_shell[13][3] = {
    {0, 0, 1},  {0, 1, -1},  {0, 1, 0},  {0, 1, 1},  {1, -1, -1}, {1, -1, 0}, {1, -1, 1},
    {1, 0, -1}, {1, 0, 0},   {1, 0, 1},  {1, 1, -1}, {1, 1, 0},   {1, 1, 1}};
// the planar grid (the paper's two-dimensional MD): slots 1..4
__constant__ int8_t c_half_ring[4][3] = {{0, 1, 0}, {1, -1, 0}, {1, 0, 0}, {1, 1, 0}};

// tasks per cell: self + half of the 3^dim - 1 neighbours
__host__ __device__ constexpr int tasks_per_cell(int dim) { return dim == 2 ? 5 : 14; }

__global__ void k_cell_keys(const uint32_t *cell, uint64_t n, uint32_t n_cells, uint32_t *keys,
                            uint32_t *ids, unsigned long long *ctr)
{
    GRID_STRIDE(i, n) {
        uint32_t c = cell[i];
        if (c >= n_cells) {
            atomicOr(&ctr[CTR_FLAGS], (unsigned long long)GC_FLAG_ID_RANGE);
            c = n_cells - 1;
        }
        keys[i] = c;
        ids[i] = (uint32_t)i;
    }
}

// cell_start[c] = first sorted index with key >= c, for c = 0 .. n_cells
__global__ void k_cell_start(const uint32_t *keys, uint64_t n, uint32_t n_cells,
                             uint32_t *start)
{
    GRID_STRIDE(i, n + 1) {
        // cells c with keys[i-1] < c <= keys[i] start at i (keys[-1] = -1,
        // keys[n] = n_cells)
        uint32_t lo = (i == 0) ? 0u : keys[i - 1] + 1u;
        uint32_t hi = (i == n) ? n_cells : keys[i];
        for (uint32_t c = lo; c <= hi; ++c) start[c] = (uint32_t)i;
    }
}

__device__ __forceinline__ void task_cells(uint64_t t, int m, int dim, uint32_t &ca,
                                           uint32_t &cb, int8_t d[3], bool &self)
{
    const int per = tasks_per_cell(dim);
    uint64_t c = t / per;
    int o = (int)(t % per);
    ca = (uint32_t)c;
    self = (o == 0);
    if (self) {
        cb = ca;
        d[0] = d[1] = d[2] = 0;
        return;
    }
    if (dim == 2) {
        int x = (int)(c % m), y = (int)(c / m);
        d[0] = c_half_ring[o - 1][0];
        d[1] = c_half_ring[o - 1][1];
        d[2] = 0;
        cb = (uint32_t)((x + d[0] + m) % m + m * ((y + d[1] + m) % m));
        return;
    }
    int x = (int)(c % m), y = (int)((c / m) % m), z = (int)(c / ((uint64_t)m * m));
    d[0] = c_half_shell[o - 1][0];
    d[1] = c_half_shell[o - 1][1];
    d[2] = c_half_shell[o - 1][2];
    int bx = (x + d[0] + m) % m, by = (y + d[1] + m) % m, bz = (z + d[2] + m) % m;
    cb = (uint32_t)(bx + m * (by + m * bz));
}

__global__ void k_md_counts(uint64_t nt, int m, int dim, const uint32_t *start, uint64_t *cnt_t,
                            uint64_t *cnt_s)
{
    GRID_STRIDE(t, nt + 1) {
        if (t == nt) {
            cnt_t[t] = 0;
            cnt_s[t] = 0;
            continue;
        }
        uint32_t ca, cb;
        int8_t d[3];
        bool self;
        task_cells(t, m, dim, ca, cb, d, self);
        cnt_t[t] = start[ca + 1] - start[ca];
        cnt_s[t] = self ? 0 : (start[cb + 1] - start[cb]);
    }
}

__global__ void k_md_fill(uint64_t nt, int m, int dim, const uint32_t *start,
                          const uint32_t *atoms,
                          const uint64_t *off_t, const uint64_t *off_s, uint64_t tgt_base,
                          uint64_t src_base, uint64_t id_base, uint32_t *tgt, uint32_t *src,
                          TaskRec *recs)
{
    GRID_STRIDE(t, nt) {
        uint32_t ca, cb;
        int8_t d[3];
        bool self;
        task_cells(t, m, dim, ca, cb, d, self);
        uint32_t a0 = start[ca], a1 = start[ca + 1];
        uint32_t b0 = start[cb], b1 = self ? start[cb] : start[cb + 1];
        uint64_t ot = off_t[t], os = off_s[t];
        for (uint32_t q = a0; q < a1; ++q) tgt[ot + (q - a0)] = atoms[q];
        for (uint32_t q = b0; q < b1; ++q) src[os + (q - b0)] = atoms[q];
        TaskRec r;
        r.task_id = id_base + t;
        r.tgt_off = tgt_base + ot;
        r.src_off = src_base + os;
        r.row_off = 0;
        r.kind = self ? GC_LJ_SELF : GC_LJ_PAIR;
        r.nt = a1 - a0;
        r.ns = b1 - b0;
        r.shift[0] = d[0];
        r.shift[1] = d[1];
        r.shift[2] = d[2];
        r.shift[3] = 0;
        recs[t] = r;
    }
}

// Per-id accumulation of one MD build's rows without a sort.  An atom of
// cell c has one row in each task touching c: c's self task and its
// half-shell tasks (c's atoms are their targets) and the half-shell tasks of
// the cells whose offset lands on c (c's atoms are their sources, after the
// targets).  One warp per cell ranks those tasks by index, so every atom's
// rows are summed in ascending row order -- the order of the general path,
// which sorts the rows by id -- with the same FP64 arithmetic: the totals
// are bit-identical to it.  A lane holds one component of one atom; a
// cell's rows in one task are consecutive, so the warp reads whole row
// ranges.  The FP64 adds bound the kernel (the FP64 pipe runs at a small
// fraction of the FP32 rate), so all 32 lanes carry them.
template <int DIM>
__global__ void k_reduce_md(const TaskRec *tasks, uint32_t n_cells, int m,
                            const uint32_t *row_id, const float4 *res, gcd4 *totals)
{
    constexpr int PER = tasks_per_cell(DIM);
    constexpr int NREF = 2 * PER - 1;
    static_assert(NREF <= 32, "one lane per task touching the cell");
    const unsigned FULL = 0xffffffffu;
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t nw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t c = gw; c < n_cells; c += nw) {
        // lane j < NREF: a task touching c and the first row of c's atoms in it
        uint64_t tj = ~0ull, rb = 0;
        if (lane < PER) {
            tj = (uint64_t)PER * c + (uint64_t)lane;
            rb = tasks[tj].row_off;
        } else if (lane < NREF) {
            const int o = lane - PER + 1;
            uint32_t cp;
            if (DIM == 2) {
                const int x = (int)(c % m), y = (int)(c / m);
                cp = (uint32_t)((x - c_half_ring[o - 1][0] + m) % m +
                                m * ((y - c_half_ring[o - 1][1] + m) % m));
            } else {
                const int x = (int)(c % m), y = (int)((c / m) % m),
                          z = (int)(c / ((uint64_t)m * m));
                cp = (uint32_t)((x - c_half_shell[o - 1][0] + m) % m +
                                m * ((y - c_half_shell[o - 1][1] + m) % m +
                                     m * ((z - c_half_shell[o - 1][2] + m) % m)));
            }
            tj = (uint64_t)PER * cp + (uint64_t)o;
            const TaskRec r = tasks[tj];
            rb = r.row_off + r.nt;
        }
        // ranks by task index (distinct); lane r then takes the rank-r task
        uint32_t rank = 0;
#pragma unroll
        for (int k = 0; k < NREF; ++k) rank += __shfl_sync(FULL, tj, k) < tj ? 1u : 0u;
        int src = 0;
#pragma unroll
        for (int r = 0; r < NREF; ++r) {
            const uint32_t b = __ballot_sync(FULL, lane < NREF && rank == (uint32_t)r);
            if (lane == r) src = __ffs(b) - 1;
        }
        const uint64_t base_r = __shfl_sync(FULL, rb, src);
        const TaskRec self = tasks[(uint64_t)PER * c];
        // lane = (atom, component): eight atoms per step keep every lane's
        // FP64 adds busy (cells hold about fourteen atoms)
        const int comp = lane & 3;
        for (uint32_t a0 = 0; a0 < self.nt; a0 += 8) {
            const uint32_t i = a0 + (uint32_t)(lane >> 2);
            const bool v = i < self.nt;
            const uint32_t id = v ? row_id[self.row_off + i] : 0u;
            double *tot = reinterpret_cast<double *>(totals + id) + comp;
            double acc = v ? *tot : 0.0;
#pragma unroll 9
            for (int r = 0; r < NREF; ++r) {
                const uint64_t row = __shfl_sync(FULL, base_r, r) + i;
                if (v) {
                    const float sv = reinterpret_cast<const float *>(res + 2 * row)[comp];
                    const float cv = reinterpret_cast<const float *>(res + 2 * row + 1)[comp];
                    acc += gc_f2d(sv) - gc_f2d(cv);
                }
            }
            if (v) *tot = acc;
        }
    }
}

}  // namespace

uint64_t gc_md_tasks(int m, int dim)
{
    const uint64_t cells = dim == 2 ? (uint64_t)m * m : (uint64_t)m * m * m;
    return (uint64_t)tasks_per_cell(dim) * cells;
}

int gc_md_reduce(gc_pool *p, FlushCtx &c)
{
    const int m = c.md_m;
    const uint32_t n_cells = c.md_dim == 2 ? (uint32_t)m * m : (uint32_t)m * m * m;
    const unsigned grid = grid_for((uint64_t)n_cells * 32, 256, p->num_sms * 16);
    ++p->stats.kernel_launches;
    if (c.md_dim == 2)
        k_reduce_md<2><<<grid, 256, 0, c.s>>>(c.tasks.as<TaskRec>(), n_cells, m,
                                              c.row_id.as<uint32_t>(), c.res.as<float4>(),
                                              p->d_totals);
    else
        k_reduce_md<3><<<grid, 256, 0, c.s>>>(c.tasks.as<TaskRec>(), n_cells, m,
                                              c.row_id.as<uint32_t>(), c.res.as<float4>(),
                                              p->d_totals);
    GC_CUDA_TRY(cudaGetLastError());
    return GC_OK;
}

static int build_md(gc_pool_t *p, const uint32_t *cell_dev, uint64_t n, int m, int dim,
                    uint64_t task_id_base, uint64_t info_out[4])
{
    if (!p || !cell_dev || n == 0 || n > 0x7FFFFFFFull || m < 3 ||
        m > (dim == 2 ? 32768 : 1024))
        return GC_ERR_ARG;
    if (n > p->cfg.id_capacity) return GC_ERR_POOL_FULL;
    MDState &S = p->md;
    int vrc = GC_OK;
    cell_dev = (const uint32_t *)gc_device_view(p, cell_dev, n * sizeof(uint32_t), S.hostcopy,
                                                &vrc);
    if (vrc != GC_OK) return vrc;
    cudaStream_t s = p->s;
    const uint32_t n_cells = dim == 2 ? (uint32_t)m * m : (uint32_t)m * m * m;
    const uint64_t nt = (uint64_t)tasks_per_cell(dim) * n_cells;
    const int maxb = p->num_sms * 16;
    GC_TRY(S.keys.reserve(n * 4));
    GC_TRY(S.keys2.reserve(n * 4));
    GC_TRY(S.ids.reserve(n * 4));
    GC_TRY(S.ids2.reserve(n * 4));
    GC_TRY(S.cell_start.reserve(((uint64_t)n_cells + 1) * 4));
    GC_TRY(S.cnt_t.reserve((nt + 1) * 8 * 2));
    GC_TRY(S.cnt_s.reserve((nt + 1) * 8 * 2));
    ++p->stats.kernel_launches;
    k_cell_keys<<<grid_for(n, 256, maxb), 256, 0, s>>>(cell_dev, n, n_cells, S.keys.as<uint32_t>(),
                                                       S.ids.as<uint32_t>(), p->d_ctr);
    int bits = 1;
    while (bits < 32 && (1ull << bits) < n_cells) ++bits;
    ++p->stats.primitive_calls;
    GC_TRY(gc_sort_pairs_u32(S.cub_tmp, S.keys.as<uint32_t>(), S.keys2.as<uint32_t>(),
                             S.ids.as<uint32_t>(), S.ids2.as<uint32_t>(), n, bits, s));
    uint32_t *start = S.cell_start.as<uint32_t>();
    ++p->stats.kernel_launches;
    k_cell_start<<<grid_for(n + 1, 256, maxb), 256, 0, s>>>(S.keys2.as<uint32_t>(), n, n_cells,
                                                            start);
    uint64_t *ct = S.cnt_t.as<uint64_t>(), *ot = ct + (nt + 1);
    uint64_t *cs = S.cnt_s.as<uint64_t>(), *os = cs + (nt + 1);
    ++p->stats.kernel_launches;
    k_md_counts<<<grid_for(nt + 1, 256, maxb), 256, 0, s>>>(nt, m, dim, start, ct, cs);
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u64(S.cub_tmp, ct, ot, nt + 1, s));
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u64(S.cub_tmp, cs, os, nt + 1, s));
    uint64_t tot_t = 0, tot_s = 0;
    unsigned long long flags = 0;
    GC_CUDA_TRY(cudaMemcpyAsync(&tot_t, ot + nt, 8, cudaMemcpyDeviceToHost, s));
    GC_CUDA_TRY(cudaMemcpyAsync(&tot_s, os + nt, 8, cudaMemcpyDeviceToHost, s));
    GC_CUDA_TRY(cudaMemcpyAsync(&flags, p->d_ctr + CTR_FLAGS, 8, cudaMemcpyDeviceToHost, s));
    GC_CUDA_TRY(cudaStreamSynchronize(s));
    if (flags & GC_FLAG_ID_RANGE) {
        GC_TRY(gc_clear_flags(p, s, GC_FLAG_ID_RANGE));
        return GC_ERR_ARG;
    }
    const bool batch_start = p->nb_tasks == 0;
    GC_TRY(gc_reserve_batch(p, nt, tot_t, tot_s));
    ++p->stats.kernel_launches;
    k_md_fill<<<grid_for(nt, 256, maxb), 256, 0, s>>>(
        nt, m, dim, start, S.ids2.as<uint32_t>(), ot, os, p->nb_tgt, p->nb_src, task_id_base,
        p->tgt_ids.as<uint32_t>() + p->nb_tgt, p->src_ids.as<uint32_t>() + p->nb_src,
        p->tasks.as<TaskRec>() + p->nb_tasks);
    GC_CUDA_TRY(cudaGetLastError());
    p->nb_tasks += nt;
    p->nb_tgt += tot_t;
    p->nb_src += tot_s;
    // a batch that holds exactly these tasks is reduced per cell at its flush
    p->md_pending = batch_start;
    p->md_pend_m = m;
    p->md_pend_dim = dim;
    S.n = n;
    S.m = m;
    S.dim = dim;
    if (info_out) {
        info_out[0] = nt;
        info_out[1] = tot_t;
        info_out[2] = tot_s;
        info_out[3] = 0;
    }
    return GC_OK;
}

extern "C" int gc_build_md_tasks(gc_pool_t *p, const uint32_t *cell_dev, uint64_t n, int m,
                                 uint64_t task_id_base, uint64_t info_out[4])
{
    return build_md(p, cell_dev, n, m, 3, task_id_base, info_out);
}

extern "C" int gc_build_md_tasks_2d(gc_pool_t *p, const uint32_t *cell_dev, uint64_t n, int m,
                                    uint64_t task_id_base, uint64_t info_out[4])
{
    return build_md(p, cell_dev, n, m, 2, task_id_base, info_out);
}

extern "C" int gc_read_md_cells(gc_pool_t *p, uint32_t *cell_start, uint32_t *cell_atoms)
{
    if (!p || p->md.n == 0) return GC_ERR_STATE;
    MDState &S = p->md;
    GC_CUDA_TRY(cudaStreamSynchronize(p->s));
    uint64_t nc = S.dim == 2 ? (uint64_t)S.m * S.m : (uint64_t)S.m * S.m * S.m;
    if (cell_start)
        GC_CUDA_TRY(cudaMemcpy(cell_start, S.cell_start.p, (nc + 1) * 4, cudaMemcpyDeviceToHost));
    if (cell_atoms)
        GC_CUDA_TRY(cudaMemcpy(cell_atoms, S.ids2.p, S.n * 4, cudaMemcpyDeviceToHost));
    return GC_OK;
}
