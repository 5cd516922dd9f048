// gc_nbody.cu -- N-body task builder on the device (Section 4.1: particles
// grouped into buckets of a Barnes-Hut tree; each bucket's tree walk yields
// one interaction list of tree nodes and particles; one work request per
// bucket).
//
// Construction without recursion or per-level launches.  After a stable
// sort of the Morton keys, every tree node is the cell at some level l that
// starts at some sorted particle i, so a node is named by (i, l):
//   - i starts a level-l cell iff l > lcp(i), the common-prefix level of
//     keys i-1 and i;
//   - the level-l cell of i has more than B particles iff some window of
//     B+1 consecutive sorted particles containing i shares its level-l
//     prefix, i.e. l <= D(i) = max over windows [j, j+B] containing i of the
//     common-prefix level of keys j and j+B;
//   - a cell is a node iff its parent has more than B particles, and a node
//     is a leaf iff it has at most B particles or l = 21.
// So particle i starts the nodes at levels lcp(i)+1 .. min(D(i)+1, 21).
// Ordering the pairs (i, l) by i, then l, is exactly depth-first preorder
// with children in octant order (a node precedes its descendants, which
// share or follow its first particle; siblings are ordered by first
// particle).  A prefix sum over the per-particle node counts numbers the
// nodes; a node's particle range end comes from a binary search on the
// sorted keys and its subtree size from the same prefix sum.
//
// The walk visits nodes in preorder with skips (no stack): an accepted or
// leaf node continues at k + size(k), an opened internal node at k + 1; the
// node array is split into preorder ranges walked independently (k_walk).
#include <cub/device/device_scan.cuh>
#include <algorithm>
#include <climits>

#include "gc_common.cuh"

int gc_launch_upload_seq(gc_pool *p, uint32_t id_base, const float4 *vals, uint64_t n);

namespace {

struct GridParams {
    double lo[3];
    double scale;   // 2^21 / L = 2^sh, L = smallest power of two >= largest extent
    float lof[3];   // lo as float (the minima are float values)
    float scalef;   // 2^sh
    float tiny;     // 2^-(sh+6): smallest nonzero |coordinate| of the FP32 path
    int fast;       // the FP32 path applies (sh in [-100, 100])
};

__device__ __forceinline__ uint32_t ord_key(float f)
{
    uint32_t b = __float_as_uint(f);
    return (b & 0x80000000u) ? ~b : (b | 0x80000000u);
}

__device__ __forceinline__ float ord_val(uint32_t k)
{
    return __uint_as_float((k & 0x80000000u) ? (k & 0x7FFFFFFFu) : ~k);
}

// bounds[0..2] = ordered-int min, bounds[3..5] = ordered-int max
__global__ void k_bbox(const float4 *x, uint64_t n, uint32_t *bounds)
{
    uint32_t mn[3] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu}, mx[3] = {0, 0, 0};
    GRID_STRIDE(i, n) {
        float4 v = x[i];
        uint32_t k[3] = {ord_key(v.x), ord_key(v.y), ord_key(v.z)};
        for (int a = 0; a < 3; ++a) {
            mn[a] = min(mn[a], k[a]);
            mx[a] = max(mx[a], k[a]);
        }
    }
    for (int a = 0; a < 3; ++a)
        for (int o = 16; o; o >>= 1) {
            mn[a] = min(mn[a], __shfl_xor_sync(0xffffffffu, mn[a], o));
            mx[a] = max(mx[a], __shfl_xor_sync(0xffffffffu, mx[a], o));
        }
    // warps -> block in shared memory, then one set of atomics per block (one
    // set per warp made the six global words a serial hot spot)
    __shared__ uint32_t wb[32][6];
    const int w = threadIdx.x >> 5, nw = (blockDim.x + 31) >> 5;
    if ((threadIdx.x & 31) == 0)
        for (int a = 0; a < 3; ++a) {
            wb[w][a] = mn[a];
            wb[w][3 + a] = mx[a];
        }
    __syncthreads();
    if (threadIdx.x < 6) {
        const int a = threadIdx.x;
        uint32_t v = wb[0][a];
        for (int q = 1; q < nw; ++q) v = a < 3 ? min(v, wb[q][a]) : max(v, wb[q][a]);
        if (a < 3) atomicMin(&bounds[a], v);
        else atomicMax(&bounds[a], v);
    }
}

__global__ void k_grid_params(const uint32_t *bounds, GridParams *gp)
{
    double ext = 0.0;
    for (int a = 0; a < 3; ++a) {
        double lo = (double)ord_val(bounds[a]);
        double hi = (double)ord_val(bounds[3 + a]);
        gp->lo[a] = lo;
        if (hi - lo > ext) ext = hi - lo;
    }
    double L = 1.0;
    if (ext > 0.0) {
        while (L < ext) L *= 2.0;
        while (L * 0.5 >= ext) L *= 0.5;
    }
    gp->scale = 2097152.0 / L;
    const int sh = ilogb(gp->scale);
    for (int a = 0; a < 3; ++a) gp->lof[a] = (float)gp->lo[a];
    gp->fast = sh >= -100 && sh <= 100;
    gp->scalef = gp->fast ? ldexpf(1.0f, sh) : 0.0f;
    gp->tiny = gp->fast ? ldexpf(1.0f, -(sh + 6)) : 0.0f;
}

__device__ __forceinline__ uint32_t quant(float x, double lo, double scale)
{
    double t = __dmul_rn(__dsub_rn((double)x, lo), scale);
    double f = floor(t);
    f = fmax(f, 0.0);
    f = fmin(f, 2097151.0);
    return (uint32_t)f;
}

// quant() in FP32, exact.  With x, lo floats, d = x - lo >= 0 and
// d <= L = 2^(21-sh), the FP64 subtraction rounds d only below
// 2^-(sh+31) (half an FP64 ulp of a number below 2^(22-sh)).  If x and lo
// are each zero or at least 2^-(sh+6) in magnitude, both are multiples of
// 2^-(sh+29) (23 fraction bits below their exponent), so d is at least
// 2^-(sh+29) away from any multiple of 2^-sh it does not equal, and the FP64
// rounding cannot carry it across one: floor(RN64(d) 2^sh) = floor(d 2^sh).
// Knuth's TwoSum gives d = s + e exactly in FP32 (s = RN32(x - lo),
// |e| <= half an ulp of s); scaled by 2^sh (exact), floor(S + E) is floor(S)
// unless S is an integer and E < 0.  Other inputs take the FP64 expression.
__device__ __forceinline__ uint32_t quant_exact(float x, int a, const GridParams &g)
{
    const float lo = g.lof[a];
    const float ax = fabsf(x), al = fabsf(lo);
    if (g.fast && (x == 0.f || ax >= g.tiny) && (lo == 0.f || al >= g.tiny) && ax < 1e37f &&
        al < 1e37f) {
        const float s = __fsub_rn(x, lo);
        const float bp = __fsub_rn(s, x);       // TwoSum of x and -lo
        const float ap = __fsub_rn(s, bp);
        const float e = __fadd_rn(__fsub_rn(x, ap), __fsub_rn(-lo, bp));
        const float S = __fmul_rn(s, g.scalef), E = __fmul_rn(e, g.scalef);
        float f = floorf(S);
        if (f == S && E < 0.f) f -= 1.f;
        f = fminf(fmaxf(f, 0.f), 2097151.f);
        return (uint32_t)f;
    }
    return quant(x, g.lo[a], g.scale);
}

// spread the 21 low bits of v to every third bit
__device__ __forceinline__ uint64_t spread3(uint32_t v)
{
    uint64_t x = v & 0x1FFFFFu;
    x = (x | (x << 32)) & 0x001F00000000FFFFull;
    x = (x | (x << 16)) & 0x001F0000FF0000FFull;
    x = (x | (x << 8)) & 0x100F00F00F00F00Full;
    x = (x | (x << 4)) & 0x10C30C30C30C30C3ull;
    x = (x | (x << 2)) & 0x1249249249249249ull;
    return x;
}

__device__ __forceinline__ uint32_t compact3(uint64_t x)
{
    x &= 0x1249249249249249ull;
    x = (x | (x >> 2)) & 0x10C30C30C30C30C3ull;
    x = (x | (x >> 4)) & 0x100F00F00F00F00Full;
    x = (x | (x >> 8)) & 0x001F0000FF0000FFull;
    x = (x | (x >> 16)) & 0x001F00000000FFFFull;
    x = (x | (x >> 32)) & 0x00000000001FFFFFull;
    return (uint32_t)x;
}

__device__ __forceinline__ uint64_t morton_of(float4 v, const GridParams &g)
{
    return spread3(quant_exact(v.x, 0, g)) | (spread3(quant_exact(v.y, 1, g)) << 1) |
           (spread3(quant_exact(v.z, 2, g)) << 2);
}

__global__ void k_keys(const float4 *x, uint64_t n, const GridParams *gp, uint64_t *keys,
                       uint32_t *ids)
{
    const GridParams g = *gp;
    GRID_STRIDE(i, n) {
        keys[i] = morton_of(x[i], g);
        ids[i] = (uint32_t)i;
    }
}

// ---- Morton order seeded by the previous build's order -------------------
//
// The tree is rebuilt at every step (Section 4.1), and between two steps the
// particles move little, so the previous step's sorted order is close to the
// new one.  The seeded order computes the new keys in the previous order and
// keeps most of it in place; the order compared is (key, id), the order of
// the stable key sort.
//   1. Tiles of SEED_TILE consecutive particles (previous order): one or
//      both particles of every descent are dropped, round after round, until
//      the tile's remainder rem_t is ascending.  The part of rem_t above U_t,
//      the median of the first 32 keys of tile t+1, is dropped too; b_t
//      elements stay (k_seed_tiles).
//   2. P_t = the largest of the last remaining elements rem_u[b_u - 1] of the
//      tiles u < t (k_seed_scan); tile t drops its elements below P_t, a_t of
//      them (k_seed_low).  A kept element of tile t is then at most
//      rem_t[b_t - 1] <= P_u < every kept element of a later tile u: the kept
//      elements, in slot order (slot = tile * SEED_TILE + index), ascend.
//      The inclusive maximum P'_t is the largest kept element of tiles <= t.
//   3. Every dropped particle ("mover") x finds the slot of the smallest kept
//      element above it (k_mover_slot: the first tile with P'_t > x, then
//      within that tile), or the end slot n.  W[q] counts the kept element of
//      slot q plus the movers assigned to it; with E the exclusive prefix sum
//      of W, the kept element of slot q lands at E[q] + W[q] - 1 and the
//      movers of slot q at E[q] + their rank by (key, id) among themselves
//      (k_mover_scatter, k_seed_place).
// The result is the stable key sort, element for element.  Which particles
// are dropped decides only the cost; if some slot collects more than
// SEED_GROUP_MAX movers the build sorts all keys instead.
constexpr int SEED_TILE = 2048, SEED_THREADS = 512, SEED_PER = SEED_TILE / SEED_THREADS;
constexpr int SEED_ROUNDS = 64;       // descent-removal rounds before a tile gives up
constexpr int SEED_GROUP_MAX = 64;    // movers per slot ranked pairwise

struct KidMax {
    uint64_t k;
    uint32_t i, h;   // h = 0: no element (below everything)
};

struct SeedTile {
    KidMax last;     // rem[b - 1]
    KidMax pe, pi;   // largest kept element of the tiles before / up to this one
    uint32_t b, a;   // remainder [0, b) after step 1; kept range [a, b)
};

struct SeedCtr {
    unsigned long long movers;
    unsigned int max_group;
    unsigned int pad;
};

__device__ __forceinline__ bool kid_gt(uint64_t ka, uint32_t ia, uint64_t kb, uint32_t ib)
{
    return ka > kb || (ka == kb && ia > ib);
}

__device__ __forceinline__ KidMax kid_max(KidMax a, KidMax b)
{
    if (!a.h) return b;
    if (!b.h) return a;
    return kid_gt(a.k, a.i, b.k, b.i) ? a : b;
}

// (k, i) is above m (every (k, i) is above "no element")
__device__ __forceinline__ bool above(uint64_t k, uint32_t i, const KidMax &m)
{
    return !m.h || kid_gt(k, i, m.k, m.i);
}

__device__ __forceinline__ KidMax shfl_up_kid(KidMax v, int o)
{
    KidMax r;
    r.k = __shfl_up_sync(0xffffffffu, v.k, o);
    r.i = __shfl_up_sync(0xffffffffu, v.i, o);
    r.h = __shfl_up_sync(0xffffffffu, v.h, o);
    return r;
}

// Append c movers per lane (the whole warp calls): returns this lane's
// first index in the mover list.
__device__ __forceinline__ unsigned long long mover_base(int c, SeedCtr *ctr)
{
    const int lane = threadIdx.x & 31;
    int incl = c;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= o) incl += v;
    }
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    unsigned long long base = 0;
    if (lane == 31 && total) base = atomicAdd(&ctr->movers, (unsigned long long)total);
    base = __shfl_sync(0xffffffffu, base, 31);
    return base + (unsigned long long)(incl - c);
}

// One block per tile; thread t owns remainder positions 4t .. 4t+3.  Each
// round every descent (p-1, p) is resolved from the four elements around
// it: drop p-1 alone if p-2 (if any) does not exceed p (p-1 is a spike),
// else drop p alone if p-1 does not exceed p+1 (if any; p is a dip), else
// drop both.  A round with a descent drops at least one particle, so the
// loop ends; after SEED_ROUNDS rounds a tile still out of order drops its
// whole remainder.
__global__ __launch_bounds__(SEED_THREADS) void k_seed_tiles(
    const float4 *x, const uint32_t *prev, uint64_t n, const GridParams *gp, uint64_t *KT,
    uint32_t *IT, uint32_t *W, SeedTile *tiles, SeedCtr *ctr, uint64_t *MK, uint32_t *MI,
    uint32_t *MH)
{
    __shared__ uint64_t sk[SEED_TILE];
    __shared__ uint32_t si[SEED_TILE];
    __shared__ int wsum[SEED_THREADS / 32];
    __shared__ int s_total, s_b;
    __shared__ KidMax s_u;
    const uint64_t t0 = (uint64_t)blockIdx.x * SEED_TILE;
    const int size = (int)(n - t0 < (uint64_t)SEED_TILE ? n - t0 : (uint64_t)SEED_TILE);
    int cnt = size;
    const GridParams g = *gp;
    const uint32_t tile = blockIdx.x;
    for (int j = threadIdx.x; j < cnt; j += SEED_THREADS) {
        const uint32_t id = prev[t0 + j];
        sk[j] = morton_of(x[id], g);
        si[j] = id;
    }
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    if (w == 0) {   // U: median of the first 32 keys of the next tile
        const uint64_t t1 = t0 + SEED_TILE;
        const int m = t1 < n ? (n - t1 < 32 ? (int)(n - t1) : 32) : 0;
        KidMax v{0, 0, 0};
        if (lane < m) {
            const uint32_t id = prev[t1 + lane];
            v.k = morton_of(x[id], g);
            v.i = id;
            v.h = 1;
        }
        int below = 0;   // elements of the sample below this lane's
        for (int q = 0; q < m; ++q) {
            const uint64_t k = __shfl_sync(0xffffffffu, v.k, q);
            const uint32_t i = __shfl_sync(0xffffffffu, v.i, q);
            below += (v.h && kid_gt(v.k, v.i, k, i)) ? 1 : 0;
        }
        const unsigned hit = __ballot_sync(0xffffffffu, v.h && below == m / 2);
        if (lane == 0) s_u = KidMax{0, 0, 0};
        __syncwarp();
        if (hit && lane == __ffs(hit) - 1) s_u = v;
    }
    __syncthreads();
    const int base = threadIdx.x * SEED_PER;
    constexpr int WIN = SEED_PER + 4;     // positions base-2 .. base+SEED_PER+1
    for (int round = 0;; ++round) {
        uint64_t k[WIN];
        uint32_t id[WIN];
#pragma unroll
        for (int q = 0; q < WIN; ++q) {
            const int pos = base - 2 + q;
            const bool in = pos >= 0 && pos < cnt;
            k[q] = in ? sk[pos] : 0;
            id[q] = in ? si[pos] : 0;
        }
        // descents at p = base .. base+SEED_PER; drop-left / drop-right
        bool dl[SEED_PER + 1], dr[SEED_PER + 1];
        bool any = false;
#pragma unroll
        for (int e = 0; e <= SEED_PER; ++e) {
            const int p = base + e, q = e + 2;
            const bool d = p >= 1 && p < cnt && kid_gt(k[q - 1], id[q - 1], k[q], id[q]);
            const bool spike = p == 1 || !kid_gt(k[q - 2], id[q - 2], k[q], id[q]);
            const bool dip = p + 1 >= cnt || !kid_gt(k[q - 1], id[q - 1], k[q + 1], id[q + 1]);
            dl[e] = d && (spike || !dip);
            dr[e] = d && !spike;
            if (e < SEED_PER) any |= d;
        }
        if (!__syncthreads_or(any)) break;
        const bool give_up = round >= SEED_ROUNDS;
        int c = 0, cd = 0;
#pragma unroll
        for (int e = 0; e < SEED_PER; ++e) {
            if (base + e >= cnt) break;
            if (!give_up && !dr[e] && !dl[e + 1]) ++c;
            else ++cd;
        }
        unsigned long long mb = mover_base(cd, ctr);
        int incl = c;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const int v = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += v;
        }
        if (lane == 31) wsum[w] = incl;
        __syncthreads();
        if (w == 0) {
            const int v = lane < SEED_THREADS / 32 ? wsum[lane] : 0;
            int inc = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const int u = __shfl_up_sync(0xffffffffu, inc, o);
                if (lane >= o) inc += u;
            }
            if (lane < SEED_THREADS / 32) wsum[lane] = inc - v;
            if (lane == SEED_THREADS / 32 - 1) s_total = inc;
        }
        __syncthreads();
        int dst = wsum[w] + incl - c;
#pragma unroll
        for (int e = 0; e < SEED_PER; ++e) {
            if (base + e >= cnt) break;
            if (!give_up && !dr[e] && !dl[e + 1]) {
                sk[dst] = k[e + 2];
                si[dst] = id[e + 2];
                ++dst;
            } else {
                MK[mb] = k[e + 2];
                MI[mb] = id[e + 2];
                MH[mb] = tile;
                ++mb;
            }
        }
        cnt = s_total;
        __syncthreads();
    }
    // b = elements not above U (the remainder ascends: one boundary)
    if (threadIdx.x == 0) s_b = (cnt && above(sk[0], si[0], s_u) && s_u.h) ? 0 : cnt;
    __syncthreads();
    if (s_u.h) {
        for (int j = threadIdx.x; j < cnt; j += SEED_THREADS)
            if (!kid_gt(sk[j], si[j], s_u.k, s_u.i) &&
                (j + 1 == cnt || kid_gt(sk[j + 1], si[j + 1], s_u.k, s_u.i)))
                s_b = j + 1;
    }
    __syncthreads();
    const int b = s_b;
    // drop [b, cnt); slots [0, b) hold the remainder
#pragma unroll
    for (int e = 0; e < SEED_PER; ++e) {
        const int j = threadIdx.x + e * SEED_THREADS;
        if (j < size) W[t0 + j] = j < b ? 1u : 0u;
        if (j < b) {
            KT[t0 + j] = sk[j];
            IT[t0 + j] = si[j];
        }
    }
    int cd = 0;
#pragma unroll
    for (int e = 0; e < SEED_PER; ++e) cd += (base + e >= b && base + e < cnt) ? 1 : 0;
    unsigned long long mb = mover_base(cd, ctr);
#pragma unroll
    for (int e = 0; e < SEED_PER; ++e) {
        const int j = base + e;
        if (j >= b && j < cnt) {
            MK[mb] = sk[j];
            MI[mb] = si[j];
            MH[mb] = tile;
            ++mb;
        }
    }
    if (threadIdx.x == 0) {
        SeedTile T{};
        T.b = (uint32_t)b;
        if (b) T.last = KidMax{sk[b - 1], si[b - 1], 1};
        tiles[tile] = T;
    }
}

// One block of 1024 threads over all tiles, 1024 at a time: exclusive and
// inclusive prefix maxima of the tiles' last remaining elements.
__global__ __launch_bounds__(1024) void k_seed_scan(SeedTile *tiles, uint32_t nt)
{
    __shared__ KidMax wmax[32];
    __shared__ KidMax carry;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if (threadIdx.x == 0) carry = KidMax{0, 0, 0};
    __syncthreads();
    for (uint32_t c0 = 0; c0 < nt; c0 += blockDim.x) {
        const uint32_t t = c0 + threadIdx.x;
        const KidMax last = t < nt ? tiles[t].last : KidMax{0, 0, 0};
        KidMax inc = last;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const KidMax v = shfl_up_kid(inc, o);
            if (lane >= o) inc = kid_max(inc, v);
        }
        KidMax exc = shfl_up_kid(inc, 1);
        if (lane == 0) exc.h = 0;
        if (lane == 31) wmax[w] = inc;
        __syncthreads();
        if (w == 0) {
            const KidMax v = lane < nw ? wmax[lane] : KidMax{0, 0, 0};
            KidMax vi = v;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) {
                const KidMax u = shfl_up_kid(vi, o);
                if (lane >= o) vi = kid_max(vi, u);
            }
            KidMax ve = shfl_up_kid(vi, 1);
            if (lane == 0) ve.h = 0;
            if (lane < nw) wmax[lane] = ve;
        }
        __syncthreads();
        const KidMax pe = kid_max(carry, kid_max(wmax[w], exc));
        const KidMax pi = kid_max(pe, last);
        if (t < nt) {
            tiles[t].pe = pe;
            tiles[t].pi = pi;
        }
        __syncthreads();   // every thread has read the carry
        if (threadIdx.x == blockDim.x - 1) carry = pi;
        __syncthreads();
    }
}

// One warp per tile: a = remainder elements below P (a prefix), dropped.
__global__ __launch_bounds__(256) void k_seed_low(const uint64_t *KT, const uint32_t *IT,
                                                  SeedTile *tiles, uint32_t nt, uint32_t *W,
                                                  SeedCtr *ctr, uint64_t *MK, uint32_t *MI,
                                                  uint32_t *MH)
{
    const uint32_t t = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
    const int lane = threadIdx.x & 31;
    if (t >= nt) return;   // whole warps leave together
    const KidMax P = tiles[t].pe;
    const uint32_t b = tiles[t].b;
    const uint64_t t0 = (uint64_t)t * SEED_TILE;
    uint32_t a = 0;
    if (P.h) {
        for (uint32_t j0 = 0; j0 < b; j0 += 32) {
            const uint32_t j = j0 + lane;
            const bool below = j < b && kid_gt(P.k, P.i, KT[t0 + j], IT[t0 + j]);
            const unsigned bal = __ballot_sync(0xffffffffu, below);
            unsigned long long mb = mover_base(below ? 1 : 0, ctr);
            if (below) {
                MK[mb] = KT[t0 + j];
                MI[mb] = IT[t0 + j];
                MH[mb] = t;
                W[t0 + j] = 0;
            }
            a += __popc(bal);
            if (bal != 0xffffffffu) break;
        }
    }
    if (lane == 0) tiles[t].a = a;
}

// Slot of the smallest kept element above each mover, or n; the mover's
// arrival index among the movers of that slot.
__global__ __launch_bounds__(256) void k_mover_slot(
    SeedCtr *ctr, const uint64_t *MK, const uint32_t *MI, const uint32_t *MH,
    const uint64_t *KT, const uint32_t *IT, const SeedTile *tiles, uint32_t nt, uint64_t n,
    uint32_t *W, uint32_t *MS, uint32_t *MA)
{
    const uint64_t m = ctr->movers;
    GRID_STRIDE(v, m) {
        const uint64_t k = MK[v];
        const uint32_t i = MI[v], hint = MH[v];
        // first tile u whose largest kept element so far is above (k, i)
        uint32_t u;
        if (!above(k, i, tiles[hint].pi) && (hint == 0 || above(k, i, tiles[hint - 1].pi))) {
            u = hint;
        } else {
            uint32_t lo = 0, hi = nt;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (above(k, i, tiles[mid].pi)) lo = mid + 1;
                else hi = mid;
            }
            u = lo;
        }
        uint64_t q = n;
        if (u < nt) {   // within tile u: the remainder elements below (k, i)
            const uint64_t t0 = (uint64_t)u * SEED_TILE;
            uint32_t lo = 0, hi = tiles[u].b;
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if (kid_gt(k, i, KT[t0 + mid], IT[t0 + mid])) lo = mid + 1;
                else hi = mid;
            }
            q = t0 + lo;
        }
        const uint32_t arr = atomicAdd(&W[q], 1u) - (q < n ? 1u : 0u);
        MS[v] = (uint32_t)q;
        MA[v] = arr;
        atomicMax(&ctr->max_group, arr + 1);
    }
}

// Movers to their slot's output range, in arrival order.
__global__ void k_mover_scatter(const uint64_t *MK, const uint32_t *MI, const uint32_t *MS,
                                const uint32_t *MA, uint64_t m, const uint32_t *E,
                                uint64_t *TK, uint32_t *TI)
{
    GRID_STRIDE(v, m) {
        const uint64_t pos = (uint64_t)E[MS[v]] + MA[v];
        TK[pos] = MK[v];
        TI[pos] = MI[v];
    }
}

// Final order: kept elements of slots [0, n), then the m movers ranked by
// (key, id) within their slot's range.
__global__ void k_seed_place(const uint64_t *KT, const uint32_t *IT, const SeedTile *tiles,
                             uint64_t n, const uint32_t *W, const uint32_t *E,
                             const uint64_t *MK, const uint32_t *MI, const uint32_t *MS,
                             uint64_t m, const uint64_t *TK, const uint32_t *TI, uint64_t *K,
                             uint32_t *I)
{
    GRID_STRIDE(v, n + m) {
        if (v < n) {
            const uint32_t t = (uint32_t)(v / SEED_TILE), j = (uint32_t)(v % SEED_TILE);
            const SeedTile &T = tiles[t];
            if (j >= T.a && j < T.b) {
                const uint64_t pos = (uint64_t)E[v] + W[v] - 1;
                K[pos] = KT[v];
                I[pos] = IT[v];
            }
        } else {
            const uint64_t u = v - n;
            const uint64_t k = MK[u];
            const uint32_t i = MI[u], q = MS[u];
            const uint32_t grp = W[q] - (q < n ? 1u : 0u);
            const uint64_t g0 = E[q];
            uint32_t r = 0;
            for (uint32_t c = 0; c < grp; ++c) r += kid_gt(k, i, TK[g0 + c], TI[g0 + c]) ? 1 : 0;
            K[g0 + r] = k;
            I[g0 + r] = i;
        }
    }
}

// deepest level l (0..21) at which keys a and b share the level-l cell
__device__ __forceinline__ int common_level(uint64_t a, uint64_t b)
{
    uint64_t x = a ^ b;
    if (x == 0) return 21;
    int hb = 63 - __clzll((long long)x);
    return 20 - hb / 3;
}

__global__ void k_lcp_win(const uint64_t *K, uint64_t n, int B, int8_t *lcp, int8_t *win)
{
    GRID_STRIDE(i, n) {
        lcp[i] = (int8_t)((i == 0) ? -1 : common_level(K[i - 1], K[i]));
        if (i + (uint64_t)B < n) win[i] = (int8_t)common_level(K[i], K[i + B]);
    }
}

__global__ void k_dmax(const int8_t *lcp, const int8_t *win, uint64_t n, int B, int8_t *dmax,
                       uint32_t *nnode)
{
    GRID_STRIDE(i, n) {
        int d = -1;
        if (n > (uint64_t)B) {
            int64_t j0 = (int64_t)i - B;
            if (j0 < 0) j0 = 0;
            int64_t j1 = (int64_t)i;
            if (j1 > (int64_t)(n - B - 1)) j1 = (int64_t)(n - B - 1);
            for (int64_t j = j0; j <= j1; ++j) d = max(d, (int)win[j]);
        }
        dmax[i] = (int8_t)d;
        int lo = (i == 0) ? 0 : lcp[i] + 1;
        int hi = min(d + 1, 21);
        nnode[i] = (hi >= lo) ? (uint32_t)(hi - lo + 1) : 0u;
    }
    if (blockIdx.x == 0 && threadIdx.x == 0) nnode[n] = 0;
}

// node_a = {first, count, subtree size, level | leaf << 8}; node_b = {cell x, y, z, 0}
__global__ void k_emit_nodes(const uint64_t *K, uint64_t n, const int8_t *lcp,
                             const int8_t *dmax, const uint32_t *node_off, uint4 *node_a,
                             uint4 *node_b, uint32_t *bcnt, int B)
{
    GRID_STRIDE(i, n) {
        int lo = (i == 0) ? 0 : lcp[i] + 1;
        int d = dmax[i];
        int hi = min(d + 1, 21);
        for (int l = lo; l <= hi; ++l) {
            uint32_t k = node_off[i] + (uint32_t)(l - lo);
            int sh = 3 * (21 - l);
            uint64_t pre = (sh >= 64) ? 0 : (K[i] >> sh);
            // end of the cell: first e > i whose key prefix differs
            uint64_t a = i + 1, b = n;
            while (a < b) {
                uint64_t mid = (a + b) >> 1;
                uint64_t pm = (sh >= 64) ? 0 : (K[mid] >> sh);
                if (pm == pre) a = mid + 1; else b = mid;
            }
            uint32_t e = (uint32_t)a;
            bool leaf = (l > d) || (l == 21);
            uint32_t cnt = e - (uint32_t)i;
            uint32_t size = node_off[e] - node_off[i] - (uint32_t)(l - lo);
            node_a[k] = make_uint4((uint32_t)i, cnt, size, (uint32_t)l | (leaf ? 256u : 0u));
            node_b[k] = make_uint4(compact3(pre), compact3(pre >> 1), compact3(pre >> 2), 0u);
            bcnt[k] = leaf ? (cnt + (uint32_t)B - 1) / (uint32_t)B : 0u;
        }
    }
}

// FP64 monopoles from prefix sums over the sorted particles: a node's
// (mass, mass-weighted position) is P[first + count] - P[first].
struct M4 {
    double m, mx, my, mz;
};

__global__ void k_mono_input(const uint32_t *sorted_ids, const float4 *x, uint64_t n, M4 *out)
{
    GRID_STRIDE(i, n + 1) {
        M4 v{0, 0, 0, 0};
        if (i < n) {
            float4 p = x[sorted_ids[i]];
            double w = (double)p.w;
            v = M4{w, w * (double)p.x, w * (double)p.y, w * (double)p.z};
        }
        out[i] = v;
    }
}

// Exclusive scan of the M4 values with a fixed association, so that the node
// values -- and every result computed from them -- repeat bit for bit from
// run to run (a decoupled look-back scan groups floating-point sums by
// timing).  Tiles of M4_TILE values: (1) each tile's sum, (2) an exclusive
// scan of the tile sums in one block, (3) each tile's exclusive scan offset
// by its tile prefix.  Within a tile every thread owns M4_PER consecutive
// values; thread sums are combined by a shuffle scan per warp and then
// across the warps in warp order.
constexpr int M4_THREADS = 256, M4_PER = 8, M4_TILE = M4_THREADS * M4_PER;

__device__ __forceinline__ M4 m4_add(const M4 &a, const M4 &b)
{
    return M4{a.m + b.m, a.mx + b.mx, a.my + b.my, a.mz + b.mz};
}

__device__ __forceinline__ M4 m4_shfl_up(const M4 &v, int o)
{
    return M4{__shfl_up_sync(0xffffffffu, v.m, o), __shfl_up_sync(0xffffffffu, v.mx, o),
              __shfl_up_sync(0xffffffffu, v.my, o), __shfl_up_sync(0xffffffffu, v.mz, o)};
}

// Exclusive block scan of one M4 per thread (M4_THREADS threads); *total
// receives the block's sum.
__device__ M4 m4_block_excl_scan(M4 v, M4 *wsum, M4 *total)
{
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    M4 x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const M4 y = m4_shfl_up(x, o);
        if (lane >= o) x = m4_add(y, x);
    }
    if (lane == 31) wsum[w] = x;
    __syncthreads();
    M4 before{0, 0, 0, 0};
    for (int q = 0; q < w; ++q) before = m4_add(before, wsum[q]);
    if (total) {
        M4 t{0, 0, 0, 0};
        for (int q = 0; q < M4_THREADS / 32; ++q) t = m4_add(t, wsum[q]);
        *total = t;
    }
    __syncthreads();
    // exclusive: the sum of the earlier warps plus the earlier lanes of this warp
    M4 ex = m4_shfl_up(x, 1);
    if (lane == 0) ex = M4{0, 0, 0, 0};
    return m4_add(before, ex);
}

__device__ __forceinline__ M4 m4_thread_sum(const M4 *in, uint64_t n, uint64_t i0)
{
    M4 acc{0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < M4_PER; ++j)
        if (i0 + j < n) acc = m4_add(acc, in[i0 + j]);
    return acc;
}

__global__ void __launch_bounds__(M4_THREADS) k_m4_tile_sum(const M4 *in, uint64_t n, M4 *tile_sum)
{
    __shared__ M4 wsum[M4_THREADS / 32];
    const uint64_t i0 = (uint64_t)blockIdx.x * M4_TILE + (uint64_t)threadIdx.x * M4_PER;
    M4 total;
    m4_block_excl_scan(m4_thread_sum(in, n, i0), wsum, &total);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = total;
}

// one block: tile sums -> exclusive tile prefixes, M4_PER tiles per thread and round
__global__ void __launch_bounds__(M4_THREADS) k_m4_scan_tiles(M4 *tile, uint64_t nt)
{
    __shared__ M4 wsum[M4_THREADS / 32];
    __shared__ M4 carry;
    if (threadIdx.x == 0) carry = M4{0, 0, 0, 0};
    __syncthreads();
    for (uint64_t r0 = 0; r0 < nt; r0 += M4_TILE) {
        const uint64_t i0 = r0 + (uint64_t)threadIdx.x * M4_PER;
        M4 v[M4_PER];
        M4 acc{0, 0, 0, 0};
#pragma unroll
        for (int j = 0; j < M4_PER; ++j) {
            v[j] = i0 + j < nt ? tile[i0 + j] : M4{0, 0, 0, 0};
            acc = m4_add(acc, v[j]);
        }
        M4 total;
        M4 run = m4_add(carry, m4_block_excl_scan(acc, wsum, &total));
#pragma unroll
        for (int j = 0; j < M4_PER; ++j) {
            if (i0 + j < nt) tile[i0 + j] = run;
            run = m4_add(run, v[j]);
        }
        __syncthreads();
        if (threadIdx.x == 0) carry = m4_add(carry, total);
        __syncthreads();
    }
}

__global__ void __launch_bounds__(M4_THREADS) k_m4_tile_scan(const M4 *in, uint64_t n,
                                                            const M4 *tile_pre, M4 *out)
{
    __shared__ M4 wsum[M4_THREADS / 32];
    const uint64_t i0 = (uint64_t)blockIdx.x * M4_TILE + (uint64_t)threadIdx.x * M4_PER;
    M4 v[M4_PER];
    M4 acc{0, 0, 0, 0};
#pragma unroll
    for (int j = 0; j < M4_PER; ++j) {
        v[j] = i0 + j < n ? in[i0 + j] : M4{0, 0, 0, 0};
        acc = m4_add(acc, v[j]);
    }
    M4 run = m4_add(tile_pre[blockIdx.x], m4_block_excl_scan(acc, wsum, nullptr));
#pragma unroll
    for (int j = 0; j < M4_PER; ++j) {
        if (i0 + j < n) out[i0 + j] = run;
        run = m4_add(run, v[j]);
    }
}

__global__ void k_mono_nodes(const uint4 *node_a, uint64_t nn, const M4 *P, float4 *node_val)
{
    GRID_STRIDE(k, nn) {
        uint4 A = node_a[k];
        M4 e = P[A.x + A.y], f = P[A.x];
        double m = e.m - f.m;
        float4 v;
        v.x = (float)(m != 0.0 ? (e.mx - f.mx) / m : 0.0);
        v.y = (float)(m != 0.0 ? (e.my - f.my) / m : 0.0);
        v.z = (float)(m != 0.0 ? (e.mz - f.mz) / m : 0.0);
        v.w = (float)m;
        node_val[k] = v;
    }
}

// bucket = {first, count, leaf node, 0}; box in doubled grid units
__global__ void k_emit_buckets(const uint4 *node_a, uint64_t nn, const uint32_t *boff,
                               const uint64_t *K, int B, uint4 *bucket, int4 *blo, int4 *bhi)
{
    GRID_STRIDE(k, nn) {
        uint4 A = node_a[k];
        if (!(A.w & 256u)) continue;
        uint32_t nb = (A.y + (uint32_t)B - 1) / (uint32_t)B;
        for (uint32_t c = 0; c < nb; ++c) {
            uint32_t f = A.x + c * (uint32_t)B;
            uint32_t cnt = min((uint32_t)B, A.y - c * (uint32_t)B);
            uint32_t b = boff[k] + c;
            bucket[b] = make_uint4(f, cnt, (uint32_t)k, 0u);
            int lo[3] = {1 << 30, 1 << 30, 1 << 30}, hi[3] = {-1, -1, -1};
            for (uint32_t q = f; q < f + cnt; ++q) {
                uint64_t key = K[q];
                int v[3] = {(int)compact3(key), (int)compact3(key >> 1), (int)compact3(key >> 2)};
                for (int a = 0; a < 3; ++a) {
                    lo[a] = min(lo[a], v[a]);
                    hi[a] = max(hi[a], v[a]);
                }
            }
            blo[b] = make_int4(2 * lo[0], 2 * lo[1], 2 * lo[2], 0);
            bhi[b] = make_int4(2 * hi[0] + 2, 2 * hi[1] + 2, 2 * hi[2] + 2, 0);
        }
    }
}

// Acceptance thresholds per level: a node of edge s (doubled units) is
// accepted iff td^2 s^2 < tn^2 d^2, i.e. (integers, tn > 0) iff
// d^2 > floor(td^2 s^2 / tn^2); with tn = 0 nothing is accepted.
struct WalkThresholds {
    int64_t t[22];
};

// The walk's view of node k, 16 bytes: W[k] = {subtree size | leaf << 31,
// centre x | level << 22, centre y | leaf count << 22, centre z} (centre in
// doubled grid units, below 2^22; the leaf count, WALK_LEAF_FAR when it does
// not fit in 10 bits, lets the count pass skip LF), and for a leaf LF[k] =
// {first particle, count}.  W[nn] is a sentinel.  Whether a node contains a bucket is a preorder test against the
// bucket's own leaf (k <= leaf < k + size), so the per-node record needs no
// particle range; the acceptance thresholds come per level from a table.
constexpr uint32_t WALK_LEAF_FAR = 1023u;   // leaf count field: read LF instead

__global__ void k_walk_nodes(const uint4 *node_a, const uint4 *node_b, uint32_t nn, uint4 *W,
                             uint2 *LF)
{
    GRID_STRIDE(k, (uint64_t)nn + 1) {
        if (k == nn) {
            W[k] = make_uint4(1u, 0u, 0u, 0u);
            continue;
        }
        const uint4 A = node_a[k], C = node_b[k];
        const uint32_t lvl = A.w & 255u;
        const uint32_t s = 1u << (22 - lvl), h = s >> 1;
        const uint32_t ln = (A.w & 256u) ? min(A.y, WALK_LEAF_FAR) : 0u;
        W[k] = make_uint4(A.z | ((A.w & 256u) << 23), (C.x * s + h) | (lvl << 22),
                          (C.y * s + h) | (ln << 22), C.z * s + h);
        LF[k] = make_uint2(A.x, A.y);
    }
}

constexpr int WALK_ANC = 24;      // > tree depth (21 levels below the root)
constexpr int WALK_RANGES = 16;   // preorder ranges of the walk (at most)

// The preorder ranges of the walk: range r = [klo[r], klo[r + 1]), equal
// node counts; for each range start its strict ancestors (root first), so a
// walk of the range knows where in it a bucket's own walk resumes.
// Range r starts at node k0 = r nn / M; its strict ancestors, root first, at
// most WALK_ANC of them.  Node j is a strict ancestor of k0 iff j < k0 <
// j + size(j), and a node's level is its depth (children are one level
// below their parent), so the ancestor at depth d is the one of level d and
// k0 has level(k0) of them: every (range, node) pair is tested on its own.
__global__ void k_walk_ranges(const uint4 *W, uint32_t nn, uint32_t M, uint32_t *klo,
                              uint32_t *anc, uint32_t *nanc)
{
    GRID_STRIDE(t, (uint64_t)M * nn) {
        const uint32_t r = (uint32_t)(t / nn), j = (uint32_t)(t - (uint64_t)r * nn);
        const uint32_t k0 = (uint32_t)((uint64_t)r * nn / M);
        if (j == 0) {
            klo[r] = k0;
            nanc[r] = min(W[k0].y >> 22, (uint32_t)WALK_ANC);
            if (r == 0) klo[M] = nn;
        }
        if (j < k0) {
            const uint4 R = W[j];
            const uint32_t l = R.y >> 22;
            if (j + (R.x & 0x7FFFFFFFu) > k0 && l < (uint32_t)WALK_ANC) anc[r * WALK_ANC + l] = j;
        }
    }
}

// Does the bucket (its leaf node lf, box lo..hi) accept node k (record R)
// as a whole?  Nodes containing the bucket are always opened.
__device__ __forceinline__ bool walk_accepts(uint32_t k, const uint4 &R, uint32_t lf,
                                             const int4 &lo, const int4 &hi, const int64_t *th)
{
    const uint32_t size = R.x & 0x7FFFFFFFu;
    if (k <= lf && lf < k + size) return false;
    const int cx = (int)(R.y & 0x3FFFFFu), cy = (int)(R.z & 0x3FFFFFu), cz = (int)R.w;
    const uint32_t dx = (uint32_t)max(0, max(lo.x - cx, cx - hi.x));
    const uint32_t dy = (uint32_t)max(0, max(lo.y - cy, cy - hi.y));
    const uint32_t dz = (uint32_t)max(0, max(lo.z - cz, cz - hi.z));
    const uint64_t d2 = (uint64_t)dx * dx + (uint64_t)dy * dy + (uint64_t)dz * dz;
    return (int64_t)d2 > th[R.y >> 22];
}

// Walk of one preorder range [klo[r], klo[r + 1]) for one bucket, one thread
// per (bucket, range) item.  Items run range-major, so a warp walks the same
// range for 32 consecutive buckets (neighbours in Morton order, similar
// paths).  The walk visits nodes in preorder with skips (no stack): an
// accepted node or an opened leaf continues after its subtree (k + size),
// an opened internal node (containing the bucket or failing the acceptance
// test) at k + 1.  Before the range, the strict ancestors of its first node
// are tested, root first: if the bucket accepts one, its walk resumes only
// where that ancestor's subtree ends (which may be inside the range or
// beyond it).  A node is emitted by the range that holds it, so the ranges'
// lists, concatenated in range order, are the depth-first list of the
// bucket's own walk.  The walk is bound by the L1 traffic of its node reads
// (lanes read different nodes): one 16-byte record per visited node, read
// after the decision; the many resident warps hide its latency.  FILL =
// false: lengths into len[b M + r]; true: entries written at off[b M + r].
// Write out the entries a lane has gathered in its 16-byte group: slot q of
// the group holds list entry (cnt - 1) - (last slot - q).
__device__ __forceinline__ void walk_flush_group(uint32_t *o, uint32_t cnt, uint32_t a0,
                                                 uint32_t &gmask, const uint32_t *g)
{
    const uint32_t sl = (a0 + cnt - 1) & 3u;
    for (uint32_t q = 0; q < 4; ++q)
        if ((gmask >> q) & 1u) o[cnt - 1 - (sl - q)] = g[q];
    gmask = 0;
}

// Launched with 128 threads per block (the per-lane groups below).
template <bool FILL>
__global__ void __launch_bounds__(128, 8) k_walk(const uint4 *W, const uint2 *LF, uint32_t M,
                                                 const uint32_t *klo, const uint32_t *anc,
                                                 const uint32_t *nanc, WalkThresholds thg,
                                                 const uint4 *bucket, const int4 *blo,
                                                 const int4 *bhi, uint64_t nb,
                                                 const uint32_t *sorted_ids, uint32_t n_part,
                                                 uint32_t *len, const uint64_t *off,
                                                 uint32_t *out)
{
    __shared__ int64_t th[22];
    __shared__ __align__(16) uint32_t grp[128][4];
    if (threadIdx.x < 22) th[threadIdx.x] = thg.t[threadIdx.x];
    __syncthreads();
    uint32_t *g = grp[threadIdx.x];
    GRID_STRIDE(t, nb * M) {
        const uint32_t r = (uint32_t)(t / nb);
        const uint64_t b = t - (uint64_t)r * nb;
        const uint32_t lf = bucket[b].z;
        const int4 lo = blo[b], hi = bhi[b];
        uint32_t k = klo[r];
        const uint32_t k1 = klo[r + 1];
        const uint32_t na = nanc[r];
        for (uint32_t j = 0; j < na; ++j) {
            const uint32_t a = anc[r * WALK_ANC + j];
            const uint4 R = W[a];
            if (walk_accepts(a, R, lf, lo, hi, th)) {
                k = max(k, a + (R.x & 0x7FFFFFFFu));
                break;
            }
        }
        uint32_t cnt = 0;
        uint32_t *o = FILL ? out + off[b * M + r] : nullptr;
        // Accepted-node entries gather in 16-byte groups aligned in the list
        // (a lane's shared-memory row) and leave as one vector store: one
        // scattered 4-byte store per entry was most of the fill pass's cost.
        // A leaf copy and the end of the walk write out a partial group.
        const uint32_t a0 = FILL ? (uint32_t)(((uintptr_t)o >> 2) & 3u) : 0u;
        uint32_t gmask = 0;
        while (k < k1) {
            const uint4 R = W[k];
            const uint32_t size = R.x & 0x7FFFFFFFu;
            if (walk_accepts(k, R, lf, lo, hi, th)) {
                if (FILL) {
                    const uint32_t slot = (a0 + cnt) & 3u;
                    g[slot] = n_part + k;
                    gmask |= 1u << slot;
                    if (slot == 3) {
                        if (gmask == 0xFu)
                            *reinterpret_cast<uint4 *>(o + cnt - 3) =
                                *reinterpret_cast<const uint4 *>(g);
                        else
                            walk_flush_group(o, cnt + 1, a0, gmask, g);
                        gmask = 0;
                    }
                }
                ++cnt;
                k += size;
            } else if (R.x >> 31 && !FILL) {   // leaf: its particle count
                uint32_t ln = R.z >> 22;
                if (ln == WALK_LEAF_FAR) ln = LF[k].y;
                cnt += ln;
                k += size;
            } else if (R.x >> 31) {      // leaf: its particles
                const uint2 L = LF[k];
                if (FILL && gmask) walk_flush_group(o, cnt, a0, gmask, g);
                if (FILL) {   // 16 loads in flight before their stores
                    const uint32_t *src = sorted_ids + L.x;
                    uint32_t *dst = o + cnt;
                    for (uint32_t q0 = 0; q0 < L.y; q0 += 16) {
                        uint32_t v[16];
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            if (q0 + u < L.y) v[u] = src[q0 + u];
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            if (q0 + u < L.y) dst[q0 + u] = v[u];
                    }
                }
                cnt += L.y;
                k += size;
            } else {
                k += 1;
            }
        }
        if (FILL && gmask) walk_flush_group(o, cnt, a0, gmask, g);
        if (!FILL) len[b * M + r] = cnt;
    }
}

__global__ void k_u32_to_u64(const uint32_t *in, uint64_t *out, uint64_t n)
{
    GRID_STRIDE(i, n) out[i] = in[i];
}

// per-bucket list offsets from the per-(bucket, range) offsets (the ranges
// of a bucket are adjacent)
__global__ void k_bucket_offsets(const uint64_t *ioff, uint64_t nb, uint32_t M, uint64_t *loff)
{
    GRID_STRIDE(b, nb + 1) loff[b] = ioff[b * M];
}

__global__ void k_nbody_tasks(const uint4 *bucket, uint64_t nb, const uint64_t *list_off,
                              uint64_t tgt_base, uint64_t src_base, uint64_t id_base,
                              TaskRec *out)
{
    GRID_STRIDE(b, nb) {
        TaskRec r;
        uint4 B = bucket[b];
        r.task_id = id_base + b;
        r.tgt_off = tgt_base + B.x;
        r.src_off = src_base + list_off[b];
        r.row_off = 0;
        r.kind = GC_GRAVITY;
        r.nt = B.y;
        r.ns = (uint32_t)(list_off[b + 1] - list_off[b]);
        r.shift[0] = r.shift[1] = r.shift[2] = r.shift[3] = 0;
        out[b] = r;
    }
}

// One leapfrog step (kick then drift) per particle: v' = fl(v + a dt),
// x' = fl(x + v' dt), FP64 arithmetic without contraction, float32 state.
__global__ void k_kick_drift(const gcd4 *acc, float4 *x, float4 *v, uint64_t n, double dt)
{
    GRID_STRIDE(i, n) {
        const gcd4 a = acc[i];
        float4 xi = x[i], vi = v[i];
        vi.x = (float)__dadd_rn((double)vi.x, __dmul_rn(a.x, dt));
        vi.y = (float)__dadd_rn((double)vi.y, __dmul_rn(a.y, dt));
        vi.z = (float)__dadd_rn((double)vi.z, __dmul_rn(a.z, dt));
        xi.x = (float)__dadd_rn((double)xi.x, __dmul_rn((double)vi.x, dt));
        xi.y = (float)__dadd_rn((double)xi.y, __dmul_rn((double)vi.y, dt));
        xi.z = (float)__dadd_rn((double)xi.z, __dmul_rn((double)vi.z, dt));
        v[i] = vi;
        x[i] = xi;
    }
}

// Current values of ids 0..n-1 in id order: a resident id's pool slot, else
// its entry of the host mirror (mapped memory, read over the host link).
__global__ void k_values_of_ids(const uint32_t *slot_of_id, const float4 *pool,
                                const float4 *mirror, uint64_t n, float4 *out)
{
    GRID_STRIDE(i, n) {
        const uint32_t s = slot_of_id[i];
        out[i] = s != GC_NONE ? pool[s] : mirror[i];
    }
}

// Sorted keys and ids (keys2, ids2) of the n particles x, seeded by the
// permutation ids2 holds from the previous build of the same n.  *done is
// false (nothing written) when a slot collected more than SEED_GROUP_MAX
// movers; *movers receives the number of particles placed afresh.
int seeded_order(gc_pool *p, const float4 *x, uint64_t n, const GridParams *gp,
                 uint64_t *movers, bool *done)
{
    NBodyState &S = p->nb;
    cudaStream_t s = p->s;
    const int maxb = p->num_sms * 16;
    const uint64_t nt = (n + SEED_TILE - 1) / SEED_TILE;
    *done = false;
    GC_TRY(S.seed_tiles.reserve(nt * sizeof(SeedTile) + sizeof(SeedCtr) + 64));
    GC_TRY(S.seed_a.reserve((n + 1) * 8 + 64));
    GC_TRY(S.seed_m.reserve(n * 24 + 64));
    GC_TRY(S.seed_key.reserve(n * 12 + 64));
    SeedTile *tiles = S.seed_tiles.as<SeedTile>();
    SeedCtr *ctr = reinterpret_cast<SeedCtr *>(tiles + nt);
    uint64_t *KT = S.keys.as<uint64_t>();       // tile remainders, slot = tile * SEED_TILE + j
    uint32_t *IT = S.ids.as<uint32_t>();
    uint32_t *W = S.seed_a.as<uint32_t>(), *E = W + (n + 1);
    uint64_t *MK = S.seed_m.as<uint64_t>();     // movers: key, id, tile, slot, arrival
    uint32_t *MI = reinterpret_cast<uint32_t *>(MK + n);
    uint32_t *MH = MI + n, *MS = MH + n, *MA = MS + n;
    uint64_t *TK = S.seed_key.as<uint64_t>();   // movers in their slots' ranges
    uint32_t *TI = reinterpret_cast<uint32_t *>(TK + n);

    GC_CUDA_TRY(cudaMemsetAsync(ctr, 0, sizeof(SeedCtr), s));
    GC_CUDA_TRY(cudaMemsetAsync(W + n, 0, 4, s));
    p->stats.kernel_launches += 4;
    k_seed_tiles<<<(unsigned)nt, SEED_THREADS, 0, s>>>(x, S.ids2.as<uint32_t>(), n, gp, KT, IT,
                                                       W, tiles, ctr, MK, MI, MH);
    k_seed_scan<<<1, 1024, 0, s>>>(tiles, (uint32_t)nt);
    k_seed_low<<<(unsigned)((nt + 7) / 8), 256, 0, s>>>(KT, IT, tiles, (uint32_t)nt, W, ctr, MK,
                                                        MI, MH);
    k_mover_slot<<<(unsigned)(p->num_sms * 8), 256, 0, s>>>(ctr, MK, MI, MH, KT, IT, tiles,
                                                            (uint32_t)nt, n, W, MS, MA);
    SeedCtr h{};
    GC_CUDA_TRY(cudaMemcpyAsync(&h, ctr, sizeof h, cudaMemcpyDeviceToHost, s));
    GC_CUDA_TRY(cudaStreamSynchronize(s));
    if (h.movers > n) return GC_ERR_CUDA;          // every particle is kept or moved, once
    if (h.max_group > SEED_GROUP_MAX) return GC_OK;   // sort all keys instead
    const uint64_t m = h.movers;
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u32(S.cub_tmp, W, E, n + 1, s));
    if (m) {
        ++p->stats.kernel_launches;
        k_mover_scatter<<<grid_for(m, 256, maxb), 256, 0, s>>>(MK, MI, MS, MA, m, E, TK, TI);
    }
    S.order_n = 0;   // ids2 is rewritten below
    ++p->stats.kernel_launches;
    k_seed_place<<<grid_for(n + m, 256, maxb), 256, 0, s>>>(
        KT, IT, tiles, n, W, E, MK, MI, MS, m, TK, TI, S.keys2.as<uint64_t>(),
        S.ids2.as<uint32_t>());
    GC_CUDA_TRY(cudaGetLastError());
    *movers = m;
    *done = true;
    return GC_OK;
}

// Fold a completed build's event times into the sums.
int nbody_timing_fold(NBodyState &S)
{
    if (!S.ev_pending) return GC_OK;
    GC_CUDA_TRY(cudaEventSynchronize(S.ev[2]));
    float a = 0.f, b = 0.f;
    GC_CUDA_TRY(cudaEventElapsedTime(&a, S.ev[0], S.ev[1]));
    GC_CUDA_TRY(cudaEventElapsedTime(&b, S.ev[0], S.ev[2]));
    S.last_order_ms = a;
    S.last_tree_ms = b;
    S.order_ms_sum += a;
    S.tree_ms_sum += b;
    ++S.timed_builds;
    S.ev_pending = false;
    return GC_OK;
}

}  // namespace

extern "C" int gc_build_nbody_tasks_resident(gc_pool_t *p, uint64_t n, int bucket_max,
                                             int theta_num, int theta_den,
                                             uint64_t task_id_base, uint64_t info_out[4])
{
    if (!p || n == 0 || n > 0x7FFFFFFFull) return GC_ERR_ARG;
    if (n >= p->cfg.id_capacity) return GC_ERR_POOL_FULL;
    NBodyState &S = p->nb;
    GC_TRY(S.hostcopy.reserve(n * sizeof(float4)));
    ++p->stats.kernel_launches;
    k_values_of_ids<<<grid_for(n, 256, p->num_sms * 16), 256, 0, p->s>>>(
        p->d_slot_of_id, p->d_pool, p->d_mirror, n, S.hostcopy.as<float4>());
    GC_CUDA_TRY(cudaGetLastError());
    return gc_build_nbody_tasks(p, S.hostcopy.as<float>(), n, bucket_max, theta_num, theta_den,
                                task_id_base, info_out);
}

extern "C" int gc_build_nbody_tasks(gc_pool_t *p, const float *xyzm_dev, uint64_t n,
                                    int bucket_max, int theta_num, int theta_den,
                                    uint64_t task_id_base, uint64_t info_out[4])
{
    if (!p || !xyzm_dev || n == 0 || n > 0x7FFFFFFFull || bucket_max < 1 || bucket_max > 4096 ||
        theta_num < 0 || theta_num > 255 || theta_den < 1 || theta_den > 255)
        return GC_ERR_ARG;
    if (((uintptr_t)xyzm_dev) % 16) return GC_ERR_ARG;
    if (n >= p->cfg.id_capacity) return GC_ERR_POOL_FULL;
    NBodyState &S = p->nb;
    GC_TRY(nbody_timing_fold(S));
    for (cudaEvent_t &e : S.ev)
        if (!e) GC_CUDA_TRY(cudaEventCreate(&e));
    GC_CUDA_TRY(cudaEventRecord(S.ev[0], p->s));
    int vrc = GC_OK;
    xyzm_dev = (const float *)gc_device_view(p, xyzm_dev, n * sizeof(float4), S.hostcopy, &vrc);
    if (vrc != GC_OK) return vrc;
    cudaStream_t s = p->s;
    const int B = bucket_max;
    const int maxb = p->num_sms * 16;
    const float4 *x = (const float4 *)xyzm_dev;

    GC_TRY(S.bounds.reserve(64 + sizeof(GridParams)));
    GC_TRY(S.keys.reserve(n * 8));
    GC_TRY(S.keys2.reserve(n * 8));
    GC_TRY(S.ids.reserve(n * 4));
    GC_TRY(S.ids2.reserve(n * 4));
    GC_TRY(S.lcp.reserve(n + 1));
    GC_TRY(S.win.reserve(n + 1));
    GC_TRY(S.dmax.reserve(n + 1));
    GC_TRY(S.nnode.reserve((n + 1) * 4));
    GC_TRY(S.node_off.reserve((n + 1) * 4));

    uint32_t *bounds = S.bounds.as<uint32_t>();
    GridParams *gp = (GridParams *)(S.bounds.as<char>() + 64);
    uint32_t init[6] = {0xFFFFFFFFu, 0xFFFFFFFFu, 0xFFFFFFFFu, 0, 0, 0};
    GC_CUDA_TRY(cudaMemcpyAsync(bounds, init, sizeof init, cudaMemcpyHostToDevice, s));
    ++p->stats.kernel_launches;
    k_bbox<<<grid_for(n, 256, maxb), 256, 0, s>>>(x, n, bounds);
    ++p->stats.kernel_launches;
    k_grid_params<<<1, 1, 0, s>>>(bounds, gp);
    // Morton order: seeded by the previous build's order of the same n
    // particles, else a full stable radix sort of the keys
    bool seeded = false;
    uint64_t resorted = n;
    if (S.order_mode == GC_ORDER_SEEDED && S.order_n == n)
        GC_TRY(seeded_order(p, x, n, gp, &resorted, &seeded));
    if (!seeded) {
        resorted = n;
        ++p->stats.kernel_launches;
        k_keys<<<grid_for(n, 256, maxb), 256, 0, s>>>(x, n, gp, S.keys.as<uint64_t>(),
                                                      S.ids.as<uint32_t>());
        S.order_n = 0;
        ++p->stats.primitive_calls;
        GC_TRY(gc_sort_pairs_u64(S.cub_tmp, S.keys.as<uint64_t>(), S.keys2.as<uint64_t>(),
                                 S.ids.as<uint32_t>(), S.ids2.as<uint32_t>(), n, 63, s));
    }
    S.order_n = n;
    GC_CUDA_TRY(cudaEventRecord(S.ev[1], s));
    const uint64_t *K = S.keys2.as<uint64_t>();
    const uint32_t *sid = S.ids2.as<uint32_t>();
    ++p->stats.kernel_launches;
    k_lcp_win<<<grid_for(n, 256, maxb), 256, 0, s>>>(K, n, B, S.lcp.as<int8_t>(),
                                                     S.win.as<int8_t>());
    ++p->stats.kernel_launches;
    k_dmax<<<grid_for(n, 256, maxb), 256, 0, s>>>(S.lcp.as<int8_t>(), S.win.as<int8_t>(), n, B,
                                                  S.dmax.as<int8_t>(), S.nnode.as<uint32_t>());
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u32(S.cub_tmp, S.nnode.as<uint32_t>(), S.node_off.as<uint32_t>(),
                                 n + 1, s));
    uint32_t NN = 0;
    GC_CUDA_TRY(cudaMemcpyAsync(&NN, S.node_off.as<uint32_t>() + n, 4, cudaMemcpyDeviceToHost, s));
    GC_CUDA_TRY(cudaStreamSynchronize(s));
    if ((uint64_t)n + NN > p->cfg.id_capacity) return GC_ERR_POOL_FULL;

    GC_TRY(S.node_a.reserve((uint64_t)NN * 16 + 16));
    GC_TRY(S.node_b.reserve((uint64_t)NN * 16 + 16));
    GC_TRY(S.node_val.reserve((uint64_t)NN * 16 + 16));
    GC_TRY(S.list_len.reserve(((uint64_t)NN + 1) * 4 * 2));   // bucket counts, then offsets
    uint32_t *bcnt = S.list_len.as<uint32_t>();
    uint32_t *boff = bcnt + (NN + 1);
    GC_CUDA_TRY(cudaMemsetAsync(bcnt + NN, 0, 4, s));
    ++p->stats.kernel_launches;
    k_emit_nodes<<<grid_for(n, 256, maxb), 256, 0, s>>>(
        K, n, S.lcp.as<int8_t>(), S.dmax.as<int8_t>(), S.node_off.as<uint32_t>(),
        S.node_a.as<uint4>(), S.node_b.as<uint4>(), bcnt, B);
    const uint64_t n_m4 = n + 1, n_tiles = (n_m4 + M4_TILE - 1) / M4_TILE;
    GC_TRY(S.mono.reserve((n_m4 * 2 + n_tiles) * sizeof(M4)));
    M4 *mono_in = S.mono.as<M4>(), *mono_pre = mono_in + n_m4, *tiles = mono_pre + n_m4;
    ++p->stats.kernel_launches;
    k_mono_input<<<grid_for(n + 1, 256, maxb), 256, 0, s>>>(sid, x, n, mono_in);
    p->stats.kernel_launches += 3;
    k_m4_tile_sum<<<(unsigned)n_tiles, M4_THREADS, 0, s>>>(mono_in, n_m4, tiles);
    k_m4_scan_tiles<<<1, M4_THREADS, 0, s>>>(tiles, n_tiles);
    k_m4_tile_scan<<<(unsigned)n_tiles, M4_THREADS, 0, s>>>(mono_in, n_m4, tiles, mono_pre);
    ++p->stats.kernel_launches;
    k_mono_nodes<<<grid_for(NN, 256, maxb), 256, 0, s>>>(S.node_a.as<uint4>(), NN, mono_pre,
                                                         S.node_val.as<float4>());
    GC_TRY(gc_launch_upload_seq(p, (uint32_t)n, S.node_val.as<float4>(), NN));
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u32(S.cub_tmp, bcnt, boff, (uint64_t)NN + 1, s));
    uint32_t NB = 0;
    GC_CUDA_TRY(cudaMemcpyAsync(&NB, boff + NN, 4, cudaMemcpyDeviceToHost, s));
    GC_CUDA_TRY(cudaStreamSynchronize(s));

    GC_TRY(S.bucket.reserve((uint64_t)NB * 16 + 16));
    GC_TRY(S.bbox.reserve((uint64_t)NB * 32 + 32));
    int4 *blo = S.bbox.as<int4>(), *bhi = blo + NB;
    ++p->stats.kernel_launches;
    k_emit_buckets<<<grid_for(NN, 256, maxb), 256, 0, s>>>(S.node_a.as<uint4>(), NN, boff, K, B,
                                                           S.bucket.as<uint4>(), blo, bhi);
    const int64_t tn2 = (int64_t)theta_num * theta_num, td2 = (int64_t)theta_den * theta_den;
    WalkThresholds th;
    for (int l = 0; l < 22; ++l) {
        const int64_t sz = (int64_t)1 << (22 - l);
        th.t[l] = tn2 ? (td2 * sz * sz) / tn2 : INT64_MAX;
    }
    // walk records and ranges (about 512 nodes per range or more)
    const uint32_t M = (uint32_t)std::max<uint64_t>(1, std::min<uint64_t>(WALK_RANGES, NN / 512));
    const uint64_t NI = (uint64_t)NB * M;                      // (bucket, range) lists
    GC_TRY(S.wnode.reserve(((uint64_t)NN + 1) * 24 + (uint64_t)(M + 1) * 4 +
                           (uint64_t)M * (WALK_ANC + 1) * 4));
    uint4 *W = S.wnode.as<uint4>();
    uint2 *LF = (uint2 *)(W + ((uint64_t)NN + 1));
    uint32_t *klo = (uint32_t *)(LF + ((uint64_t)NN + 1));
    uint32_t *anc = klo + (M + 1), *nanc = anc + (uint64_t)M * WALK_ANC;
    ++p->stats.kernel_launches;
    k_walk_nodes<<<grid_for((uint64_t)NN + 1, 256, maxb), 256, 0, s>>>(
        S.node_a.as<uint4>(), S.node_b.as<uint4>(), NN, W, LF);
    ++p->stats.kernel_launches;
    k_walk_ranges<<<grid_for((uint64_t)M * NN, 256, maxb), 256, 0, s>>>(W, NN, M, klo, anc, nanc);
    GC_TRY(S.list_off.reserve((NI + 1) * 8 * 2 + ((uint64_t)NB + 1) * 8));
    GC_TRY(S.win.reserve((NI + 1) * 4));   // reused: (bucket, range) list lengths
    uint32_t *llen = S.win.as<uint32_t>();
    uint64_t *llen64 = S.list_off.as<uint64_t>();
    uint64_t *ioff = llen64 + (NI + 1);                       // per-(bucket, range) offsets
    uint64_t *loff = ioff + (NI + 1);                         // per-bucket offsets
    const unsigned walk_blocks = grid_for(NI, 128, 1 << 20);
    ++p->stats.kernel_launches;
    k_walk<false><<<walk_blocks, 128, 0, s>>>(W, LF, M, klo, anc, nanc, th, S.bucket.as<uint4>(),
                                              blo, bhi, NB, sid, (uint32_t)n, llen, nullptr,
                                              nullptr);
    GC_CUDA_TRY(cudaMemsetAsync(llen + NI, 0, 4, s));
    ++p->stats.kernel_launches;
    k_u32_to_u64<<<grid_for(NI + 1, 256, maxb), 256, 0, s>>>(llen, llen64, NI + 1);
    ++p->stats.primitive_calls;
    GC_TRY(gc_exclusive_scan_u64(S.cub_tmp, llen64, ioff, NI + 1, s));
    ++p->stats.kernel_launches;
    k_bucket_offsets<<<grid_for((uint64_t)NB + 1, 256, maxb), 256, 0, s>>>(ioff, NB, M, loff);
    uint64_t NL = 0;
    GC_CUDA_TRY(cudaMemcpyAsync(&NL, loff + NB, 8, cudaMemcpyDeviceToHost, s));
    GC_CUDA_TRY(cudaStreamSynchronize(s));

    // append the tasks to the pending batch
    const bool batch_start = p->nb_tasks == 0;
    GC_TRY(gc_reserve_batch(p, NB, n, NL));
    uint32_t *dt = p->tgt_ids.as<uint32_t>() + p->nb_tgt;
    uint32_t *ds = p->src_ids.as<uint32_t>() + p->nb_src;
    TaskRec *recs = p->tasks.as<TaskRec>() + p->nb_tasks;
    ++p->stats.kernel_launches;
    k_walk<true><<<walk_blocks, 128, 0, s>>>(W, LF, M, klo, anc, nanc, th, S.bucket.as<uint4>(),
                                             blo, bhi, NB, sid, (uint32_t)n, nullptr, ioff, ds);
    GC_CUDA_TRY(cudaMemcpyAsync(dt, sid, n * 4, cudaMemcpyDeviceToDevice, s));
    ++p->stats.kernel_launches;
    k_nbody_tasks<<<grid_for(NB, 256, maxb), 256, 0, s>>>(S.bucket.as<uint4>(), NB, loff,
                                                          p->nb_tgt, p->nb_src, task_id_base,
                                                          recs);
    GC_CUDA_TRY(cudaGetLastError());
    p->nb_tasks += NB;
    p->nb_tgt += n;
    p->nb_src += NL;
    // a batch that holds exactly these tasks has one row per particle
    p->nb_pend_tasks = batch_start ? NB : 0;
    S.n = n;
    S.n_nodes = NN;
    S.n_buckets = NB;
    S.n_list = NL;
    S.n_walk_items = NI;
    GC_CUDA_TRY(cudaEventRecord(S.ev[2], s));
    S.ev_pending = true;
    ++S.builds;
    if (seeded) ++S.seeded_builds;
    S.last_resorted = resorted;
    if (info_out) {
        info_out[0] = NN;
        info_out[1] = NB;
        info_out[2] = NL;
        info_out[3] = resorted;
    }
    return GC_OK;
}

extern "C" int gc_nbody_set_order(gc_pool_t *p, int mode)
{
    if (!p || (mode != GC_ORDER_FULL && mode != GC_ORDER_SEEDED)) return GC_ERR_ARG;
    p->nb.order_mode = mode;
    return GC_OK;
}

extern "C" int gc_nbody_stats(gc_pool_t *p, gc_nbody_stats_t *out)
{
    if (!p || !out) return GC_ERR_ARG;
    NBodyState &S = p->nb;
    GC_TRY(nbody_timing_fold(S));
    out->builds = S.builds;
    out->seeded_builds = S.seeded_builds;
    out->last_resorted = S.last_resorted;
    out->timed_builds = S.timed_builds;
    out->last_order_ms = S.last_order_ms;
    out->last_tree_ms = S.last_tree_ms;
    out->order_ms_sum = S.order_ms_sum;
    out->tree_ms_sum = S.tree_ms_sum;
    return GC_OK;
}

extern "C" int gc_read_nbody_tree(gc_pool_t *p, uint32_t *sorted_ids, uint64_t *sorted_keys,
                                  uint8_t *level, uint32_t *cell3, uint32_t *first,
                                  uint32_t *count, uint8_t *leaf, uint32_t *size,
                                  float *node_xyzm, uint32_t *bucket_first,
                                  uint32_t *bucket_count, uint32_t *bucket_node,
                                  uint64_t *list_off, uint32_t *list_ids)
{
    if (!p || p->nb.n == 0) return GC_ERR_STATE;
    NBodyState &S = p->nb;
    GC_CUDA_TRY(cudaStreamSynchronize(p->s));
    const uint64_t n = S.n, NN = S.n_nodes, NB = S.n_buckets;
    if (sorted_ids) GC_CUDA_TRY(cudaMemcpy(sorted_ids, S.ids2.p, n * 4, cudaMemcpyDeviceToHost));
    if (sorted_keys) GC_CUDA_TRY(cudaMemcpy(sorted_keys, S.keys2.p, n * 8, cudaMemcpyDeviceToHost));
    if (level || first || count || leaf || size || cell3) {
        std::vector<uint4> a(NN), b(NN);
        GC_CUDA_TRY(cudaMemcpy(a.data(), S.node_a.p, NN * 16, cudaMemcpyDeviceToHost));
        GC_CUDA_TRY(cudaMemcpy(b.data(), S.node_b.p, NN * 16, cudaMemcpyDeviceToHost));
        for (uint64_t k = 0; k < NN; ++k) {
            if (first) first[k] = a[k].x;
            if (count) count[k] = a[k].y;
            if (size) size[k] = a[k].z;
            if (level) level[k] = (uint8_t)(a[k].w & 255u);
            if (leaf) leaf[k] = (uint8_t)((a[k].w >> 8) & 1u);
            if (cell3) {
                cell3[3 * k] = b[k].x;
                cell3[3 * k + 1] = b[k].y;
                cell3[3 * k + 2] = b[k].z;
            }
        }
    }
    if (node_xyzm) GC_CUDA_TRY(cudaMemcpy(node_xyzm, S.node_val.p, NN * 16, cudaMemcpyDeviceToHost));
    if (bucket_first || bucket_count || bucket_node) {
        std::vector<uint4> bk(NB);
        GC_CUDA_TRY(cudaMemcpy(bk.data(), S.bucket.p, NB * 16, cudaMemcpyDeviceToHost));
        for (uint64_t b = 0; b < NB; ++b) {
            if (bucket_first) bucket_first[b] = bk[b].x;
            if (bucket_count) bucket_count[b] = bk[b].y;
            if (bucket_node) bucket_node[b] = bk[b].z;
        }
    }
    const uint64_t *loff = S.list_off.as<uint64_t>() + 2 * (S.n_walk_items + 1);
    if (list_off) GC_CUDA_TRY(cudaMemcpy(list_off, loff, (NB + 1) * 8, cudaMemcpyDeviceToHost));
    if (list_ids) {
        // the lists live in the batch source array (pending, or last flushed)
        const uint32_t *src = nullptr;
        uint64_t base = 0;
        if (p->nb_src >= S.n_list && p->nb_tasks >= NB) {
            src = p->src_ids.as<uint32_t>();
            base = p->nb_src - S.n_list;
        } else if (p->last >= 0 && p->ctx[p->last].valid && p->ctx[p->last].n_src >= S.n_list) {
            const FlushCtx &c = p->ctx[p->last];
            GC_CUDA_TRY(cudaEventSynchronize(c.ev_done));
            src = c.src_ids.as<uint32_t>();
            base = c.n_src - S.n_list;
        }
        if (!src) return GC_ERR_STATE;
        GC_CUDA_TRY(cudaMemcpy(list_ids, src + base, S.n_list * 4, cudaMemcpyDeviceToHost));
    }
    return GC_OK;
}

// One time step around the force computation (Section 4.1): leapfrog kick
// with the accelerations acc (4 doubles per particle, e.g. the pool's
// per-id totals after the step's flush), drift, and the new positions
// uploaded into the pool in place (ids 0..n-1).
extern "C" int gc_nbody_kick_drift(gc_pool_t *p, const double *acc_dev, float *xyzm_dev,
                                   float *vel_dev, uint64_t n, double dt)
{
    if (!p || !acc_dev || !xyzm_dev || !vel_dev) return GC_ERR_ARG;
    if (n == 0) return GC_OK;
    if (n > p->cfg.id_capacity || ((uintptr_t)xyzm_dev | (uintptr_t)vel_dev) % 16 ||
        ((uintptr_t)acc_dev) % 32)
        return GC_ERR_ARG;
    GC_TRY(order_after_scatters(p));   // the accelerations of batches in flight
    GC_TRY(gc_apply_totals_reset(p, p->s));
    ++p->stats.kernel_launches;
    k_kick_drift<<<grid_for(n, 256, p->num_sms * 16), 256, 0, p->s>>>(
        (const gcd4 *)acc_dev, (float4 *)xyzm_dev, (float4 *)vel_dev, n, dt);
    GC_CUDA_TRY(cudaGetLastError());
    return gc_launch_upload_seq(p, 0, (const float4 *)xyzm_dev, n);
}
