// Counting kernels of libtc: edge sampling with degrees (Section 3.1), the
// degree partition (Section 3.2), source bucketing and the sorted-list
// intersections that count the triangles of both classes.
//
// Counting scheme.  Every kept edge is directed from the endpoint of lower
// (deg_p, id) to the higher one, so each triangle {a, b, c} with
// rank(a) < rank(b) < rank(c) is seen exactly once: at source a, middle
// vertex b in N+(a), and c in N+(a) n N+(b).  Light vertices have lower
// degree than heavy ones, so a triangle has a light vertex iff its lowest
// vertex a is light: T_L sums |N+(a) n N+(b)| over light sources a, T_H over
// heavy sources (whose out-neighbours are all heavy).
#include "kernels.h"

namespace tcg {

// ======================================================================
// Sampling + degrees
// ======================================================================

__device__ __forceinline__ uint32_t sample_one(uint64_t k, uint64_t seed_mix, uint64_t thr,
                                               uint32_t *__restrict__ deg)
{
    if (!keep_edge(k, seed_mix, thr)) return 0;
    atomicAdd(deg + (k >> 32), 1u);
    atomicAdd(deg + (uint32_t)k, 1u);
    return 1;
}

__global__ void __launch_bounds__(256) k_sample_degree(const uint64_t *__restrict__ ekey, uint64_t m,
                                                       uint64_t seed_mix, uint64_t thr,
                                                       uint32_t *__restrict__ deg, DevState *st)
{
    uint32_t kept = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const ulonglong2 *e2 = reinterpret_cast<const ulonglong2 *>(ekey);
    for (uint64_t i = tid; i < m / 2; i += stride) {
        const ulonglong2 k = ld_stream_u64x2(e2 + i);
        kept += sample_one(k.x, seed_mix, thr, deg);
        kept += sample_one(k.y, seed_mix, thr, deg);
    }
    if ((m & 1) && tid == 0) kept += sample_one(ekey[m - 1], seed_mix, thr, deg);
    kept = warp_sum(kept);
    if (lane_id() == 0 && kept) atomicAdd(&st->m_sampled, (unsigned long long)kept);
}

static unsigned grid_for(uint64_t work, int threads, unsigned cap)
{
    uint64_t b = ceil_div(work, (uint64_t)threads);
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

void sample_degree(const CountBuffers &b, uint64_t seed_mix, uint64_t thr, cudaStream_t s)
{
    if (b.m == 0) return;
    k_sample_degree<<<grid_for(b.m / 2 + 1, 256, 152 * 8), 256, 0, s>>>(b.ekey, b.m, seed_mix, thr, b.deg,
                                                                        b.st); note_launch();
}

// ======================================================================
// Degree partition: heavy <=> deg_p^2 > m_p (Section 3.2, in integers)
// ======================================================================

__global__ void k_partition(const uint32_t *__restrict__ deg, uint32_t n, DevState *st,
                            uint8_t *__restrict__ heavy)
{
    const unsigned long long mp = st->m_sampled;
    uint32_t h = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const unsigned long long d = deg[u];
        const uint8_t f = d * d > mp;
        heavy[u] = f;
        h += f;
    }
    h = warp_sum(h);
    if (lane_id() == 0 && h) atomicAdd(&st->n_heavy, h);
}

void partition(const CountBuffers &b, cudaStream_t s)
{
    k_partition<<<grid_for(b.n, 256, 152 * 8), 256, 0, s>>>(b.deg, b.n, b.st, b.heavy); note_launch();
}

// ======================================================================
// Kept-edge list in canonical order (inspection entry point only)
// ======================================================================

constexpr int KC_THREADS = 1024;
constexpr int KC_ITEMS = RX_TILE / KC_THREADS;

__global__ void __launch_bounds__(KC_THREADS) k_kept_count(const uint64_t *__restrict__ ekey, uint64_t m,
                                                           uint64_t seed_mix, uint64_t thr,
                                                           uint32_t *__restrict__ tile_cnt)
{
    __shared__ uint32_t wt[33];
    const uint64_t base = (uint64_t)blockIdx.x * RX_TILE;
    uint32_t c = 0;
    for (int j = 0; j < KC_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * KC_THREADS + threadIdx.x;
        if (i < m && keep_edge(ekey[i], seed_mix, thr)) ++c;
    }
    c = block_sum(c, wt);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = c;
}

__global__ void __launch_bounds__(KC_THREADS) k_kept_scatter(const uint64_t *__restrict__ ekey, uint64_t m,
                                                             uint64_t seed_mix, uint64_t thr,
                                                             const uint32_t *__restrict__ tile_off,
                                                             uint64_t *__restrict__ out)
{
    __shared__ uint32_t wt[33];
    const uint64_t base = (uint64_t)blockIdx.x * RX_TILE;
    uint32_t carry = tile_off[blockIdx.x];
    for (int j = 0; j < KC_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * KC_THREADS + threadIdx.x;
        const uint64_t k = i < m ? ekey[i] : 0;
        const bool f = i < m && keep_edge(k, seed_mix, thr);
        uint32_t tot;
        const uint32_t ex = block_excl_scan((uint32_t)f, wt, &tot);
        if (f) out[carry + ex] = k;
        carry += tot;
    }
}

void compact_kept(const CountBuffers &b, uint64_t seed_mix, uint64_t thr, uint64_t *out, uint32_t *tile_cnt,
                  uint32_t *scan_scratch, cudaStream_t s)
{
    const uint64_t nt = ceil_div(b.m, RX_TILE);
    if (nt == 0) return;
    k_kept_count<<<(unsigned)nt, KC_THREADS, 0, s>>>(b.ekey, b.m, seed_mix, thr, tile_cnt); note_launch();
    scan_excl_u32(tile_cnt, nt, nullptr, scan_scratch, s);
    k_kept_scatter<<<(unsigned)nt, KC_THREADS, 0, s>>>(b.ekey, b.m, seed_mix, thr, tile_cnt, out); note_launch();
}

// ======================================================================
// Source buckets by out-degree d+ (sources with d+ < 2 close no triangle)
//   bucket 0: 2 <= d+ <= 32  -> one warp per source, list front
//   bucket 1: d+ > 32        -> one block per source, list back
// ======================================================================

constexpr uint32_t SMALL_MAX = 32;

__global__ void k_buckets(const uint32_t *__restrict__ rowptr, uint32_t n, uint32_t *__restrict__ list,
                          DevState *st)
{
    const unsigned lane = lane_id();
    const unsigned lt = lanemask_lt();
    const uint64_t wstride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += wstride) {
        const uint64_t u = base + lane;
        uint32_t d = 0;
        if (u < n) d = rowptr[u + 1] - rowptr[u];
        const bool b0 = d >= 2 && d <= SMALL_MAX, b1 = d > SMALL_MAX;
        const unsigned m0 = __ballot_sync(FULL, b0), m1 = __ballot_sync(FULL, b1);
        uint32_t o0 = 0, o1 = 0;
        if (lane == 0) {
            if (m0) o0 = atomicAdd(&st->nlist[0], (unsigned)__popc(m0));
            if (m1) o1 = atomicAdd(&st->nlist[1], (unsigned)__popc(m1));
        }
        o0 = __shfl_sync(FULL, o0, 0);
        o1 = __shfl_sync(FULL, o1, 0);
        if (b0) list[o0 + __popc(m0 & lt)] = (uint32_t)u;
        if (b1) list[n - 1 - (o1 + __popc(m1 & lt))] = (uint32_t)u;
    }
}

void build_buckets(const CountBuffers &b, cudaStream_t s)
{
    k_buckets<<<grid_for(b.n, 256, 152 * 8), 256, 0, s>>>(b.rowptr, b.n, b.list, b.st); note_launch();
}

// ======================================================================
// Intersections
// ======================================================================

// Largest i in [0, cnt) with pre[i] <= e, for non-decreasing pre with
// pre[0] = 0 <= e.
__device__ __forceinline__ uint32_t seg_of(const uint32_t *pre, uint32_t cnt, uint32_t e)
{
    uint32_t lo = 0, hi = cnt;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (pre[mid] <= e) lo = mid; else hi = mid;
    }
    return lo;
}

// Is w in the sorted list a[0, len)?
__device__ __forceinline__ bool contains(const uint32_t *a, uint32_t len, uint32_t w)
{
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (a[mid] < w) lo = mid + 1; else hi = mid;
    }
    return lo < len && a[lo] == w;
}

constexpr int IW_THREADS = 256;
constexpr int IW_WARPS = IW_THREADS / 32;

// One warp per source u with 2 <= d+(u) <= 32.  N+(u) is staged in shared
// memory; the concatenation of N+(v) over v in N+(u) is walked 32 elements
// at a time (one per lane, coalesced within each list) and every element w
// is binary-searched in N+(u).
__global__ void __launch_bounds__(IW_THREADS) k_isect_warp(const uint32_t *__restrict__ rowptr,
                                                           const uint32_t *__restrict__ col,
                                                           const uint32_t *__restrict__ list,
                                                           const uint8_t *__restrict__ heavy, DevState *st)
{
    __shared__ uint32_t s_nu[IW_WARPS][SMALL_MAX];
    __shared__ uint32_t s_vb[IW_WARPS][SMALL_MAX];
    __shared__ uint32_t s_pre[IW_WARPS][SMALL_MAX + 1];
    __shared__ unsigned long long s_red[4][IW_WARPS];
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const uint32_t nl = st->nlist[0];
    const uint32_t gw = blockIdx.x * IW_WARPS + w, nwarps = gridDim.x * IW_WARPS;
    unsigned long long cl = 0, ch = 0, ws = 0, wn = 0;
    for (uint32_t idx = gw; idx < nl; idx += nwarps) {
        const uint32_t u = list[idx];
        const uint32_t beg = rowptr[u], d = rowptr[u + 1] - beg;
        uint32_t x = 0, vb = 0, len = 0;
        if (lane < d) {
            x = col[beg + lane];
            vb = rowptr[x];
            len = rowptr[x + 1] - vb;
        }
        s_nu[w][lane] = x;
        s_vb[w][lane] = vb;
        const uint32_t inc = warp_incl_scan(len);
        s_pre[w][lane] = inc - len;
        const uint32_t W = __shfl_sync(FULL, inc, 31);
        __syncwarp();
        uint32_t c = 0;
        for (uint32_t e = lane; e < W; e += 32) {
            const uint32_t i = seg_of(s_pre[w], d, e);
            const uint32_t y = col[s_vb[w][i] + (e - s_pre[w][i])];
            c += contains(s_nu[w], d, y);
        }
        c = warp_sum(c);
        if (heavy[u]) ch += c; else cl += c;
        ws += d;
        wn += W;
        __syncwarp();
    }
    if (lane == 0) {
        s_red[0][w] = cl;
        s_red[1][w] = ch;
        s_red[2][w] = ws;
        s_red[3][w] = wn;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        unsigned long long t = 0;
        for (int i = 0; i < IW_WARPS; ++i) t += s_red[threadIdx.x][i];
        unsigned long long *dst[4] = {&st->t_light, &st->t_heavy, &st->src_elems, &st->nbr_elems};
        if (t) atomicAdd(dst[threadIdx.x], t);
    }
}

constexpr int IB_THREADS = 256;

// One block per source u with d+(u) > 32, taken from a global work cursor.
// N+(u) is staged in shared memory when it fits (cap elements), otherwise
// searched in place.  Chunks of IB_THREADS out-neighbours v are processed at
// a time: a block scan of d+(v) lays the chunk's lists end to end and the
// block walks that concatenation, one element per thread.
__global__ void __launch_bounds__(IB_THREADS) k_isect_block(const uint32_t *__restrict__ rowptr,
                                                            const uint32_t *__restrict__ col,
                                                            const uint32_t *__restrict__ list, uint32_t n,
                                                            const uint8_t *__restrict__ heavy, DevState *st,
                                                            uint32_t cap)
{
    extern __shared__ uint32_t s_nu[];
    __shared__ uint32_t s_pre[IB_THREADS];
    __shared__ uint32_t s_vb[IB_THREADS];
    __shared__ uint32_t wt[33];
    __shared__ unsigned long long wr[33];
    __shared__ uint32_t s_idx;
    const uint32_t nl = st->nlist[1];
    unsigned long long cl = 0, ch = 0, ws = 0, wn = 0;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(&st->cursor[1], 1u);
        __syncthreads();
        const uint32_t idx = s_idx;
        if (idx >= nl) break;
        const uint32_t u = list[n - 1 - idx];
        const uint32_t beg = rowptr[u], d = rowptr[u + 1] - beg;
        const uint32_t *nu = col + beg;
        if (d <= cap) {
            for (uint32_t i = threadIdx.x; i < d; i += IB_THREADS) s_nu[i] = col[beg + i];
            nu = s_nu;
        }
        __syncthreads();
        uint32_t c = 0;
        for (uint32_t c0 = 0; c0 < d; c0 += IB_THREADS) {
            const uint32_t t = c0 + threadIdx.x;
            uint32_t vb = 0, len = 0;
            if (t < d) {
                const uint32_t x = nu[t];
                vb = rowptr[x];
                len = rowptr[x + 1] - vb;
            }
            uint32_t W;
            const uint32_t ex = block_excl_scan(len, wt, &W);
            wn += W;
            s_pre[threadIdx.x] = ex;
            s_vb[threadIdx.x] = vb;
            __syncthreads();
            const uint32_t cnt = min((uint32_t)IB_THREADS, d - c0);
            for (uint32_t e = threadIdx.x; e < W; e += IB_THREADS) {
                const uint32_t i = seg_of(s_pre, cnt, e);
                const uint32_t y = col[s_vb[i] + (e - s_pre[i])];
                c += contains(nu, d, y);
            }
            __syncthreads();
        }
        if (heavy[u]) ch += c; else cl += c;
        ws += d;
        __syncthreads();  // s_idx and s_nu are rewritten by the next source
    }
    cl = block_sum(cl, wr);
    if (threadIdx.x == 0 && cl) atomicAdd(&st->t_light, cl);
    ch = block_sum(ch, wr);
    if (threadIdx.x == 0 && ch) atomicAdd(&st->t_heavy, ch);
    // ws and wn are block-uniform: thread 0 reports them
    if (threadIdx.x == 0 && ws) atomicAdd(&st->src_elems, ws);
    if (threadIdx.x == 0 && wn) atomicAdd(&st->nbr_elems, wn);
}

void intersect(const CountBuffers &b, int max_smem_bytes, cudaStream_t s)
{
    if (b.n == 0 || b.m == 0) return;
    k_isect_warp<<<152 * 8, IW_THREADS, 0, s>>>(b.rowptr, b.col, b.list, b.heavy, b.st); note_launch();
    if (max_smem_bytes > 48 * 1024)
        cudaFuncSetAttribute(k_isect_block, cudaFuncAttributeMaxDynamicSharedMemorySize, max_smem_bytes);
    const uint32_t cap = (uint32_t)(max_smem_bytes / 4);
    k_isect_block<<<152 * 4, IB_THREADS, (size_t)cap * 4, s>>>(b.rowptr, b.col, b.list, b.n, b.heavy, b.st,
                                                              cap); note_launch();
}

// ======================================================================
// Finaliser: the Section 3.1 rescale in float64, on the device
// ======================================================================

__global__ void k_finalize(const DevState *st, uint64_t m, uint32_t n, double p, tc_result *out)
{
    const double p3 = __dmul_rn(__dmul_rn(p, p), p);
    out->m = m;
    out->m_sampled = st->m_sampled;
    out->n = n;
    out->n_heavy = st->n_heavy;
    out->t_light = st->t_light;
    out->t_heavy = st->t_heavy;
    out->estimate = __dadd_rn(__ddiv_rn((double)st->t_light, p3), __ddiv_rn((double)st->t_heavy, p3));
    out->src_elems = st->src_elems;
    out->nbr_elems = st->nbr_elems;
    for (int i = 0; i < 8; ++i) out->ms[i] = 0.0f;
}

void finalize(const CountBuffers &b, double p, tc_result *out_dev, cudaStream_t s)
{
    k_finalize<<<1, 1, 0, s>>>(b.st, b.m, b.n, p, out_dev); note_launch();
}

}  // namespace tcg
