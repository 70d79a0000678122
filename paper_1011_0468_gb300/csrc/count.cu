// Counting kernels of libtc, part 1: edge sampling with degrees
// (Section 3.1), the degree partition (Section 3.2), the kept-edge export and
// the float64 rescale.  The intersections are in isect.cu.
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
                                                       uint32_t *__restrict__ deg, DevState *st, BatchView bv,
                                                       uint32_t *__restrict__ tile_cnt)
{
    __shared__ uint32_t wt[33];
    uint32_t kept = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t tid = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (tile_cnt) {
        // whole RX_TILE-key tiles per block, with the kept count of each
        const ulonglong2 *e2 = reinterpret_cast<const ulonglong2 *>(ekey);
        const uint64_t nt = (m + RX_TILE - 1) / RX_TILE;
        for (uint64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
            uint32_t c = 0;
            const uint64_t b2 = tile * (RX_TILE / 2);
#pragma unroll
            for (int j = 0; j < RX_TILE / 2 / 256; ++j) {
                const uint64_t i = b2 + (uint64_t)j * 256 + threadIdx.x;
                if (2 * i + 1 < m) {
                    const ulonglong2 k = ld_stream_u64x2(e2 + i);
                    c += sample_one(k.x, seed_mix, thr, deg);
                    c += sample_one(k.y, seed_mix, thr, deg);
                } else if (2 * i < m) {
                    c += sample_one(ekey[2 * i], seed_mix, thr, deg);
                }
            }
            kept += c;
            c = block_sum(c, wt);
            if (threadIdx.x == 0) tile_cnt[tile] = c;
        }
    } else if (bv.k == 0) {
        const ulonglong2 *e2 = reinterpret_cast<const ulonglong2 *>(ekey);
        for (uint64_t i = tid; i < m / 2; i += stride) {
            const ulonglong2 k = ld_stream_u64x2(e2 + i);
            kept += sample_one(k.x, seed_mix, thr, deg);
            kept += sample_one(k.y, seed_mix, thr, deg);
        }
        if ((m & 1) && tid == 0) kept += sample_one(ekey[m - 1], seed_mix, thr, deg);
    } else {
        // batch: each edge with its own graph's (p, seed); kept edges are
        // also counted per graph
        const unsigned lane = lane_id();
        for (uint64_t base = tid - lane; base < m; base += stride) {
            const uint64_t i = base + lane, ii = i < m ? i : m - 1;
            const uint64_t key = ld_stream_u64(ekey + ii);
            uint32_t g;
            g = find_part_warp(bv.eoff, bv.k, ii);
            const uint64_t vo = __ldg(bv.voff + g);
            const bool f = i < m && keep_edge(key - ((vo << 32) | vo), __ldg(bv.seed_mix + g), __ldg(bv.thr + g));
            if (f) {
                atomicAdd(deg + (key >> 32), 1u);
                atomicAdd(deg + (uint32_t)key, 1u);
                ++kept;
            }
            const unsigned peers = __match_any_sync(FULL, g);
            const unsigned c = __popc(__ballot_sync(FULL, f) & peers);
            if (c && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(bv.m_p + g, (unsigned long long)c);
        }
    }
    kept = warp_sum(kept);
    if (lane_id() == 0 && kept) atomicAdd(&st->m_sampled, (unsigned long long)kept);
}

unsigned grid_for(uint64_t work, int threads, unsigned cap)
{
    uint64_t b = ceil_div(work, (uint64_t)threads);
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
}

void sample_degree(const CountBuffers &b, uint64_t seed_mix, uint64_t thr, cudaStream_t s, uint32_t *tile_cnt)
{
    if (b.m == 0) return;
    k_sample_degree<<<grid_for(b.m / 2 + 1, 256, 152 * 8), 256, 0, s>>>(b.ekey, b.m, seed_mix, thr, b.deg,
                                                                        b.st, b.bv, b.bv.k ? nullptr : tile_cnt);
    note_launch();
}

// ======================================================================
// Degree partition: heavy <=> deg_p^2 > m_p (Section 3.2, in integers)
// ======================================================================

__global__ void k_partition(const uint32_t *__restrict__ deg, uint32_t n, DevState *st,
                            uint8_t *__restrict__ heavy, BatchView bv)
{
    uint32_t h = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    if (bv.k == 0) {
        const unsigned long long mp = st->m_sampled;
        for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
            const unsigned long long d = deg[u];
            const uint8_t f = d * d > mp;
            heavy[u] = f;
            h += f;
        }
    } else {
        // batch: each vertex against its own graph's m_p
        const unsigned lane = lane_id();
        for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
            const uint64_t u = base + lane;
            const uint32_t uu = (uint32_t)(u < n ? u : n - 1);
            const uint32_t g = find_part_warp(bv.voff, bv.k, uu);
            const unsigned long long d = deg[uu], mp = bv.m_p[g];
            const bool f = u < n && d * d > mp;
            if (u < n) heavy[u] = f;
            h += f;
            const unsigned peers = __match_any_sync(FULL, g);
            const unsigned c = __popc(__ballot_sync(FULL, f) & peers);
            if (c && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(bv.n_heavy + g, c);
        }
    }
    h = warp_sum(h);
    if (lane_id() == 0 && h) atomicAdd(&st->n_heavy, h);
}

void partition(const CountBuffers &b, cudaStream_t s)
{
    k_partition<<<grid_for(b.n, 256, 152 * 8), 256, 0, s>>>(b.deg, b.n, b.st, b.heavy, b.bv);
    note_launch();
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

void kept_scatter(const CountBuffers &b, uint64_t seed_mix, uint64_t thr, uint64_t *out, uint32_t *tile_cnt,
                  uint32_t *scan_scratch, cudaStream_t s)
{
    const uint64_t nt = ceil_div(b.m, RX_TILE);
    if (nt == 0) return;
    scan_excl_u32(tile_cnt, nt, nullptr, scan_scratch, s);
    k_kept_scatter<<<(unsigned)nt, KC_THREADS, 0, s>>>(b.ekey, b.m, seed_mix, thr, tile_cnt, out);
    note_launch();
}

void compact_kept(const CountBuffers &b, uint64_t seed_mix, uint64_t thr, uint64_t *out, uint32_t *tile_cnt,
                  uint32_t *scan_scratch, cudaStream_t s)
{
    const uint64_t nt = ceil_div(b.m, RX_TILE);
    if (nt == 0) return;
    k_kept_count<<<(unsigned)nt, KC_THREADS, 0, s>>>(b.ekey, b.m, seed_mix, thr, tile_cnt);
    note_launch();
    scan_excl_u32(tile_cnt, nt, nullptr, scan_scratch, s);
    k_kept_scatter<<<(unsigned)nt, KC_THREADS, 0, s>>>(b.ekey, b.m, seed_mix, thr, tile_cnt, out);
    note_launch();
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
    out->partners = st->partners;
    out->heavy_mma_flops = st->heavy_kchunks * 2ull * 128ull * 128ull * 64ull;
    for (int i = 0; i < 8; ++i) out->ms[i] = 0.0f;
}

void finalize(const CountBuffers &b, double p, tc_result *out_dev, cudaStream_t s)
{
    k_finalize<<<1, 1, 0, s>>>(b.st, b.m, b.n, p, out_dev);
    note_launch();
}

// One result per graph of a batch (same float64 rescale per graph).
__global__ void k_finalize_batch(BatchView bv, const double *__restrict__ p, tc_result *__restrict__ out)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g >= bv.k) return;
    const double pg = p[g];
    const double p3 = __dmul_rn(__dmul_rn(pg, pg), pg);
    tc_result r;
    r.m = bv.eoff[g + 1] - bv.eoff[g];
    r.m_sampled = bv.m_p[g];
    r.n = bv.voff[g + 1] - bv.voff[g];
    r.n_heavy = bv.n_heavy[g];
    r.t_light = bv.t_light[g];
    r.t_heavy = bv.t_heavy[g];
    r.estimate = __dadd_rn(__ddiv_rn((double)r.t_light, p3), __ddiv_rn((double)r.t_heavy, p3));
    r.src_elems = r.nbr_elems = r.partners = r.heavy_mma_flops = 0;
    for (int i = 0; i < 8; ++i) r.ms[i] = 0.0f;
    out[g] = r;
}

void finalize_batch(const CountBuffers &b, const double *p_dev, tc_result *out_dev, cudaStream_t s)
{
    k_finalize_batch<<<grid_for(b.bv.k, 128, 1u << 20), 128, 0, s>>>(b.bv, p_dev, out_dev);
    note_launch();
}

}  // namespace tcg
