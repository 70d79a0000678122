// Counting kernels of libtc, part 1: the degree partition (Section 3.2) and
// the float64 rescale (Section 3.1).  Sampling and the CSR are in csr.cu, the
// intersections in isect.cu.
#include "kernels.h"

namespace tcg {

unsigned grid_for(uint64_t work, int threads, unsigned cap)
{
    uint64_t b = ceil_div(work, (uint64_t)threads);
    if (b > cap) b = cap;
    return (unsigned)(b ? b : 1);
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
        uint32_t lim = 0;
        for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
            const unsigned long long d = deg[u];
            const uint8_t f = d * d > mp;
            heavy[u] = f;
            h += f;
            if (!f && d) lim = (uint32_t)u + 1;
        }
        if (lim) atomicMax(&st->light_lim, lim);
    } else {
        // batch: each vertex against its own graph's m_p; every warp takes a
        // contiguous run of 32-vertex groups, so its graph only moves forward
        const unsigned lane = lane_id();
        const uint64_t groups = ((uint64_t)n + 31) / 32, nwarps = stride / 32;
        const uint64_t wid = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) / 32;
        const uint64_t g_lo = groups * wid / nwarps, g_hi = groups * (wid + 1) / nwarps;
        uint32_t gw = g_lo < g_hi ? find_part(bv.voff, bv.k, (uint32_t)(g_lo * 32)) : 0u, lim = 0;
        for (uint64_t grp = g_lo; grp < g_hi; ++grp) {
            const uint64_t u = grp * 32 + lane;
            const uint32_t uu = (uint32_t)(u < n ? u : n - 1);
            const uint32_t g = find_part_warp_from(bv.voff, bv.k, uu, gw);
            gw = __shfl_sync(FULL, g, 31);
            const unsigned long long d = deg[uu], mp = bv.m_p[g];
            const bool f = u < n && d * d > mp;
            if (u < n) heavy[u] = f;
            h += f;
            if (u < n && !f && d) lim = uu + 1;
            const unsigned peers = __match_any_sync(FULL, g);
            const unsigned c = __popc(__ballot_sync(FULL, f) & peers);
            if (c && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(bv.n_heavy + g, c);
        }
        lim = __reduce_max_sync(FULL, lim);
        if (lane == 0 && lim) atomicMax(&st->light_lim, lim);
    }
    h = warp_sum(h);
    if (lane_id() == 0 && h) atomicAdd(&st->n_heavy, h);
}

// Single graph with static rows: only rank ids at or above DevState::cand_lo
// can be heavy (k_sample_keep); their sampled degree is the kept out-degree
// (rowptr) plus the kept in-degree (spread, or the static one when every edge
// is kept).  The rest are light, and light_lim is at least cand_lo.  Each
// counter of spread then becomes its vertex's in-list cursor (the static
// reservation inres).
// With m_orig != 0 the flags come from the whole graph instead (the
// alternative reading of Section 3.2): heavy <=> (full degree)^2 > m_orig,
// the full degree being the static row length (frow) plus the static
// in-degree (inres).  Those vertices are a suffix of the rank order, so
// every light vertex counts toward light_lim.
__global__ void k_partition_cand(const uint32_t *__restrict__ dplus, uint32_t *__restrict__ spread, int hbits,
                                 const uint32_t *__restrict__ inres, bool all_kept, uint32_t n, uint32_t core_base,
                                 DevState *st, uint32_t *__restrict__ deg, uint8_t *__restrict__ heavy,
                                 const uint32_t *__restrict__ frow, unsigned long long m_orig)
{
    uint32_t below = 0;  // heavy vertices below the dense core's base
    const unsigned long long mp = st->m_sampled;
    const uint32_t cand = st->cand_all ? 0u : st->cand_lo;
    uint32_t h = 0, lim = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        uint32_t d = dplus[u];
        uint8_t f = 0;
        uint32_t *sp = spread + hot_index((uint32_t)u, hbits);
        if (u >= cand) d += all_kept ? inres[u + 1] - inres[u] : *sp;
        if (m_orig) {
            const unsigned long long full = (frow[u + 1] - frow[u]) + (inres[u + 1] - inres[u]);
            f = full * full > m_orig;
            if (!f) lim = (uint32_t)u + 1;
        } else if (u >= cand) {
            f = (unsigned long long)d * d > mp;
            if (!f && d) lim = (uint32_t)u + 1;
        }
        *sp = inres[u];  // u's in-list cursor from here on (the compaction appends at it)
        deg[u] = d;
        heavy[u] = f;
        h += f;
        below += f && u < core_base;
    }
    below = warp_sum(below);
    if (lane_id() == 0 && below) atomicAdd(&st->heavy_below, below);
    if (blockIdx.x == 0 && threadIdx.x == 0) lim = max(lim, min(cand, n));
    if (lim) atomicMax(&st->light_lim, lim);
    h = warp_sum(h);
    if (lane_id() == 0 && h) atomicAdd(&st->n_heavy, h);
}

void partition(const CountBuffers &b, cudaStream_t s)
{
    if (b.static_rows) {
        k_partition_cand<<<grid_for(b.n, 256, 152 * 8), 256, 0, s>>>(b.rowptr, b.spread,
                                                                     hot_bits(b.n), b.inptr,
                                                                     b.all_kept, b.n, b.core_base, b.st, b.deg,
                                                                     b.heavy, b.frow, b.frow ? b.m_orig : 0ull);
    } else {
        k_partition<<<grid_for(b.n, 256, 152 * 8), 256, 0, s>>>(b.deg, b.n, b.st, b.heavy, b.bv);
    }
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
    // with the core block on, the triangles inside the core that have a light
    // vertex are its count minus the all-heavy ones (every heavy vertex is in
    // the core, so all of T_H lies inside it)
    const unsigned long long t_light = st->t_light + (st->core_on ? st->t_core - st->t_heavy : 0ull);
    out->t_light = t_light;
    out->t_heavy = st->t_heavy;
    out->estimate = __dadd_rn(__ddiv_rn((double)t_light, p3), __ddiv_rn((double)st->t_heavy, p3));
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
