// Triple sampling (Section 3.2) after edge sparsification (Section 3.1): the
// "simple" and "hybrid" estimators of the paper's experiments.
//
// U is a set of vertex triples holding every triangle, built vertex by
// vertex in id order over the sampled graph's symmetric adjacency (each
// neighbour list sorted by id):
//   - a light vertex (every vertex in the simple mode) contributes its
//     wedges, the C(d, 2) pairs {N(u)[a], N(u)[b]}, a < b, numbered
//     b (b - 1) / 2 + a;
//   - in the hybrid mode a heavy vertex (deg_p^2 > m_p, the partition of
//     Section 3.2 on the sample) contributes its 2-paths u - v - w, v in
//     N(u), w in N(v): sum over v in N(u) of deg(v) of them, numbered by v's
//     position and then w's.
// A wedge v-u-w closes iff vw is an edge, a 2-path iff w != u and uw is an
// edge; each triangle is in U once per light corner and twice per heavy
// corner.  Sample i is triple floor(h_i |U| / 2^64), h_i = splitmix64(i ^
// splitmix64(~seed)), and the estimate is |U| (2 c_w + c_p) / (6 s) / p^3
// (c_w, c_p: closed wedges and 2-paths among the s samples).
//
// Layout: the whole graph's symmetric adjacency in original ids (soff /
// snbr, built on the first call and kept); per count, the kept part of it
// (p < 1: compacted by the keep rule of Section 3.1, order preserved), the
// per-vertex triple counts and their 64-bit prefix, and for heavy rows the
// 2-path prefix of every list position.  The sampling kernel then maps each
// draw to its triple with binary searches and checks closure by a binary
// search of the shorter of the two sorted lists.
#include <algorithm>

#include "kernels.h"

namespace tcg {

constexpr int TR_THREADS = 256;

// ---------------------------------------------------------------- build

// Both directions of every canonical key: (u, v) and (v, u).
__global__ void k_sym_keys(const uint64_t *__restrict__ orig, uint64_t m, uint64_t *__restrict__ keys)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const uint64_t k = orig[i];
        keys[2 * i] = k;
        keys[2 * i + 1] = (k << 32) | (k >> 32);
    }
}

// soff[x] = first sorted key with source >= x (x <= n); snbr = targets.
__global__ void k_sym_rows(const uint64_t *__restrict__ keys, uint64_t len, uint32_t n, uint32_t *__restrict__ soff,
                           uint32_t *__restrict__ snbr)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    const uint64_t t0 = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t x = t0; x <= n; x += stride) {
        const uint64_t target = x << 32;
        uint64_t lo = 0, hi = len;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (keys[mid] < target) lo = mid + 1; else hi = mid;
        }
        soff[x] = (uint32_t)lo;
    }
    for (uint64_t i = t0; i < len; i += stride) snbr[i] = (uint32_t)keys[i];
}

// ---------------------------------------------------------------- sample

// Kept neighbours of row u (one warp per row): the count, or with out != 0
// the kept neighbours themselves at out[off[u] ..], in list order.
template <bool WRITE>
__global__ void k_keep_rows(const uint32_t *__restrict__ soff, const uint32_t *__restrict__ snbr, uint32_t n,
                            uint64_t seed_mix, uint64_t thr, uint32_t *__restrict__ cnt_or_off,
                            uint32_t *__restrict__ out)
{
    const unsigned lane = lane_id();
    const uint64_t warps = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    for (uint64_t u = ((uint64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += warps) {
        const uint32_t b = soff[u], e = soff[u + 1];
        uint32_t pos = WRITE ? cnt_or_off[u] : 0u;
        for (uint32_t j0 = b; j0 < e; j0 += 32) {
            const uint32_t j = j0 + lane;
            bool keep = false;
            uint32_t w = 0;
            if (j < e) {
                w = snbr[j];
                const uint32_t a = min((uint32_t)u, w), c = max((uint32_t)u, w);
                keep = keep_edge(((uint64_t)a << 32) | c, seed_mix, thr);
            }
            const unsigned bal = __ballot_sync(FULL, keep);
            if (WRITE && keep) out[pos + __popc(bal & lanemask_lt())] = w;
            pos += __popc(bal);
        }
        if (!WRITE && lane == 0) cnt_or_off[u] = pos;
    }
}

// Class of every vertex and its share of U: wedges C(d, 2), or for a heavy
// vertex (hybrid) a place in the list of rows whose 2-paths are counted next.
__global__ void k_triple_classes(const uint32_t *__restrict__ off, uint32_t n, bool hybrid,
                                 unsigned long long *__restrict__ cnt, uint32_t *__restrict__ hlist, uint32_t hcap,
                                 TripleDev *td, uint64_t samples)
{
    const unsigned long long mp = off[n] / 2;
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        td->m_p = mp;
        td->samples = samples ? samples : mp;
        cnt[n] = 0;
    }
    uint32_t h = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const unsigned long long d = off[u + 1] - off[u];
        if (hybrid && d * d > mp) {
            const uint32_t slot = atomicAdd(&td->nlist, 1u);
            if (slot < hcap) hlist[slot] = (uint32_t)u; else atomicOr(&td->err, ERR_OVERFLOW);
            cnt[u] = 0;  // k_path_rows
            ++h;
        } else {
            cnt[u] = d * (d - (d > 0 ? 1ull : 0ull)) / 2;
        }
    }
    h = warp_sum(h);
    if (lane_id() == 0 && h) atomicAdd(&td->n_heavy, h);
}

// One block per heavy row u: qpre[j] = 2-paths through the neighbours
// before position j (sum of their degrees), cnt[u] = all of u's 2-paths.
__global__ void __launch_bounds__(TR_THREADS) k_path_rows(const uint32_t *__restrict__ off,
                                                          const uint32_t *__restrict__ nbr,
                                                          const uint32_t *__restrict__ hlist, uint32_t hcap,
                                                          const TripleDev *td, uint32_t *__restrict__ qpre,
                                                          unsigned long long *__restrict__ cnt)
{
    __shared__ unsigned long long wt[33];
    const uint32_t nl = min(td->nlist, hcap);
    for (uint32_t k = blockIdx.x; k < nl; k += gridDim.x) {
        const uint32_t u = hlist[k], b = off[u], e = off[u + 1];
        unsigned long long carry = 0;
        for (uint32_t j0 = b; j0 < e; j0 += TR_THREADS) {
            const uint32_t j = j0 + threadIdx.x;
            unsigned long long x = 0;
            if (j < e) {
                const uint32_t v = nbr[j];
                x = off[v + 1] - off[v];
            }
            unsigned long long tot;
            const unsigned long long ex = block_excl_scan(x, wt, &tot);
            if (j < e) qpre[j] = (uint32_t)(carry + ex);
            carry += tot;
        }
        if (threadIdx.x == 0) cnt[u] = carry;
    }
}

__device__ __forceinline__ bool sorted_has(const uint32_t *__restrict__ a, uint32_t len, uint32_t w)
{
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < w) lo = mid + 1; else hi = mid;
    }
    return lo < len && __ldg(a + lo) == w;
}

// Is {x, y} an edge?  Binary search of the shorter sorted list.
__device__ __forceinline__ bool has_edge(const uint32_t *__restrict__ off, const uint32_t *__restrict__ nbr, uint32_t x,
                                         uint32_t y)
{
    const uint32_t bx = __ldg(off + x), dx = __ldg(off + x + 1) - bx;
    const uint32_t by = __ldg(off + y), dy = __ldg(off + y + 1) - by;
    return dx <= dy ? sorted_has(nbr + bx, dx, y) : sorted_has(nbr + by, dy, x);
}

// The s draws: each maps its hash to a triple of U and checks closure.
__global__ void k_triple_samples(const uint32_t *__restrict__ off, const uint32_t *__restrict__ nbr,
                                 const unsigned long long *__restrict__ pre, const uint32_t *__restrict__ qpre,
                                 uint32_t n, bool hybrid, uint64_t tmix, TripleDev *td)
{
    const unsigned long long U = pre[n], s = td->samples, mp = td->m_p;
    unsigned long long cw = 0, cp = 0;
    if (U > 0) {
        const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
        for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += stride) {
            const unsigned long long r = __umul64hi(splitmix64(i ^ tmix), U);
            uint32_t lo = 0, hi = n;  // the vertex u with pre[u] <= r < pre[u + 1]
            while (hi - lo > 1) {
                const uint32_t mid = lo + ((hi - lo) >> 1);
                if (__ldg(pre + mid) <= r) lo = mid; else hi = mid;
            }
            const uint32_t u = lo, bu = __ldg(off + u), du = __ldg(off + u + 1) - bu;
            const unsigned long long k = r - __ldg(pre + u);
            if (!(hybrid && (unsigned long long)du * du > mp)) {
                // wedge k: the largest b >= 1 with b (b - 1) / 2 <= k, then a
                unsigned long long b = (unsigned long long)((1.0 + __dsqrt_rn(1.0 + 8.0 * (double)k)) * 0.5);
                if (b < 1) b = 1;
                while (b > 1 && b * (b - 1) / 2 > k) --b;
                while ((b + 1) * b / 2 <= k) ++b;
                const unsigned long long a = k - b * (b - 1) / 2;
                const uint32_t v = __ldg(nbr + bu + a), w = __ldg(nbr + bu + b);
                cw += has_edge(off, nbr, v, w);
            } else {
                // 2-path k: the last position j of u's row with qpre <= k
                uint32_t j = 0, jhi = du;
                while (jhi - j > 1) {
                    const uint32_t mid = j + ((jhi - j) >> 1);
                    if (__ldg(qpre + bu + mid) <= k) j = mid; else jhi = mid;
                }
                const uint32_t v = __ldg(nbr + bu + j);
                const uint32_t w = __ldg(nbr + __ldg(off + v) + (uint32_t)(k - __ldg(qpre + bu + j)));
                cp += w != u && has_edge(off, nbr, u, w);
            }
        }
    }
    cw = warp_sum(cw);
    cp = warp_sum(cp);
    if (lane_id() == 0) {
        if (cw) atomicAdd(&td->closed_wedge, cw);
        if (cp) atomicAdd(&td->closed_path, cp);
    }
}

__global__ void k_triple_finalize(const TripleDev *td, const unsigned long long *__restrict__ pre, uint32_t n,
                                  uint64_t m, double p, uint32_t mode, tc_triple_result *out)
{
    const unsigned long long U = pre[n], s = td->samples;
    tc_triple_result r;
    r.m = m;
    r.m_sampled = td->m_p;
    r.n = n;
    r.n_heavy = td->n_heavy;
    r.universe = U;
    r.samples = s;
    r.closed_wedge = td->closed_wedge;
    r.closed_path = td->closed_path;
    r.mode = mode;
    r.ms = 0.0f;
    r.estimate = 0.0;
    if (U && s) {
        const double raw = __ddiv_rn(__dmul_rn((double)U, (double)(2ull * r.closed_wedge + r.closed_path)),
                                     __dmul_rn(6.0, (double)s));
        r.estimate = __ddiv_rn(raw, __dmul_rn(__dmul_rn(p, p), p));
    }
    *out = r;
}

// ---------------------------------------------------------------- host

void triples_build(const uint64_t *orig, uint64_t m, uint32_t n, int nbits, TripleBuffers &tb, uint64_t *tmpA,
                   uint64_t *tmpB, uint32_t *hist, uint32_t *scan, cudaStream_t s)
{
    const uint64_t len = 2 * m;
    if (len == 0) {
        cudaMemsetAsync(tb.soff, 0, ((uint64_t)n + 1) * 4, s);
        return;
    }
    k_sym_keys<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(orig, m, tmpA);
    note_launch();
    uint64_t *a = tmpA, *b = tmpB;
    for (int half = 0; half < 2; ++half) {
        int shift = half ? 32 : 0;
        const int P = (nbits + RX_MAX_BITS - 1) / RX_MAX_BITS;
        for (int i = 0; i < P; ++i) {
            const int w = nbits / P + (i < nbits % P ? 1 : 0);
            radix_pass(a, len, shift, w, hist, scan, b, s);
            std::swap(a, b);
            shift += w;
        }
    }
    k_sym_rows<<<grid_for(std::max<uint64_t>(len, (uint64_t)n + 1), 256, 152 * 16), 256, 0, s>>>(a, len, n, tb.soff,
                                                                                                 tb.snbr);
    note_launch();
}

void triples_count(const TripleBuffers &tb, uint64_t seed_mix, uint64_t thr, uint64_t seed, uint64_t samples,
                   bool hybrid, double p, tc_triple_result *out_dev, cudaStream_t s)
{
    const uint32_t n = tb.n;
    TripleDev *td = tb.dev;
    cudaMemsetAsync(td, 0, sizeof(TripleDev), s);
    const uint32_t *off = tb.soff, *nbr = tb.snbr;
    const unsigned rows_grid = grid_for((uint64_t)n * 32, TR_THREADS, 152 * 16);
    if (thr < (1ull << 53) && tb.m > 0) {  // the sample of Section 3.1, rows kept in order
        k_keep_rows<false><<<rows_grid, TR_THREADS, 0, s>>>(tb.soff, tb.snbr, n, seed_mix, thr, tb.off_p, nullptr);
        note_launch();
        cudaMemsetAsync(tb.off_p + n, 0, 4, s);
        scan_excl_u32(tb.off_p, (uint64_t)n + 1, nullptr, tb.scan32, s);
        k_keep_rows<true><<<rows_grid, TR_THREADS, 0, s>>>(tb.soff, tb.snbr, n, seed_mix, thr, tb.off_p, tb.nbr_p);
        note_launch();
        off = tb.off_p;
        nbr = tb.nbr_p;
    }
    k_triple_classes<<<grid_for(n, TR_THREADS, 152 * 8), TR_THREADS, 0, s>>>(off, n, hybrid, tb.cnt, tb.hlist, tb.hcap,
                                                                           td, samples);
    note_launch();
    if (hybrid && tb.hcap) {
        k_path_rows<<<std::min<uint32_t>(tb.hcap, 152 * 8), TR_THREADS, 0, s>>>(off, nbr, tb.hlist, tb.hcap, td,
                                                                               tb.qpre, tb.cnt);
        note_launch();
    }
    scan_excl_u64(tb.cnt, (uint64_t)n + 1, nullptr, tb.scan64, s);
    k_triple_samples<<<152 * 8, TR_THREADS, 0, s>>>(off, nbr, tb.cnt, tb.qpre, n, hybrid, splitmix64(~seed), td);
    note_launch();
    k_triple_finalize<<<1, 1, 0, s>>>(td, tb.cnt, n, tb.m, p, hybrid ? 1u : 0u, out_dev);
    note_launch();
}

}  // namespace tcg
