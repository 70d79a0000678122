// The degree-oriented CSR of the sampled graph, built by one compaction.
//
// Orientation.  Every edge is directed from its endpoint of lower rank,
// rank = (degree in the whole graph, id): a total order, so each triangle
// {a, b, c} with rank(a) < rank(b) < rank(c) is seen exactly once, from the
// pair (a -> b), as the common out-neighbour c of a and b (the counts of
// Section 3.2 do not depend on the order; ranking by degree keeps every
// out-degree below (2 m)^(1/2)).  The rank is fixed when the graph is
// created, and the graph is stored relabeled in rank order: vertex ids are
// ranks and the canonical key list (u < v, sorted) is sorted by rank.  The
// kept keys of a sample, in that order, therefore already are the oriented
// rows, each sorted by rank, and the CSR of a count is a stream compaction.
// The sampling hash still reads each edge's original key, so a sample is
// the one Section 3.1 draws on the original graph.
#include "kernels.h"

namespace tcg {

// ======================================================================
// Relabeling (graph creation)
// ======================================================================

__global__ void k_full_degree(const uint64_t *__restrict__ ekey, uint64_t m, uint32_t *__restrict__ deg)
{
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < m; base += stride) {
        const uint64_t i = base + lane;
        const uint64_t k = i < m ? ekey[i] : ~0ull;
        const uint32_t u = (uint32_t)(k >> 32);
        const unsigned peers = __match_any_sync(FULL, u);  // keys are sorted: runs of a lower endpoint
        if (i < m) {
            if (lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(deg + u, (unsigned)__popc(peers));
            atomicAdd(deg + (uint32_t)k, 1u);
        }
    }
}

// Rank sort items of the vertices: single graph (rank key << 32 | id) with
// the full degree as key; batch union (graph << 48 | min(degree, 65535) << 32
// | id), so that every graph keeps its contiguous id range.
__global__ void k_vertex_items(const uint32_t *__restrict__ deg, uint32_t n, const uint32_t *__restrict__ voff,
                               uint32_t k, uint64_t *__restrict__ items)
{
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += stride) {
        const uint64_t v = base + lane;
        const uint32_t vv = (uint32_t)(v < n ? v : n - 1);
        uint64_t key;
        if (k == 0) {
            key = (uint64_t)deg[vv];
        } else {
            const uint32_t g = find_part_warp(voff, k, vv);
            key = ((uint64_t)g << 16) | (uint64_t)min(deg[vv], 0xffffu);
        }
        if (v < n) items[v] = (key << 32) | vv;
    }
}

__global__ void k_rank_of(const uint64_t *__restrict__ sorted, uint32_t n, uint32_t *__restrict__ perm,
                          uint32_t *__restrict__ rank)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t r = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; r < n; r += stride) {
        const uint32_t v = (uint32_t)sorted[r];
        perm[r] = v;
        rank[v] = (uint32_t)r;
    }
}

__global__ void k_original_keys(const uint64_t *__restrict__ rel, uint64_t m, const uint32_t *__restrict__ perm,
                                uint64_t *__restrict__ orig)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const uint64_t k = rel[i];
        const uint32_t a = __ldg(perm + (k >> 32)), b = __ldg(perm + (uint32_t)k);
        orig[i] = ((uint64_t)min(a, b) << 32) | max(a, b);
    }
}

// Stable LSD radix sort of items on bits [lo, hi), ping-ponging between a
// and b; returns the buffer holding the result.
static uint64_t *sort_bits(uint64_t *a, uint64_t *b, uint64_t count, int lo, int hi, uint32_t *hist,
                           uint32_t *scan, cudaStream_t s)
{
    const int bits = hi - lo;
    if (bits <= 0 || count == 0) return a;
    const int P = (bits + RX_MAX_BITS - 1) / RX_MAX_BITS;
    int shift = lo;
    for (int i = 0; i < P; ++i) {
        const int w = bits / P + (i < bits % P ? 1 : 0);
        radix_pass(a, count, shift, w, hist, scan, b, s);
        std::swap(a, b);
        shift += w;
    }
    return a;
}

static int bits_of(uint64_t x)
{
    int b = 1;
    while (b < 64 && (1ull << b) < x) ++b;
    return b;
}

// ---- keys in rank order without a key sort: every canonical edge goes to
// the row of its lower rank (rows counted and placed with atomics), then
// each row is sorted by its higher rank: a bitonic network in registers for
// rows of up to 16 entries, a warp in shared memory up to 1024, a block for
// the rest.

__device__ __forceinline__ void rank_pair(uint64_t key, const uint32_t *__restrict__ rank, uint32_t &u, uint32_t &v)
{
    const uint32_t a = __ldg(rank + (key >> 32)), b = __ldg(rank + (uint32_t)key);
    u = min(a, b);
    v = max(a, b);
}

// Keys come grouped by their original source, whose rank is the lower one
// for most of its edges: one atomic per run of a row in a warp.
__global__ void k_row_count(const uint64_t *__restrict__ ekey, uint64_t m, const uint32_t *__restrict__ rank,
                            uint32_t *__restrict__ cnt)
{
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < m; base += stride) {
        const uint64_t i = base + lane;
        uint32_t u = 0xffffffffu, v;
        if (i < m) rank_pair(ekey[i], rank, u, v);
        const unsigned grp = __match_any_sync(FULL, u);
        if (i < m && lane == (unsigned)(__ffs(grp) - 1)) atomicAdd(cnt + u, (unsigned)__popc(grp));
    }
}

// cur[u] starts at the row's first slot.
__global__ void k_row_place(const uint64_t *__restrict__ ekey, uint64_t m, const uint32_t *__restrict__ rank,
                            uint32_t *__restrict__ cur, uint64_t *__restrict__ rows)
{
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < m; base += stride) {
        const uint64_t i = base + lane;
        uint32_t u = 0xffffffffu, v = 0;
        if (i < m) rank_pair(ekey[i], rank, u, v);
        const unsigned grp = __match_any_sync(FULL, u);
        const int lead = __ffs(grp) - 1;
        uint32_t q = 0;
        if (i < m && (int)lane == lead) q = atomicAdd(cur + u, (unsigned)__popc(grp));
        q = __shfl_sync(FULL, q, lead) + __popc(grp & lanemask_lt());
        if (i < m) rows[q] = ((uint64_t)u << 32) | v;
    }
}

constexpr uint32_t ROW_SMALL = 16, ROW_SMEM = 32768;  // ROW_MID: kernels.h

// Ascending bitonic network over N (a power of two) register values.
template <int N>
__device__ __forceinline__ void bitonic_regs(uint32_t (&a)[N])
{
#pragma unroll
    for (int k = 2; k <= N; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1)
#pragma unroll
            for (int i = 0; i < N; ++i) {
                const int l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint32_t x = a[i], y = a[l];
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
}

template <int N>
__device__ __forceinline__ void sort_row_regs(const uint64_t *__restrict__ rows, uint32_t b, uint32_t len, uint32_t u,
                                              uint64_t *__restrict__ rel)
{
    uint32_t a[N];
#pragma unroll
    for (int i = 0; i < N; ++i) a[i] = (uint32_t)i < len ? (uint32_t)rows[b + i] : 0xffffffffu;
    bitonic_regs<N>(a);
#pragma unroll
    for (int i = 0; i < N; ++i)
        if ((uint32_t)i < len) rel[b + i] = ((uint64_t)u << 32) | a[i];
}

// Rows of up to ROW_SMALL entries, one thread each; longer rows are listed
// (mid rows from the front of list, the rest from its back; cnt[0], cnt[1]).
__global__ void k_rows_small(const uint64_t *__restrict__ rows, const uint32_t *__restrict__ frow, uint32_t n,
                             uint64_t *__restrict__ rel, uint32_t *__restrict__ list, uint32_t cap,
                             uint32_t *__restrict__ cnt)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride) {
        const uint32_t b = frow[x], len = frow[x + 1] - b, u = (uint32_t)x;
        if (len == 0) continue;
        if (len == 1)
            rel[b] = rows[b];
        else if (len <= 8)
            sort_row_regs<8>(rows, b, len, u, rel);
        else if (len <= ROW_SMALL)
            sort_row_regs<16>(rows, b, len, u, rel);
        else if (len <= ROW_MID)
            list[atomicAdd(cnt, 1u)] = u;
        else
            list[cap - 1 - atomicAdd(cnt + 1, 1u)] = u;
    }
}

// Ascending bitonic sort of a[0, P) (P a power of two) by `threads`
// cooperating threads with index t; sync() between steps.
template <class Sync>
__device__ __forceinline__ void bitonic_shared(uint32_t *a, uint32_t P, uint32_t t, uint32_t threads, Sync sync)
{
    for (uint32_t k = 2; k <= P; k <<= 1)
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            for (uint32_t i = t; i < P; i += threads) {
                const uint32_t l = i ^ j;
                if (l > i) {
                    const bool up = (i & k) == 0;
                    const uint32_t x = a[i], y = a[l];
                    if ((x > y) == up) {
                        a[i] = y;
                        a[l] = x;
                    }
                }
            }
            sync();
        }
}

struct BlockSync {
    __device__ void operator()() const { __syncthreads(); }
};

__device__ __forceinline__ uint32_t pow2_at_least(uint32_t x)
{
    uint32_t p = 1;
    while (p < x) p <<= 1;
    return p;
}

// Ascending bitonic sort of P = 32 V values held by a warp: value t of lane
// l sits at position l + 32 t.  Partners less than 32 apart are exchanged by
// shuffles, the others inside a lane's registers.
template <int V>
__device__ __forceinline__ void bitonic_warp(uint32_t (&a)[V])
{
    const unsigned lane = lane_id();
#pragma unroll
    for (int k = 2; k <= 32 * V; k <<= 1)
#pragma unroll
        for (int j = k >> 1; j > 0; j >>= 1) {
            if (j >= 32) {
                const int jt = j / 32;
#pragma unroll
                for (int t = 0; t < V; ++t) {
                    if ((t & jt) == 0) {
                        const bool up = (((uint32_t)lane + 32u * t) & (uint32_t)k) == 0;
                        const uint32_t x = a[t], y = a[t | jt];
                        if ((x > y) == up) {
                            a[t] = y;
                            a[t | jt] = x;
                        }
                    }
                }
            } else {
                const bool lower = (lane & (unsigned)j) == 0;
#pragma unroll
                for (int t = 0; t < V; ++t) {
                    const bool up = (((uint32_t)lane + 32u * t) & (uint32_t)k) == 0;
                    const uint32_t o = __shfl_xor_sync(FULL, a[t], j);
                    a[t] = (lower == up) ? min(a[t], o) : max(a[t], o);
                }
            }
        }
}

template <int V>
__device__ __forceinline__ void sort_row_warp(const uint64_t *__restrict__ rows, uint32_t b, uint32_t len, uint32_t u,
                                              uint64_t *__restrict__ rel)
{
    const unsigned lane = lane_id();
    uint32_t a[V];
#pragma unroll
    for (int t = 0; t < V; ++t) {
        const uint32_t i = lane + 32u * t;
        a[t] = i < len ? (uint32_t)rows[b + i] : 0xffffffffu;
    }
    bitonic_warp<V>(a);
#pragma unroll
    for (int t = 0; t < V; ++t) {
        const uint32_t i = lane + 32u * t;
        if (i < len) rel[b + i] = ((uint64_t)u << 32) | a[t];
    }
}

// Listed rows of up to ROW_MID entries: one warp each, in registers.
__global__ void __launch_bounds__(256) k_rows_mid(const uint64_t *__restrict__ rows, const uint32_t *__restrict__ frow,
                                                  const uint32_t *__restrict__ list, const uint32_t *__restrict__ cnt,
                                                  uint64_t *__restrict__ rel)
{
    static_assert(ROW_MID == 32 * 32, "at most 32 values per lane");
    const uint32_t rows_n = cnt[0];
    for (uint32_t r = blockIdx.x * 8 + (threadIdx.x >> 5); r < rows_n; r += gridDim.x * 8) {
        const uint32_t u = list[r], b = frow[u], len = frow[u + 1] - b;
        if (len <= 32)
            sort_row_warp<1>(rows, b, len, u, rel);
        else if (len <= 64)
            sort_row_warp<2>(rows, b, len, u, rel);
        else if (len <= 128)
            sort_row_warp<4>(rows, b, len, u, rel);
        else if (len <= 256)
            sort_row_warp<8>(rows, b, len, u, rel);
        else if (len <= 512)
            sort_row_warp<16>(rows, b, len, u, rel);
        else
            sort_row_warp<32>(rows, b, len, u, rel);
    }
}

// Listed rows longer than ROW_MID: one block each, in dynamic shared memory
// up to ROW_SMEM entries, else in global memory (the row's 8 * len bytes of
// gscratch hold its padded 32-bit values: the padded length is below 2 len).
__global__ void __launch_bounds__(1024) k_rows_large(const uint64_t *__restrict__ rows,
                                                     const uint32_t *__restrict__ frow,
                                                     const uint32_t *__restrict__ list, uint32_t cap,
                                                     const uint32_t *__restrict__ cnt, uint64_t *__restrict__ rel,
                                                     uint32_t *__restrict__ gscratch)
{
    extern __shared__ uint32_t s_big[];
    const uint32_t rows_n = cnt[1];
    for (uint32_t r = blockIdx.x; r < rows_n; r += gridDim.x) {
        const uint32_t u = list[cap - 1 - r], b = frow[u], len = frow[u + 1] - b, P = pow2_at_least(len);
        uint32_t *a = P <= ROW_SMEM ? s_big : gscratch + 2 * (uint64_t)b;
        for (uint32_t i = threadIdx.x; i < P; i += blockDim.x) a[i] = i < len ? (uint32_t)rows[b + i] : 0xffffffffu;
        __syncthreads();
        bitonic_shared(a, P, threadIdx.x, blockDim.x, BlockSync());  // orders global writes of the block too
        for (uint32_t i = threadIdx.x; i < len; i += blockDim.x) rel[b + i] = ((uint64_t)u << 32) | a[i];
        __syncthreads();
    }
}

uint64_t *relabel(const uint64_t *ekey, uint64_t m, uint32_t n, const uint32_t *voff, uint32_t k,
                  const Relabeled &out, const RelabelScratch &sc, cudaStream_t s, bool deg_ready)
{
    if (!deg_ready) {
        cudaMemsetAsync(sc.deg, 0, (size_t)n * 4, s);
        if (m > 0) {
            k_full_degree<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(ekey, m, sc.deg);
            note_launch();
        }
    }
    k_vertex_items<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(sc.deg, n, voff, k, sc.vA);
    note_launch();
    // stable sort by the rank key: degree bits only (ids are already in order)
    const int key_bits = k == 0 ? bits_of((uint64_t)std::max<uint64_t>(2 * m, 1) + 1) : 16 + bits_of(k + 1);
    const uint64_t *sorted = sort_bits(sc.vA, sc.vB, n, 32, 32 + std::min(key_bits, 32), sc.hist, sc.scan, s);
    k_rank_of<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(sorted, n, out.perm, out.rank);
    note_launch();
    if (m == 0) return out.rel;
    // rows in rank order: offsets (vB), cursors (vA), unsorted rows in
    // out.orig (ekey may be out.rel), sorted into out.rel; the lists of long
    // rows go to hist (m / 17 + 1 <= its length), their counts to scan
    uint32_t *frow = reinterpret_cast<uint32_t *>(sc.vB), *cur = reinterpret_cast<uint32_t *>(sc.vA);
    cudaMemsetAsync(frow, 0, ((size_t)n + 1) * 4, s);
    k_row_count<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(ekey, m, out.rank, frow);
    note_launch();
    scan_excl_u32(frow, (uint64_t)n + 1, nullptr, sc.scan, s);
    cudaMemcpyAsync(cur, frow, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    k_row_place<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(ekey, m, out.rank, cur, out.orig);
    note_launch();
    const uint32_t cap = (uint32_t)(m / (ROW_SMALL + 1) + 1);
    cudaMemsetAsync(sc.scan, 0, 8, s);
    k_rows_small<<<grid_for(n, 256, 152 * 16), 256, 0, s>>>(out.orig, frow, n, out.rel, sc.hist, cap, sc.scan);
    note_launch();
    k_rows_mid<<<152 * 8, 256, 0, s>>>(out.orig, frow, sc.hist, sc.scan, out.rel);
    note_launch();
    static bool large_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || !large_set[dev]) {
        if (cudaFuncSetAttribute(k_rows_large, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(ROW_SMEM * 4)) ==
                cudaSuccess &&
            dev >= 0 && dev < 64)
            large_set[dev] = true;
    }
    k_rows_large<<<152, 1024, ROW_SMEM * 4, s>>>(out.orig, frow, sc.hist, cap, sc.scan, out.rel,
                                                  reinterpret_cast<uint32_t *>(sc.kB));
    note_launch();
    k_original_keys<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(out.rel, m, out.perm, out.orig);
    note_launch();
    return out.rel;
}

// ======================================================================
// Sampling, sampled degrees and row counts (one read of the edge list)
// ======================================================================

// Per RX_TILE-edge tile: the Section 3.1 keep test on the original key of
// each edge, kept out-degrees (dplus, one atomic per run of a source: the
// list is sorted by source), kept in-degrees (spread, at hot_index), the
// tile's kept count and one keep bit per edge (32-edge words, in list order).
__global__ void __launch_bounds__(256) k_sample_rows(const uint64_t *__restrict__ rel,
                                                     const uint64_t *__restrict__ orig, uint64_t m,
                                                     uint64_t seed_mix, uint64_t thr, uint32_t *__restrict__ spread,
                                                     int hbits, uint32_t *__restrict__ dplus,
                                                     uint32_t *__restrict__ keepw, uint32_t *__restrict__ tile_cnt,
                                                     DevState *st, BatchView bv)
{
    __shared__ uint32_t wt[33];
    __shared__ uint32_t s_g;  // batch: graph of the tile's first edge
    const unsigned lane = lane_id();
    const uint64_t nt = (m + RX_TILE - 1) / RX_TILE;
    uint32_t kept_total = 0;
    for (uint64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        uint32_t c = 0;
        if (bv.k != 0) {
            if (threadIdx.x == 0) s_g = find_part(bv.eoff, bv.k, tile * RX_TILE);
            __syncthreads();
        }
        uint32_t gw = bv.k != 0 ? s_g : 0u;  // parts advance with the warp's edges
#pragma unroll 4
        for (int j = 0; j < RX_ITEMS; ++j) {
            const uint64_t i = tile * RX_TILE + (uint64_t)j * 256 + threadIdx.x;
            const uint64_t ii = i < m ? i : m - 1;
            const uint64_t o = ld_stream_u64(orig + ii);
            bool f;
            uint32_t g = 0;
            if (bv.k == 0) {
                f = i < m && keep_edge(o, seed_mix, thr);
            } else {
                g = find_part_warp_from(bv.eoff, bv.k, ii, gw);
                gw = __shfl_sync(FULL, g, 31);
                const uint64_t vo = __ldg(bv.voff + g);
                f = i < m && keep_edge(o - ((vo << 32) | vo), __ldg(bv.seed_mix + g), __ldg(bv.thr + g));
            }
            const unsigned word = __ballot_sync(FULL, f);
            if (lane == 0 && i - lane < m) keepw[(i - lane) >> 5] = word;
            if (word == 0) continue;  // warp-uniform
            const uint64_t r = f ? ld_stream_u64(rel + i) : 0ull;  // rank-order keys of the kept edges only
            const uint32_t u = f ? (uint32_t)(r >> 32) : 0xffffffffu;
            const unsigned peers = __match_any_sync(FULL, u);
            if (f) {
                if (lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(dplus + u, (uint32_t)__popc(peers));
                atomicAdd(spread + hot_index((uint32_t)r, hbits), 1u);
                ++c;
            }
            if (bv.k != 0) {
                const unsigned gp = __match_any_sync(FULL, g);
                const unsigned cg = __popc(word & gp);
                if (cg && lane == (unsigned)(__ffs(gp) - 1)) atomicAdd(bv.m_p + g, (unsigned long long)cg);
            }
        }
        if (bv.k != 0) __syncthreads();  // s_g is rewritten for the next tile
        kept_total += c;
        c = block_sum(c, wt);
        if (threadIdx.x == 0) tile_cnt[tile] = c;
    }
    kept_total = warp_sum(kept_total);
    if (lane == 0 && kept_total) atomicAdd(&st->m_sampled, (unsigned long long)kept_total);
}

// Sampled degree = kept out-degree + kept in-degree.
__global__ void k_degrees(const uint32_t *__restrict__ dplus, const uint32_t *__restrict__ spread, int hbits,
                          uint32_t n, uint32_t *__restrict__ deg)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        deg[x] = dplus[x] + spread[hot_index((uint32_t)x, hbits)];
}

// ---------------------------------------------------------------------
// Single graph.  Static rows (at creation): frow, the row offsets of the
// full graph in the rank-order key list, and inres, the offsets of the
// in-list reservations (full in-degrees = full degree - out-degree).  Per
// count the kept out-degrees are popcounts of the keep bits over each row,
// and kept in-degrees are counted only for the vertices that can be heavy.
// ---------------------------------------------------------------------

// Full out-degree of every rank id (one atomic per run of a source in a warp).
__global__ void k_full_outdeg(const uint64_t *__restrict__ rel, uint64_t m, uint32_t *__restrict__ outd)
{
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < m; base += stride) {
        const uint64_t i = base + lane;
        const uint32_t u = i < m ? (uint32_t)(ld_stream_u64(rel + i) >> 32) : 0xffffffffu;
        const unsigned peers = __match_any_sync(FULL, u);
        if (i < m && lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(outd + u, (unsigned)__popc(peers));
    }
}

// ind[x] = full degree of rank id x - its out-degree; ind[n] = 0.
__global__ void k_full_indeg(const uint32_t *__restrict__ perm, const uint32_t *__restrict__ deg_orig,
                             const uint32_t *__restrict__ outd, uint32_t n, uint32_t *__restrict__ ind)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n; x += stride)
        ind[x] = x < n ? __ldg(deg_orig + __ldg(perm + x)) - outd[x] : 0u;
}

__global__ void k_count_above(const uint32_t *__restrict__ deg, uint32_t n, uint32_t thr,
                              unsigned long long *__restrict__ out)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    uint32_t c = 0;
    for (uint64_t v = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) c += deg[v] > thr;
    c = __reduce_add_sync(FULL, c);
    if (lane_id() == 0 && c) atomicAdd(out, (unsigned long long)c);
}

void count_above(const uint32_t *deg, uint32_t n, uint32_t thr, unsigned long long *out, cudaStream_t s)
{
    cudaMemsetAsync(out, 0, sizeof(unsigned long long), s);
    if (n) k_count_above<<<grid_for(n, 256, 152 * 8), 256, 0, s>>>(deg, n, thr, out);
    note_launch();
}

void static_rows(const uint64_t *rel, uint64_t m, uint32_t n, const uint32_t *perm, const uint32_t *deg_orig,
                 uint32_t *frow, uint32_t *inres, uint32_t *scan, cudaStream_t s)
{
    const uint64_t n1 = (uint64_t)n + 1;
    cudaMemsetAsync(frow, 0, n1 * 4, s);
    if (m > 0) {
        k_full_outdeg<<<grid_for(m, 256, 152 * 16), 256, 0, s>>>(rel, m, frow);
        note_launch();
    }
    k_full_indeg<<<grid_for(n1, 256, 152 * 8), 256, 0, s>>>(perm, deg_orig, frow, n, inres);
    note_launch();
    scan_excl_u32(frow, n1, nullptr, scan, s);
    scan_excl_u32(inres, n1, nullptr, scan, s);
}

// Probe work of the p = 1 count among the top ranks, the candidates of the
// dense core: for every edge a -> b of the full graph (rank ids, rows in
// rank order) with a >= n - (core_min << (levels - 1)), the entries its pair
// streams: the part of a's row after b when a's row is the shorter, else b's
// whole row.  w[k] += that for the smallest core core_min << k holding a.
// Pairs of two heavy vertices (full degree d, d^2 > m) are left out: the
// heavy block takes them whether or not a core runs.
__global__ void k_core_work(const uint64_t *__restrict__ rel, const uint32_t *__restrict__ frow,
                            const uint32_t *__restrict__ inres, uint32_t n, uint64_t lo, uint64_t m,
                            uint32_t core_min, int levels, unsigned long long *__restrict__ w)
{
    unsigned long long acc[CORE_LEVELS_MAX] = {};  // this thread's sums, reduced once at the end
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = lo + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        const uint64_t e = rel[i];
        const uint32_t a = (uint32_t)(e >> 32), b = (uint32_t)e;
        const uint32_t fa = frow[a], da = frow[a + 1] - fa, db = frow[b + 1] - frow[b];
        const uint64_t fda = da + (inres[a + 1] - inres[a]), fdb = db + (inres[b + 1] - inres[b]);
        if (fda * fda > m && fdb * fdb > m) continue;
        const uint32_t pos = (uint32_t)(i - fa);
        const uint32_t str = da < db ? da - pos - 1 : db;
#pragma unroll
        for (int k = 0; k < CORE_LEVELS_MAX; ++k)  // the smallest core holding a
            if (k < levels && (k + 1 == levels || n - a <= (core_min << k)) &&
                (k == 0 || n - a > (core_min << (k - 1))))
                acc[k] += str;
    }
#pragma unroll
    for (int k = 0; k < CORE_LEVELS_MAX; ++k) {
        const unsigned long long v = warp_sum(acc[k]);
        if (lane_id() == 0 && v) atomicAdd(w + k, v);
    }
}

void core_work(const uint64_t *rel, const uint32_t *frow, const uint32_t *inres, uint32_t n, uint64_t m,
               uint32_t core_min, int levels, unsigned long long *w, cudaStream_t s)
{
    cudaMemsetAsync(w, 0, CORE_LEVELS_MAX * sizeof(unsigned long long), s);
    const uint64_t span = (uint64_t)core_min << (levels - 1);
    if (m == 0 || levels < 1 || levels > CORE_LEVELS_MAX || span > n) return;
    uint32_t lo_row = n - (uint32_t)span, lo = 0;
    cudaMemcpyAsync(&lo, frow + lo_row, 4, cudaMemcpyDeviceToHost, s);  // first edge of the top rows
    if (cudaStreamSynchronize(s) != cudaSuccess) return;
    k_core_work<<<grid_for(m - lo, 256, 152 * 8), 256, 0, s>>>(rel, frow, inres, n, lo, m, core_min, levels, w);
    note_launch();
}

// Smallest rank id whose full degree d has d^2 > m_lo (n if none): full
// degrees grow with the rank.
__device__ uint32_t cand_lo_of(const uint32_t *__restrict__ frow, const uint32_t *__restrict__ inres, uint32_t n,
                               uint64_t m_lo)
{
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = lo + (hi - lo) / 2;
        const unsigned long long d = (frow[mid + 1] - frow[mid]) + (inres[mid + 1] - inres[mid]);
        if (d * d > m_lo) hi = mid; else lo = mid + 1;
    }
    return lo;
}

// The Section 3.1 keep test of every edge (on its original key): keep bits
// (32-edge words in list order), kept edges per RX_TILE tile and m_p.  With
// m_p >= m_lo a heavy vertex has full degree^2 > m_lo, so the kept in-degrees
// are counted (spread, at hot_index) only for rank ids at or above that
// bound (DevState::cand_lo), from the kept edges' rank-order keys.  At p = 1
// every edge is kept: no hashing, and the in-degrees are the static ones.
__global__ void __launch_bounds__(256) k_sample_keep(const uint64_t *__restrict__ rel,
                                                     const uint64_t *__restrict__ orig, uint64_t m,
                                                     uint64_t seed_mix, uint64_t thr, uint32_t n,
                                                     const uint32_t *__restrict__ frow,
                                                     const uint32_t *__restrict__ inres, uint64_t m_lo,
                                                     uint32_t *__restrict__ spread, int hbits,
                                                     uint32_t *__restrict__ keepw, uint32_t *__restrict__ tile_cnt,
                                                     DevState *st)
{
    __shared__ uint32_t wt[33];
    __shared__ uint32_t s_cand;
    const unsigned lane = lane_id();
    const bool all = thr >= (1ull << 53);
    if (threadIdx.x == 0) {
        s_cand = cand_lo_of(frow, inres, n, m_lo);
        if (blockIdx.x == 0) st->cand_lo = s_cand;
    }
    __syncthreads();
    const uint32_t cand = s_cand;
    const bool count_in = !all && cand < n;
    const uint64_t nt = (m + RX_TILE - 1) / RX_TILE;
    uint32_t kept_total = 0;
    // keep test of a full tile: (h >> 11) < thr  <=>  h < thr * 2^11 (thr < 2^53 here)
    const uint64_t thr11 = all ? 0ull : thr << 11;
    for (uint64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        uint32_t c = 0;
        const bool full = (tile + 1) * RX_TILE <= m;
        constexpr int SU = 4;  // edges per thread in flight
#pragma unroll 1
        for (int j0 = 0; j0 < RX_ITEMS; j0 += SU) {
            bool f[SU];
            if (all) {
#pragma unroll
                for (int q = 0; q < SU; ++q) f[q] = tile * RX_TILE + (uint64_t)(j0 + q) * 256 + threadIdx.x < m;
            } else if (full) {
                const uint64_t *ot = orig + tile * RX_TILE + threadIdx.x;
                uint64_t o[SU];
#pragma unroll
                for (int q = 0; q < SU; ++q) o[q] = ld_stream_u64(ot + (j0 + q) * 256);
#pragma unroll
                for (int q = 0; q < SU; ++q) f[q] = splitmix64(o[q] ^ seed_mix) < thr11;
            } else {
                uint64_t o[SU];
#pragma unroll
                for (int q = 0; q < SU; ++q) {
                    const uint64_t i = tile * RX_TILE + (uint64_t)(j0 + q) * 256 + threadIdx.x;
                    o[q] = ld_stream_u64(orig + (i < m ? i : m - 1));
                }
#pragma unroll
                for (int q = 0; q < SU; ++q) {
                    const uint64_t i = tile * RX_TILE + (uint64_t)(j0 + q) * 256 + threadIdx.x;
                    f[q] = i < m && keep_edge(o[q], seed_mix, thr);
                }
            }
#pragma unroll
            for (int q = 0; q < SU; ++q) {
                const unsigned word = __ballot_sync(FULL, f[q]);
                const uint64_t w = tile * (RX_TILE / 32) + (uint64_t)(j0 + q) * 8 + (threadIdx.x >> 5);
                if (lane == 0 && w * 32 < m) keepw[w] = word;
                c += f[q];
            }
            if (count_in) {
#pragma unroll
                for (int q = 0; q < SU; ++q) {
                    const uint64_t i = tile * RX_TILE + (uint64_t)(j0 + q) * 256 + threadIdx.x;
                    if (f[q]) {
                        const uint32_t v = (uint32_t)ld_stream_u64(rel + i);
                        if (v >= cand) atomicAdd(spread + hot_index(v, hbits), 1u);
                    }
                }
            }
        }
        kept_total += c;
        c = block_sum(c, wt);
        if (threadIdx.x == 0) tile_cnt[tile] = c;
    }
    kept_total = warp_sum(kept_total);
    if (lane == 0 && kept_total) atomicAdd(&st->m_sampled, (unsigned long long)kept_total);
}

// Only if the sample came out below m_lo (the candidates might then miss a
// heavy vertex): the kept in-degrees of the rank ids below cand_lo too, and
// DevState::cand_all for the partition.
__global__ void __launch_bounds__(256) k_in_fallback(const uint64_t *__restrict__ rel, uint64_t m,
                                                     const uint32_t *__restrict__ keepw, uint64_t m_lo,
                                                     uint32_t *__restrict__ spread, int hbits, DevState *st)
{
    if (st->m_sampled >= m_lo) return;
    const uint32_t cand = st->cand_lo;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->cand_all = 1;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += stride) {
        if (!((keepw[i >> 5] >> (i & 31)) & 1u)) continue;
        const uint32_t v = (uint32_t)rel[i];
        if (v < cand) atomicAdd(spread + hot_index(v, hbits), 1u);
    }
}

// Kept out-degree of every rank id: the keep bits over its row; dplus[n] = 0.
__global__ void k_out_degrees(const uint32_t *__restrict__ frow, const uint32_t *__restrict__ keepw, uint32_t n,
                              uint32_t *__restrict__ dplus)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n; x += stride) {
        uint32_t d = 0;
        if (x < n) {
            const uint32_t b = frow[x], e = frow[x + 1];
            if (b < e) {
                const uint32_t wb = b >> 5, we = (e - 1) >> 5;
                for (uint32_t w = wb; w <= we; ++w) {
                    uint32_t word = __ldg(keepw + w);
                    if (w == wb) word &= 0xffffffffu << (b & 31);
                    if (w == we) word &= 0xffffffffu >> (31 - ((e - 1) & 31));
                    d += __popc(word);
                }
            }
        }
        dplus[x] = d;
    }
}

void sample_rows(const RowsArgs &a, cudaStream_t s)
{
    const int hb = hot_bits(a.n);
    if (a.frow) {
        cudaMemsetAsync(a.spread, 0, hot_size(a.n) * 4, s);
        if (a.m > 0) {
            const uint64_t nt = ceil_div(a.m, RX_TILE);
            k_sample_keep<<<grid_for(nt, 1, 152 * 8), 256, 0, s>>>(a.rel, a.orig, a.m, a.seed_mix, a.thr, a.n, a.frow,
                                                                     a.inptr, a.m_lo, a.spread, hb, a.keepw,
                                                                     a.tile_cnt, a.st);
            note_launch();
            k_in_fallback<<<152 * 4, 256, 0, s>>>(a.rel, a.m, a.keepw, a.m_lo, a.spread, hb, a.st);
            note_launch();
        }
        k_out_degrees<<<grid_for((uint64_t)a.n + 1, 256, 152 * 8), 256, 0, s>>>(a.frow, a.keepw, a.n, a.rowptr);
        note_launch();
        return;
    }
    cudaMemsetAsync(a.rowptr, 0, ((size_t)a.n + 1) * 4, s);
    cudaMemsetAsync(a.spread, 0, hot_size(a.n) * 4, s);
    if (a.m > 0) {
        const uint64_t nt = ceil_div(a.m, RX_TILE);
        k_sample_rows<<<grid_for(nt, 1, 152 * 8), 256, 0, s>>>(a.rel, a.orig, a.m, a.seed_mix, a.thr, a.spread, hb,
                                                                 a.rowptr, a.keepw, a.tile_cnt, a.st, a.bv);
        note_launch();
    }
    k_degrees<<<grid_for(a.n, 256, 152 * 8), 256, 0, s>>>(a.rowptr, a.spread, hb, a.n, a.deg);
    note_launch();
}

// ======================================================================
// The CSR: padded columns and in-lists
// ======================================================================

__device__ __forceinline__ uint32_t pad_of(uint32_t d) { return (4u - (d & 3u)) & 3u; }

// dplus holds the kept out-degrees: ptrp[x] = pad count of row x and
// P[x] = in-degree deg - d+ of x (x < n), the room of x's in-list; ptrp[n]
// = P[n] = 0.  deg[x] is replaced by d+ (the partition has used it).
__global__ void k_row_counts(const uint32_t *__restrict__ dplus, uint32_t *__restrict__ deg, uint32_t n,
                             uint32_t *__restrict__ ptrp, uint32_t *__restrict__ P, uint32_t *__restrict__ ocnt)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n; x += stride) {
        const uint32_t dp = x < n ? dplus[x] : 0u;
        ptrp[x] = pad_of(dp);
        if (P) P[x] = x < n ? deg[x] - dp : 0u;
        if (x < n) {
            deg[x] = dp;
            ocnt[x] = 0;
        }
    }
}

// In-list cursors at hot_index: cursor of v = start of v's in-list.
__global__ void k_cursors(const uint32_t *__restrict__ P, uint32_t n, int hbits, uint32_t *__restrict__ spread)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < n; x += stride)
        spread[hot_index((uint32_t)x, hbits)] = P[x];
}

// One kept edge per live lane: (u -> v) at list index i, CSR position k.
// All lanes of the warp call it (the out-list appends are warp-aggregated).
struct ScatterArgs {
    const uint64_t *rel;
    const uint32_t *padoff, *rowptr, *dplus;
    uint32_t *colp, *cursor, *ocnt;
    uint2 *inlist, *olist;
    int hbits;
    // heavy flags; pairs left to the dense blocks: light_lim when the heavy
    // block runs (else lim = EMPTY), the core's base when it runs
    const uint8_t *heavy;
    uint32_t lim, core_lo;
};

__device__ __forceinline__ void scatter_edge(const ScatterArgs &a, bool live, uint64_t i, uint32_t k, unsigned lt)
{
    uint32_t u = 0, v = 0;
    bool out = false;
    uint2 ev = make_uint2(0, 0);
    if (live) {
        const uint64_t r = ld_stream_u64(a.rel + i);
        u = (uint32_t)(r >> 32);
        v = (uint32_t)r;
        const uint32_t pos = k + __ldg(a.padoff + u);
        a.colp[pos] = v;
        const bool dense_pair =
            u >= a.core_lo || (v >= a.lim && __ldg(a.heavy + u) && __ldg(a.heavy + v));  // see ScatterArgs
        if (!dense_pair && k + 1 < __ldg(a.rowptr + u + 1)) {  // so d+(u) >= 2
            const uint32_t du = __ldg(a.dplus + u), dv = __ldg(a.dplus + v);
            if (du < dv) {  // entry: position of v in u's row; entries after it | u's heavy flag << 31
                const uint32_t q = atomicAdd(a.cursor + hot_index(v, a.hbits), 1u);
                const uint32_t after = __ldg(a.rowptr + u + 1) - k - 1;
                a.inlist[q] = make_uint2(pos, after | ((uint32_t)__ldg(a.heavy + u) << 31));
            } else if (dv >= 1) {  // entry: v, d+(v) | v's flag << 31 (if u is heavy)
                out = true;
                ev = make_uint2(v, dv | (__ldg(a.heavy + u) ? (uint32_t)__ldg(a.heavy + v) << 31 : 0u));
            }
        }
    }
    const unsigned act = __ballot_sync(FULL, out);
    if (out) {
        const unsigned grp = __match_any_sync(act, u);  // lanes of this warp with the same row
        const int lead = __ffs(grp) - 1;
        uint32_t q = 0;
        if ((int)lane_id() == lead) q = atomicAdd(a.ocnt + u, (unsigned)__popc(grp));
        q = __shfl_sync(grp, q, lead) + __popc(grp & lt);
        a.olist[__ldg(a.rowptr + u) + q] = ev;
    }
}

// The same for N kept-or-not edges of a thread at once, in phases: every
// edge's key and the random reads it needs, then the in-list cursor atomics,
// then the writes, so that the reads and atomics of the N edges are in flight
// together instead of one edge's chain after another.
template <int N>
__device__ __forceinline__ void scatter_edges(const ScatterArgs &a, const bool (&live)[N], const uint64_t (&i)[N],
                                              const uint32_t (&k)[N], unsigned lt)
{
    uint32_t u[N], v[N], pos[N], du[N], dv[N], row_end[N];
    bool cand[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        u[j] = v[j] = pos[j] = du[j] = dv[j] = row_end[j] = 0;
        cand[j] = false;
        if (live[j]) {
            const uint64_t r = ld_stream_u64(a.rel + i[j]);
            u[j] = (uint32_t)(r >> 32);
            v[j] = (uint32_t)r;
            pos[j] = k[j] + __ldg(a.padoff + u[j]);
            row_end[j] = __ldg(a.rowptr + u[j] + 1);
            const bool dense_pair =
                u[j] >= a.core_lo || (v[j] >= a.lim && __ldg(a.heavy + u[j]) && __ldg(a.heavy + v[j]));
            cand[j] = !dense_pair && k[j] + 1 < row_end[j];  // so d+(u) >= 2
            if (cand[j]) {
                du[j] = __ldg(a.dplus + u[j]);
                dv[j] = __ldg(a.dplus + v[j]);
            }
        }
    }
    uint32_t q[N];
#pragma unroll
    for (int j = 0; j < N; ++j) {
        q[j] = 0;
        if (cand[j] && du[j] < dv[j]) q[j] = atomicAdd(a.cursor + hot_index(v[j], a.hbits), 1u);
    }
#pragma unroll
    for (int j = 0; j < N; ++j) {
        if (live[j]) a.colp[pos[j]] = v[j];
        bool out = false;
        uint2 ev = make_uint2(0, 0);
        if (cand[j]) {
            const uint32_t hu = __ldg(a.heavy + u[j]);
            if (du[j] < dv[j]) {  // entry: position of v in u's row; entries after it | u's heavy flag << 31
                a.inlist[q[j]] = make_uint2(pos[j], (row_end[j] - k[j] - 1) | (hu << 31));
            } else if (dv[j] >= 1) {  // entry: v, d+(v) | v's flag << 31 (if u is heavy)
                out = true;
                ev = make_uint2(v[j], dv[j] | (hu ? (uint32_t)__ldg(a.heavy + v[j]) << 31 : 0u));
            }
        }
        const unsigned act = __ballot_sync(FULL, out);
        if (out) {
            const unsigned grp = __match_any_sync(act, u[j]);  // lanes of this warp with the same row
            const int lead = __ffs(grp) - 1;
            uint32_t qo = 0;
            if ((int)lane_id() == lead) qo = atomicAdd(a.ocnt + u[j], (unsigned)__popc(grp));
            qo = __shfl_sync(grp, qo, lead) + __popc(grp & lt);
            a.olist[__ldg(a.rowptr + u[j]) + qo] = ev;
        }
    }
}

// Position of the k-th (from 0) set bit of w; k < popcount(w).
__device__ __forceinline__ uint32_t nth_set_bit(uint32_t w, uint32_t k)
{
    uint32_t pos = 0;
#pragma unroll
    for (uint32_t s = 16; s >= 1; s >>= 1) {
        const uint32_t c = __popc(w & ((1u << s) - 1u));
        if (k >= c) {
            k -= c;
            w >>= s;
            pos += s;
        }
    }
    return pos;
}

// Writes every kept edge (u -> v) at its place in the padded rows (its
// index among the kept edges, which is its CSR position, plus the padding
// before row u) and, when u's row goes on past v (else the pair closes no
// triangle), hands the pair to its owner (isect.cu): to v's in-list as (u,
// that position) if d+(u) < d+(v) (cursors at hot_index), else, if d+(v) >=
// 1, to u's out-list (ocnt: per-row counts, one atomic per run of u in a
// warp).  Within a list the order is that of the atomics.  A tile with at
// most half its edges kept hands its kept edges to the threads one after
// another (the word and bit of kept edge e found from the word prefixes)
// instead of one edge slot per thread.
template <int NB>
__global__ void __launch_bounds__(256) k_rows_scatter(const uint64_t *__restrict__ rel, uint64_t m,
                                                      const uint32_t *__restrict__ keepw,
                                                      const uint32_t *__restrict__ tile_off,
                                                      const uint32_t *__restrict__ padoff,
                                                      const uint32_t *__restrict__ rowptr,
                                                      const uint32_t *__restrict__ dplus,
                                                      uint32_t *__restrict__ colp, uint32_t *__restrict__ cursor,
                                                      int hbits, uint2 *__restrict__ inlist,
                                                      uint2 *__restrict__ olist, uint32_t *__restrict__ ocnt,
                                                      const uint8_t *__restrict__ heavy, uint32_t core_base,
                                                      const DevState *st)
{
    constexpr int WORDS = RX_TILE / 32;  // 128 keep words per tile
    __shared__ uint32_t s_word[WORDS], s_pre[WORDS];
    __shared__ uint32_t wt[33];
    const bool dense = st->dense != 0;
    const ScatterArgs a{rel,   padoff, rowptr, dplus, colp, cursor, ocnt, inlist, olist, hbits, heavy,
                        dense ? st->light_lim : 0xffffffffu, dense && st->core_on ? core_base : 0xffffffffu};
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5;
    const unsigned lt = lanemask_lt();
    const uint64_t nt = (m + RX_TILE - 1) / RX_TILE;
    for (uint64_t tile = blockIdx.x; tile < nt; tile += gridDim.x) {
        const uint64_t w0 = tile * WORDS, nw = (m + 31) / 32;
        uint32_t c = 0;
        if (threadIdx.x < WORDS) {
            const uint32_t word = w0 + threadIdx.x < nw ? keepw[w0 + threadIdx.x] : 0u;
            s_word[threadIdx.x] = word;
            c = __popc(word);
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan(c, wt, &tot);  // word order = list order
        if (threadIdx.x < WORDS) s_pre[threadIdx.x] = ex;
        __syncthreads();
        const uint32_t base = tile_off[tile];
        if (tot <= RX_TILE / 2) {
            for (uint32_t e0 = 0; e0 < tot; e0 += 256) {
                const uint32_t e = e0 + threadIdx.x;
                const bool live = e < tot;
                uint64_t i = 0;
                if (live) {
                    uint32_t lo = 0, hi = WORDS - 1;  // last word with s_pre <= e holds kept edge e
                    while (lo < hi) {
                        const uint32_t mid = (lo + hi + 1) >> 1;
                        if (s_pre[mid] <= e) lo = mid; else hi = mid - 1;
                    }
                    i = tile * RX_TILE + lo * 32 + nth_set_bit(s_word[lo], e - s_pre[lo]);
                }
                scatter_edge(a, live, i, base + e, lt);
            }
        } else if (NB == 1) {
#pragma unroll 4
            for (int j = 0; j < RX_ITEMS; ++j) {
                const uint32_t wi = j * 8 + warp;  // word of this warp's 32 edges
                const uint32_t word = s_word[wi];
                scatter_edge(a, (word >> lane) & 1u, tile * RX_TILE + (uint64_t)j * 256 + threadIdx.x,
                             base + s_pre[wi] + __popc(word & lt), lt);
            }
        } else {  // NB edges of a thread in flight together
            for (int j0 = 0; j0 < RX_ITEMS; j0 += NB) {
                bool live[NB];
                uint64_t i[NB];
                uint32_t k[NB];
#pragma unroll
                for (int jj = 0; jj < NB; ++jj) {
                    const int j = j0 + jj;
                    const uint32_t wi = j * 8 + warp;  // word of this warp's 32 edges
                    const uint32_t word = s_word[wi];
                    live[jj] = (word >> lane) & 1u;
                    i[jj] = tile * RX_TILE + (uint64_t)j * 256 + threadIdx.x;
                    k[jj] = base + s_pre[wi] + __popc(word & lt);
                }
                scatter_edges<NB>(a, live, i, k, lt);
            }
        }
        __syncthreads();  // s_word / s_pre are rewritten for the next tile
    }
}

// Row x's padding (SENT) and ptrp[x] = padded start | pad count; ptrp holds
// the exclusive scan of the pad counts and rowptr the row offsets.  Also the
// end of x's in-list (its cursor at hot_index) into inend[x].
__global__ void k_pad_finish(const uint32_t *__restrict__ rowptr, uint32_t n, uint32_t *__restrict__ ptrp,
                             uint32_t *__restrict__ colp, const uint32_t *__restrict__ cursor, int hbits,
                             uint32_t *__restrict__ inend)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n; x += stride) {
        const uint32_t start = rowptr[x] + ptrp[x];
        if (x == n) {
            ptrp[x] = start;
            continue;
        }
        inend[x] = cursor[hot_index((uint32_t)x, hbits)];
        const uint32_t d = rowptr[x + 1] - rowptr[x], pad = pad_of(d);
        for (uint32_t i = 0; i < pad; ++i) colp[start + d + i] = SENT;
        ptrp[x] = start | pad;
    }
}

void build_rows(const RowsArgs &a, cudaStream_t s)
{
    const uint64_t n1 = (uint64_t)a.n + 1;
    const int hb = hot_bits(a.n);
    // single graph: the in-list reservations are the static ones (inptr)
    k_row_counts<<<grid_for(n1, 256, 152 * 8), 256, 0, s>>>(a.rowptr, a.deg, a.n, a.ptrp, a.frow ? nullptr : a.inptr,
                                                          a.ocnt);
    note_launch();
    scan_excl_pair(a.ptrp, a.rowptr, n1, a.scan, s);
    if (!a.frow) scan_excl_u32(a.inptr, n1, nullptr, a.scan, s);
    if (a.m > 0) {
        const uint64_t nt = ceil_div(a.m, RX_TILE);
        scan_excl_u32(a.tile_cnt, nt, nullptr, a.scan, s);
    }
    if (!a.frow) {  // single graph: the partition set the cursors
        k_cursors<<<grid_for(a.n, 256, 152 * 8), 256, 0, s>>>(a.inptr, a.n, hb, a.spread);
        note_launch();
    }
    if (a.m > 0) {
        const uint64_t nt = ceil_div(a.m, RX_TILE);
        auto kern = a.scatter4 ? k_rows_scatter<4> : k_rows_scatter<1>;
        kern<<<grid_for(nt, 1, 152 * 8), 256, 0, s>>>(a.rel, a.m, a.keepw, a.tile_cnt, a.ptrp, a.rowptr, a.deg, a.colp,
                                                       a.spread, hb, a.inlist, a.olist, a.ocnt, a.heavy, a.core_base,
                                                       a.st);
        note_launch();
    }
    k_pad_finish<<<grid_for(n1, 256, 152 * 8), 256, 0, s>>>(a.rowptr, a.n, a.ptrp, a.colp, a.spread, hb, a.inend);
    note_launch();
}

}  // namespace tcg
