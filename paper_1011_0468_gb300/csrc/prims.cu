// Data-movement primitives of libtc: device-wide exclusive scan, stable LSD
// radix passes over 64-bit items, and the canonicalisation of raw edge lists.
//
// The CSR of the sampled graph is built by a stable radix sort of the
// oriented kept edges (src << 32 | dst) on the src bits only.  The first pass
// reads the canonical edge list directly and fuses the edge sampling of
// Section 3.1 and the degree orientation into its loader, so the kept-edge
// list is never materialised.  Because the canonical list is sorted by
// (min, max), a stable sort on src alone leaves every row sorted by dst.
#include "kernels.h"

namespace tcg {

// ======================================================================
// Exclusive scan (reduce -> spine -> downsweep), 4096 elements per block.
// ======================================================================

constexpr int SC_THREADS = 1024;
constexpr int SC_ITEMS = SC_CHUNK / SC_THREADS;  // 4

// Effective scan length: len, or for a device-counted item list the digit
// histograms of its tiles only.
__device__ __forceinline__ uint64_t scan_len(uint64_t len, const unsigned long long *dyn_items, uint32_t dyn_bins)
{
    if (!dyn_items) return len;
    const uint64_t l = (uint64_t)dyn_bins * ((*dyn_items + RX_TILE - 1) / RX_TILE);
    return l < len ? l : len;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(const uint32_t *__restrict__ a, uint64_t len,
                                                            uint32_t *__restrict__ part,
                                                            const unsigned long long *dyn_items, uint32_t dyn_bins)
{
    __shared__ uint32_t wt[33];
    len = scan_len(len, dyn_items, dyn_bins);
    const uint64_t base = (uint64_t)blockIdx.x * SC_CHUNK;
    if (base >= len) return;  // uniform across the block
    uint32_t s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        uint64_t i = base + (uint64_t)j * SC_THREADS + threadIdx.x;
        if (i < len) s += a[i];
    }
    s = block_sum(s, wt);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

// One block scans the per-block sums in place (exclusive); writes the
// grand total to total_out when non-NULL.
__global__ void __launch_bounds__(SC_THREADS) k_scan_spine(uint32_t *part, uint64_t len, uint32_t *total_out,
                                                           const unsigned long long *dyn_items, uint32_t dyn_bins)
{
    __shared__ uint32_t wt[33];
    const uint64_t nparts = (scan_len(len, dyn_items, dyn_bins) + SC_CHUNK - 1) / SC_CHUNK;
    uint32_t carry = 0;
    for (uint64_t base = 0; base < nparts; base += SC_THREADS) {
        uint64_t i = base + threadIdx.x;
        uint32_t x = i < nparts ? part[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan(x, wt, &tot);
        if (i < nparts) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan_down(uint32_t *a, uint64_t len, const uint32_t *__restrict__ part,
                                                          const unsigned long long *dyn_items, uint32_t dyn_bins)
{
    __shared__ uint32_t wt[33];
    len = scan_len(len, dyn_items, dyn_bins);
    const uint64_t base = (uint64_t)blockIdx.x * SC_CHUNK;
    if (base >= len) return;  // uniform across the block
    uint32_t carry = part[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        uint64_t i = base + (uint64_t)j * SC_THREADS + threadIdx.x;
        uint32_t x = i < len ? a[i] : 0u;
        uint32_t tot;
        uint32_t ex = block_excl_scan(x, wt, &tot);
        if (i < len) a[i] = carry + ex;
        carry += tot;
    }
}

uint64_t scan_scratch_elems(uint64_t len) { return ceil_div(len, SC_CHUNK) + 1; }

void scan_excl_u32(uint32_t *a, uint64_t len, uint32_t *total, uint32_t *scratch, cudaStream_t s,
                   const unsigned long long *dyn_items, uint32_t dyn_bins)
{
    if (len == 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return;
    }
    const uint64_t nb = ceil_div(len, SC_CHUNK);
    k_scan_reduce<<<(unsigned)nb, SC_THREADS, 0, s>>>(a, len, scratch, dyn_items, dyn_bins); note_launch();
    k_scan_spine<<<1, SC_THREADS, 0, s>>>(scratch, len, total, dyn_items, dyn_bins); note_launch();
    k_scan_down<<<(unsigned)nb, SC_THREADS, 0, s>>>(a, len, scratch, dyn_items, dyn_bins); note_launch();
}

// ======================================================================
// Stable LSD radix pass.
// ======================================================================

// Loads item i of a pass; returns false when the item does not take part
// (an edge that the sampling drops).
// g: the batch graph of item i (batch unions only).
__device__ __forceinline__ bool load_item(const ItemSource &src, uint64_t i, uint64_t &item, uint32_t g)
{
    if (src.kind == ItemSource::PLAIN) {
        item = ld_stream_u64(src.in + i);
        return true;
    }
    const uint64_t key = ld_stream_u64(src.in + i);
    if (src.kind == ItemSource::ORIENT) {
        item = orient(key, src.deg);
        return true;
    }
    if (src.bv.k == 0) {
        if (!keep_edge(key, src.seed_mix, src.thr)) return false;
    } else {
        const uint64_t vo = __ldg(src.bv.voff + g);
        if (!keep_edge(key - ((vo << 32) | vo), __ldg(src.bv.seed_mix + g), __ldg(src.bv.thr + g))) return false;
    }
    item = orient(key, src.deg);
    return true;
}

// Batch graph of item i for every lane of a full warp (indices consecutive
// across lanes); 0 unless the source samples a batch union.
__device__ __forceinline__ uint32_t item_graph(const ItemSource &src, uint64_t i, uint64_t n)
{
    if (src.kind != ItemSource::SAMPLE_ORIENT || src.bv.k == 0) return 0;
    return find_part_warp(src.bv.eoff, src.bv.k, i < n ? i : n - 1);
}

// Per-tile digit counts (per-warp shared histograms, summed at the end), plus
// the out-degree histogram (first pass).
__global__ void __launch_bounds__(RX_THREADS) k_radix_count(ItemSource src, int shift, int width,
                                                            uint32_t *__restrict__ hist, uint32_t ntiles,
                                                            uint32_t *__restrict__ dplus)
{
    constexpr int NW = RX_THREADS / 32;
    __shared__ uint32_t cnt[NW][RX_BINS];
    const uint64_t n = src.n_dev ? *src.n_dev : src.n_host;
    const uint32_t tile = blockIdx.x;
    if (src.n_dev) {  // device-counted items: only their tiles have histograms
        const uint64_t nt = (n + RX_TILE - 1) / RX_TILE;
        if (tile >= nt) return;  // uniform across the block
        ntiles = (uint32_t)nt;
    }
    const int nb = 1 << width;
    const unsigned warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < NW * RX_BINS; i += RX_THREADS) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)tile * RX_TILE;
    if (base < n) {
        const uint32_t mask = (uint32_t)nb - 1;
        for (int j = 0; j < RX_ITEMS; ++j) {
            const uint64_t i = base + (uint64_t)j * RX_THREADS + threadIdx.x;
            uint64_t item = 0;
            const uint32_t g = item_graph(src, i, n);
            const bool valid = i < n && load_item(src, i, item, g);
            if (valid) atomicAdd(&cnt[warp][(uint32_t)(item >> shift) & mask], 1u);
            if (dplus) {
                // runs of one source are common (canonical order): one atomic per run
                const uint32_t x = valid ? (uint32_t)(item >> 32) : 0xffffffffu;
                const unsigned peers = __match_any_sync(FULL, x);
                if (valid && lane_id() == (unsigned)(__ffs(peers) - 1)) atomicAdd(dplus + x, (uint32_t)__popc(peers));
            }
        }
    }
    __syncthreads();
    for (int d = threadIdx.x; d < nb; d += RX_THREADS) {
        uint32_t c = 0;
#pragma unroll
        for (int w = 0; w < NW; ++w) c += cnt[w][d];
        hist[(uint64_t)d * ntiles + tile] = c;
    }
}

// Stable scatter of one tile: rank every item within its digit (warp
// order, then item order), sort the tile by digit in shared memory, and
// write each digit's run to its global offset with consecutive threads on
// consecutive positions.  With in-lists, each item is also appended to its
// dst's list; a thread issues all its appends before writing any entry.
__global__ void __launch_bounds__(RX_THREADS) k_radix_scatter(ItemSource src, int shift, int width,
                                                              const uint32_t *__restrict__ offs, uint32_t ntiles,
                                                              uint64_t *__restrict__ out,
                                                              uint32_t *__restrict__ out_low32, InListArgs in,
                                                              const uint32_t *__restrict__ padoff)
{
    constexpr int NW = RX_THREADS / 32;
    static_assert(RX_BINS == RX_THREADS, "one digit per thread in the tile scan");
    __shared__ uint64_t s_items[RX_TILE];
    __shared__ uint32_t whist[NW][RX_BINS];
    __shared__ uint32_t tstart[RX_BINS];  // first local position of each digit in the sorted tile
    __shared__ uint32_t tbase[RX_BINS];   // global position of each digit's run
    __shared__ uint32_t wt[33];
    const uint64_t n = src.n_dev ? *src.n_dev : src.n_host;
    const uint32_t tile = blockIdx.x;
    const uint64_t base = (uint64_t)tile * RX_TILE;
    if (base >= n) return;  // uniform across the block
    if (src.n_dev) ntiles = (uint32_t)((n + RX_TILE - 1) / RX_TILE);  // histogram stride of this pass
    const int nb = 1 << width;
    const uint32_t mask = (uint32_t)nb - 1;
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    for (int i = threadIdx.x; i < NW * RX_BINS; i += RX_THREADS) (&whist[0][0])[i] = 0;
    for (int d = threadIdx.x; d < nb; d += RX_THREADS) tbase[d] = offs[(uint64_t)d * ntiles + tile];

    uint64_t items[RX_ITEMS];
    uint32_t packed[RX_ITEMS];  // digit << 16 | rank within (warp, digit); ~0 = absent
    const uint64_t seg = base + (uint64_t)warp * 32 * RX_ITEMS;
    const unsigned lt = lanemask_lt();
#pragma unroll
    for (int j = 0; j < RX_ITEMS; ++j) {  // all loads first
        const uint64_t i = seg + (uint64_t)j * 32 + lane;
        items[j] = 0;
        const uint32_t g = item_graph(src, i, n);
        packed[j] = (i < n && load_item(src, i, items[j], g)) ? 0u : 0xffffffffu;
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RX_ITEMS; ++j) {
        const bool valid = packed[j] == 0u;
        const uint32_t d = valid ? ((uint32_t)(items[j] >> shift) & mask) : 0xffffffffu;
        const unsigned peers = __match_any_sync(FULL, d);
        uint32_t r = 0;
        if (valid) r = whist[warp][d] + (uint32_t)__popc(peers & lt);
        __syncwarp();
        if (valid && lane == (unsigned)(__ffs(peers) - 1)) whist[warp][d] += (uint32_t)__popc(peers);
        __syncwarp();
        packed[j] = valid ? ((d << 16) | r) : 0xffffffffu;
    }
    __syncthreads();
    // per digit: offsets of the warps' runs, and the digit's start in the tile
    uint32_t tot = 0;
    {
        const int d = threadIdx.x;  // RX_BINS == RX_THREADS
        if (d < nb) {
#pragma unroll
            for (int w = 0; w < NW; ++w) {
                const uint32_t c = whist[w][d];
                whist[w][d] = tot;
                tot += c;
            }
        }
    }
    uint32_t count;  // valid items of the tile
    const uint32_t start = block_excl_scan(tot, wt, &count);
    tstart[threadIdx.x] = start;
    __syncthreads();
#pragma unroll
    for (int j = 0; j < RX_ITEMS; ++j) {
        if (packed[j] == 0xffffffffu) continue;
        const uint32_t d = packed[j] >> 16, r = packed[j] & 0xffffu;
        s_items[tstart[d] + whist[warp][d] + r] = items[j];
    }
    __syncthreads();
    uint32_t q[RX_ITEMS];
#pragma unroll
    for (int k = 0; k < RX_ITEMS; ++k) {
        const uint32_t i = threadIdx.x + k * RX_THREADS;
        q[k] = 0xffffffffu;
        if (i < count) {
            const uint64_t item = s_items[i];
            const uint32_t d = (uint32_t)(item >> shift) & mask;
            const uint32_t pos = tbase[d] + (i - tstart[d]);
            if (out_low32)
                out_low32[padoff ? pos + __ldg(padoff + (item >> 32)) : pos] = (uint32_t)item;
            else
                out[pos] = item;
            if (in.P) q[k] = atomicAdd(in.P + (uint32_t)item + 1, 1u);
        }
    }
    if (in.P) {
#pragma unroll
        for (int k = 0; k < RX_ITEMS; ++k)
            if (q[k] != 0xffffffffu) in.inlist[q[k]] = (uint32_t)(s_items[threadIdx.x + k * RX_THREADS] >> 32);
    }
}

void radix_pass(const ItemSource &src, uint64_t n_max, int shift, int width, uint32_t *hist,
                uint32_t *scan_scratch, uint32_t *dplus, uint64_t *out, uint32_t *out_low32,
                const InListArgs *in, cudaStream_t s, const uint32_t *padoff)
{
    const InListArgs inl = in ? *in : InListArgs{nullptr, nullptr, 0};
    const uint64_t ntiles = ceil_div(n_max, RX_TILE);
    if (ntiles == 0) return;
    k_radix_count<<<(unsigned)ntiles, RX_THREADS, 0, s>>>(src, shift, width, hist, (uint32_t)ntiles, dplus); note_launch();
    scan_excl_u32(hist, ntiles << width, nullptr, scan_scratch, s, src.n_dev, 1u << width);
    k_radix_scatter<<<(unsigned)ntiles, RX_THREADS, 0, s>>>(src, shift, width, hist, (uint32_t)ntiles, out,
                                                            out_low32, inl, padoff); note_launch();
}

// ======================================================================
// Canonicalisation of raw pairs (graph creation).
// ======================================================================

__global__ void k_canon_keys(const uint32_t *__restrict__ pairs, uint64_t m_in, uint32_t n,
                             uint64_t *__restrict__ keys, DevState *st)
{
    unsigned bad = 0, unsorted = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m_in; i += stride) {
        const uint2 e = make_uint2(pairs[2 * i], pairs[2 * i + 1]);  // 4-byte alignment suffices
        uint64_t k;
        if (e.x >= n || e.y >= n) {
            bad = 1;
            k = ~0ull;
        } else if (e.x == e.y) {
            k = ~0ull;
        } else {
            const uint32_t u = min(e.x, e.y), v = max(e.x, e.y);
            k = ((uint64_t)u << 32) | v;
        }
        keys[i] = k;
        // the list is already canonical iff every pair is (u < v) and the
        // sequence strictly increases
        if (e.x >= e.y) {
            unsorted++;
        } else if (i > 0) {
            const uint2 q = make_uint2(pairs[2 * i - 2], pairs[2 * i - 1]);
            if (!(q.x < e.x || (q.x == e.x && q.y < e.y))) unsorted++;
        }
    }
    if (__any_sync(FULL, bad) && lane_id() == 0) atomicOr(&st->err, ERR_ENDPOINT);
    unsorted = warp_sum(unsorted);
    if (unsorted && lane_id() == 0) atomicAdd(&st->unsorted, unsorted);
}

void canon_keys(const uint32_t *pairs, uint64_t m_in, uint32_t n, uint64_t *keys, DevState *st,
                cudaStream_t s)
{
    if (m_in == 0) return;
    const uint64_t blocks = std::min<uint64_t>(ceil_div(m_in, 256), 152ull * 16);
    k_canon_keys<<<(unsigned)blocks, 256, 0, s>>>(pairs, m_in, n, keys, st); note_launch();
}

constexpr int UQ_THREADS = 1024;
constexpr int UQ_ITEMS = RX_TILE / UQ_THREADS;  // 4

__device__ __forceinline__ bool unique_flag(const uint64_t *keys, uint64_t i)
{
    const uint64_t k = keys[i];
    return k != ~0ull && (i == 0 || keys[i - 1] != k);
}

__global__ void __launch_bounds__(UQ_THREADS) k_unique_count(const uint64_t *__restrict__ keys, uint64_t m,
                                                             uint32_t *__restrict__ tile_cnt)
{
    __shared__ uint32_t wt[33];
    const uint64_t base = (uint64_t)blockIdx.x * RX_TILE;
    uint32_t c = 0;
#pragma unroll
    for (int j = 0; j < UQ_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * UQ_THREADS + threadIdx.x;
        if (i < m && unique_flag(keys, i)) ++c;
    }
    c = block_sum(c, wt);
    if (threadIdx.x == 0) tile_cnt[blockIdx.x] = c;
}

__global__ void __launch_bounds__(UQ_THREADS) k_unique_scatter(const uint64_t *__restrict__ keys, uint64_t m,
                                                               const uint32_t *__restrict__ tile_off,
                                                               uint64_t *__restrict__ out)
{
    __shared__ uint32_t wt[33];
    const uint64_t base = (uint64_t)blockIdx.x * RX_TILE;
    uint32_t carry = tile_off[blockIdx.x];
#pragma unroll
    for (int j = 0; j < UQ_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * UQ_THREADS + threadIdx.x;
        const bool f = i < m && unique_flag(keys, i);
        uint32_t tot;
        const uint32_t ex = block_excl_scan((uint32_t)f, wt, &tot);
        if (f) out[carry + ex] = keys[i];
        carry += tot;
    }
}

__global__ void k_store_count(const uint32_t *total, DevState *st) { st->m_canon = *total; }

void unique_keys(const uint64_t *keys, uint64_t m_in, uint64_t *out, uint32_t *tile_cnt,
                 uint32_t *scan_scratch, DevState *st, cudaStream_t s)
{
    const uint64_t nt = ceil_div(m_in, RX_TILE);
    if (nt == 0) {
        cudaMemsetAsync(&st->m_canon, 0, sizeof(st->m_canon), s);
        return;
    }
    k_unique_count<<<(unsigned)nt, UQ_THREADS, 0, s>>>(keys, m_in, tile_cnt); note_launch();
    scan_excl_u32(tile_cnt, nt, tile_cnt + nt, scan_scratch, s);
    k_unique_scatter<<<(unsigned)nt, UQ_THREADS, 0, s>>>(keys, m_in, tile_cnt, out); note_launch();
    k_store_count<<<1, 1, 0, s>>>(tile_cnt + nt, st); note_launch();
}

}  // namespace tcg

namespace tcg {

// ======================================================================
// Padded rows (see SENT in kernels.h).
// ======================================================================

__device__ __forceinline__ uint32_t pad_of(uint32_t d) { return (4u - (d & 3u)) & 3u; }

// Once the out-degrees d+ are counted (dplus): ptrp[x] = pad count of row x,
// and P[1 + x] = in-degree deg - d+ of x (x < n); ptrp[n] = P[n + 1] = 0,
// P[0] = 0.
__global__ void k_row_counts(const uint32_t *__restrict__ dplus, const uint32_t *__restrict__ deg, uint32_t n,
                             uint32_t *__restrict__ ptrp, uint32_t *__restrict__ P)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n; x += stride) {
        const uint32_t dp = x < n ? dplus[x] : 0u;
        ptrp[x] = pad_of(dp);
        P[x + 1] = x < n ? deg[x] - dp : 0u;
        if (x == 0) P[0] = 0;
    }
}

// ptrp holds the exclusive scan of the pad counts and rowptr the row
// offsets: write each row's padding and turn ptrp into padded starts
// tagged with the pad count.
__global__ void k_pad_finish(const uint32_t *__restrict__ rowptr, uint32_t n, uint32_t *__restrict__ ptrp,
                             uint32_t *__restrict__ colp)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x <= n; x += stride) {
        const uint32_t start = rowptr[x] + ptrp[x];
        if (x == n) {
            ptrp[x] = start;
            continue;
        }
        const uint32_t d = rowptr[x + 1] - rowptr[x], pad = pad_of(d);
        for (uint32_t i = 0; i < pad; ++i) colp[start + d + i] = SENT;
        ptrp[x] = start | pad;
    }
}

void csr_build(const CsrArgs &a, uint32_t **col, uint32_t **inlist, cudaStream_t s)
{
    cudaMemsetAsync(a.rowptr, 0, ((size_t)a.n + 1) * 4, s);
    cudaMemsetAsync(a.inptr, 0, ((size_t)a.n + 2) * 4, s);
    // digit widths: at most RX_MAX_BITS each, as even as possible, >= 2 passes
    int P = (a.nbits + RX_MAX_BITS - 1) / RX_MAX_BITS, widths[8];
    for (int i = 0; i < P; ++i) widths[i] = a.nbits / P + (i < a.nbits % P ? 1 : 0);
    if (P == 1) {
        widths[0] = (a.nbits + 1) / 2;
        widths[1] = a.nbits / 2;
        P = 2;
    }
    uint64_t *bufs[2] = {a.bufA, a.bufB};
    const uint64_t *in = a.ekey;
    int cur = 0, shift = 32;
    for (int p = 0; p < P; ++p) {
        const bool last = p + 1 == P;
        ItemSource src;
        if (p == 0 && a.kept) {
            src = ItemSource{ItemSource::ORIENT, a.kept, 0, a.m_sampled_dev, a.deg, 0, 0};
        } else if (p == 0) {
            src = ItemSource{ItemSource::SAMPLE_ORIENT, a.ekey, a.m, nullptr, a.deg, a.seed_mix, a.thr};
            src.bv = a.bv;
        } else {
            src = ItemSource{ItemSource::PLAIN, in, 0, a.m_sampled_dev, nullptr, 0, 0};
        }
        uint64_t *out = bufs[cur];
        InListArgs il{a.inptr, nullptr, a.n};
        if (last) {
            // padded columns in colp, the in-lists in the output buffer (the
            // input buffer is still being read)
            *col = a.colp;
            *inlist = reinterpret_cast<uint32_t *>(out);
            il.inlist = *inlist;
        }
        radix_pass(src, a.m, shift, widths[p], a.hist, a.scan, p == 0 ? a.rowptr : nullptr, last ? nullptr : out,
                   last ? *col : nullptr, last ? &il : nullptr, s, last ? a.ptrp : nullptr);
        if (p == 0) {
            // out-degrees are complete: pad offsets and in-list offsets for
            // the last pass
            k_row_counts<<<grid_for((uint64_t)a.n + 1, 256, 152 * 8), 256, 0, s>>>(a.rowptr, a.deg, a.n, a.ptrp,
                                                                                   a.inptr);
            note_launch();
            scan_excl_u32(a.ptrp, (uint64_t)a.n + 1, nullptr, a.scan, s);
            scan_excl_u32(a.inptr + 1, (uint64_t)a.n + 1, nullptr, a.scan, s);
        }
        in = out;
        cur ^= 1;
        shift += widths[p];
    }
    scan_excl_u32(a.rowptr, (uint64_t)a.n + 1, nullptr, a.scan, s);
    k_pad_finish<<<grid_for((uint64_t)a.n + 1, 256, 152 * 8), 256, 0, s>>>(a.rowptr, a.n, a.ptrp, a.colp);
    note_launch();
}

}  // namespace tcg
