// Data-movement primitives of libtc: device-wide exclusive scan, stable LSD
// radix passes over 64-bit items (graph creation: canonical order and rank
// order), and the canonicalisation of raw edge lists.
#include "kernels.h"

namespace tcg {

// ======================================================================
// Exclusive scan (reduce -> spine -> downsweep), 4096 elements per block.
// ======================================================================

constexpr int SC_THREADS = 1024;
constexpr int SC_ITEMS = SC_CHUNK / SC_THREADS;  // 4

template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_scan_reduce(const T *__restrict__ a, uint64_t len,
                                                            T *__restrict__ part)
{
    __shared__ T wt[33];
    const uint64_t base = (uint64_t)blockIdx.x * SC_CHUNK;
    T s = 0;
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
template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_scan_spine(T *part, uint64_t nparts, T *total_out)
{
    __shared__ T wt[33];
    T carry = 0;
    for (uint64_t base = 0; base < nparts; base += SC_THREADS) {
        uint64_t i = base + threadIdx.x;
        T x = i < nparts ? part[i] : T(0);
        T tot;
        T ex = block_excl_scan(x, wt, &tot);
        if (i < nparts) part[i] = carry + ex;
        carry += tot;
    }
    if (threadIdx.x == 0 && total_out) *total_out = carry;
}

template <typename T>
__global__ void __launch_bounds__(SC_THREADS) k_scan_down(T *a, uint64_t len, const T *__restrict__ part)
{
    __shared__ T wt[33];
    const uint64_t base = (uint64_t)blockIdx.x * SC_CHUNK;
    T carry = part[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        uint64_t i = base + (uint64_t)j * SC_THREADS + threadIdx.x;
        T x = i < len ? a[i] : T(0);
        T tot;
        T ex = block_excl_scan(x, wt, &tot);
        if (i < len) a[i] = carry + ex;
        carry += tot;
    }
}

// Two arrays scanned together: (a << 32 | b) per element, so that one pass
// scans both (the sums of b stay below 2^32).
__global__ void __launch_bounds__(SC_THREADS) k_scan2_reduce(const uint32_t *__restrict__ a,
                                                             const uint32_t *__restrict__ b, uint64_t len,
                                                             unsigned long long *__restrict__ part)
{
    __shared__ unsigned long long wt[33];
    const uint64_t base = (uint64_t)blockIdx.x * SC_CHUNK;
    unsigned long long s = 0;
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * SC_THREADS + threadIdx.x;
        if (i < len) s += ((unsigned long long)a[i] << 32) | b[i];
    }
    s = block_sum(s, wt);
    if (threadIdx.x == 0) part[blockIdx.x] = s;
}

__global__ void __launch_bounds__(SC_THREADS) k_scan2_spine(unsigned long long *part, uint64_t nparts)
{
    __shared__ unsigned long long wt[33];
    unsigned long long carry = 0;
    for (uint64_t base = 0; base < nparts; base += SC_THREADS) {
        const uint64_t i = base + threadIdx.x;
        const unsigned long long x = i < nparts ? part[i] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan(x, wt, &tot);
        if (i < nparts) part[i] = carry + ex;
        carry += tot;
    }
}

__global__ void __launch_bounds__(SC_THREADS) k_scan2_down(uint32_t *a, uint32_t *b, uint64_t len,
                                                           const unsigned long long *__restrict__ part)
{
    __shared__ unsigned long long wt[33];
    const uint64_t base = (uint64_t)blockIdx.x * SC_CHUNK;
    unsigned long long carry = part[blockIdx.x];
#pragma unroll
    for (int j = 0; j < SC_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * SC_THREADS + threadIdx.x;
        const unsigned long long x = i < len ? ((unsigned long long)a[i] << 32) | b[i] : 0ull;
        unsigned long long tot;
        const unsigned long long ex = carry + block_excl_scan(x, wt, &tot);
        if (i < len) {
            a[i] = (uint32_t)(ex >> 32);
            b[i] = (uint32_t)ex;
        }
        carry += tot;
    }
}

uint64_t scan_scratch_elems(uint64_t len) { return 2 * (ceil_div(len, SC_CHUNK) + 1); }

void scan_excl_pair(uint32_t *a, uint32_t *b, uint64_t len, uint32_t *scratch, cudaStream_t s)
{
    if (len == 0) return;
    const uint64_t nb = ceil_div(len, SC_CHUNK);
    unsigned long long *part = reinterpret_cast<unsigned long long *>(scratch);
    k_scan2_reduce<<<(unsigned)nb, SC_THREADS, 0, s>>>(a, b, len, part); note_launch();
    k_scan2_spine<<<1, SC_THREADS, 0, s>>>(part, nb); note_launch();
    k_scan2_down<<<(unsigned)nb, SC_THREADS, 0, s>>>(a, b, len, part); note_launch();
}

void scan_excl_u32(uint32_t *a, uint64_t len, uint32_t *total, uint32_t *scratch, cudaStream_t s)
{
    if (len == 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(uint32_t), s);
        return;
    }
    const uint64_t nb = ceil_div(len, SC_CHUNK);
    k_scan_reduce<uint32_t><<<(unsigned)nb, SC_THREADS, 0, s>>>(a, len, scratch); note_launch();
    k_scan_spine<uint32_t><<<1, SC_THREADS, 0, s>>>(scratch, nb, total); note_launch();
    k_scan_down<uint32_t><<<(unsigned)nb, SC_THREADS, 0, s>>>(a, len, scratch); note_launch();
}

void scan_excl_u64(unsigned long long *a, uint64_t len, unsigned long long *total, unsigned long long *scratch,
                   cudaStream_t s)
{
    if (len == 0) {
        if (total) cudaMemsetAsync(total, 0, sizeof(unsigned long long), s);
        return;
    }
    const uint64_t nb = ceil_div(len, SC_CHUNK);
    k_scan_reduce<unsigned long long><<<(unsigned)nb, SC_THREADS, 0, s>>>(a, len, scratch); note_launch();
    k_scan_spine<unsigned long long><<<1, SC_THREADS, 0, s>>>(scratch, nb, total); note_launch();
    k_scan_down<unsigned long long><<<(unsigned)nb, SC_THREADS, 0, s>>>(a, len, scratch); note_launch();
}

// ======================================================================
// Stable LSD radix pass.
// ======================================================================

// Per-tile digit counts (per-warp shared histograms, summed at the end).
__global__ void __launch_bounds__(RX_THREADS) k_radix_count(const uint64_t *__restrict__ in, uint64_t n, int shift,
                                                            int width, uint32_t *__restrict__ hist, uint32_t ntiles)
{
    constexpr int NW = RX_THREADS / 32;
    __shared__ uint32_t cnt[NW][RX_BINS];
    const uint32_t tile = blockIdx.x;
    const int nb = 1 << width;
    const unsigned warp = threadIdx.x >> 5;
    for (int i = threadIdx.x; i < NW * RX_BINS; i += RX_THREADS) (&cnt[0][0])[i] = 0;
    __syncthreads();
    const uint64_t base = (uint64_t)tile * RX_TILE;
    const uint32_t mask = (uint32_t)nb - 1;
    for (int j = 0; j < RX_ITEMS; ++j) {
        const uint64_t i = base + (uint64_t)j * RX_THREADS + threadIdx.x;
        if (i < n) atomicAdd(&cnt[warp][(uint32_t)(ld_stream_u64(in + i) >> shift) & mask], 1u);
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
// consecutive positions.
__global__ void __launch_bounds__(RX_THREADS) k_radix_scatter(const uint64_t *__restrict__ in, uint64_t n, int shift,
                                                              int width, const uint32_t *__restrict__ offs,
                                                              uint32_t ntiles, uint64_t *__restrict__ out)
{
    constexpr int NW = RX_THREADS / 32;
    static_assert(RX_BINS == RX_THREADS, "one digit per thread in the tile scan");
    __shared__ uint64_t s_items[RX_TILE];
    __shared__ uint32_t whist[NW][RX_BINS];
    __shared__ uint32_t tstart[RX_BINS];  // first local position of each digit in the sorted tile
    __shared__ uint32_t tbase[RX_BINS];   // global position of each digit's run
    __shared__ uint32_t wt[33];
    const uint32_t tile = blockIdx.x;
    const uint64_t base = (uint64_t)tile * RX_TILE;
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
        items[j] = i < n ? ld_stream_u64(in + i) : 0;
        packed[j] = i < n ? 0u : 0xffffffffu;
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
    uint32_t count;  // items of the tile
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
    for (uint32_t i = threadIdx.x; i < count; i += RX_THREADS) {
        const uint64_t item = s_items[i];
        const uint32_t d = (uint32_t)(item >> shift) & mask;
        out[tbase[d] + (i - tstart[d])] = item;
    }
}

void radix_pass(const uint64_t *in, uint64_t n, int shift, int width, uint32_t *hist, uint32_t *scan_scratch,
                uint64_t *out, cudaStream_t s)
{
    const uint64_t ntiles = ceil_div(n, RX_TILE);
    if (ntiles == 0) return;
    k_radix_count<<<(unsigned)ntiles, RX_THREADS, 0, s>>>(in, n, shift, width, hist, (uint32_t)ntiles); note_launch();
    scan_excl_u32(hist, ntiles << width, nullptr, scan_scratch, s);
    k_radix_scatter<<<(unsigned)ntiles, RX_THREADS, 0, s>>>(in, n, shift, width, hist, (uint32_t)ntiles, out);
    note_launch();
}

// ======================================================================
// Canonicalisation of raw pairs (graph creation).
// ======================================================================

// pairs may be device memory or pinned host memory mapped into the device's
// address space (read once, one pair per lane; its predecessor comes from
// the next lower lane).  With deg, also the degree of every endpoint of a
// valid pair (one atomic per run of a lower endpoint in a warp): the full
// degrees when the list turns out canonical.
template <bool ALIGNED8>
__global__ void k_canon_keys(const uint32_t *__restrict__ pairs, uint64_t m_in, uint32_t n,
                             uint64_t *__restrict__ keys, DevState *st, uint32_t *__restrict__ deg)
{
    unsigned bad = 0, unsorted = 0;
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < m_in; base += stride) {
        const uint64_t i = base + lane;
        uint2 e = make_uint2(0, 0);
        if (i < m_in)
            e = ALIGNED8 ? reinterpret_cast<const uint2 *>(pairs)[i] : make_uint2(pairs[2 * i], pairs[2 * i + 1]);
        uint2 q = make_uint2(__shfl_up_sync(FULL, e.x, 1), __shfl_up_sync(FULL, e.y, 1));
        if (lane == 0 && i > 0 && i < m_in) q = make_uint2(pairs[2 * i - 2], pairs[2 * i - 1]);
        if (deg) {
            const bool ok = i < m_in && e.x < n && e.y < n && e.x != e.y;
            const uint32_t u = ok ? min(e.x, e.y) : 0xffffffffu;
            const unsigned peers = __match_any_sync(FULL, u);
            if (ok) {
                if (lane == (unsigned)(__ffs(peers) - 1)) atomicAdd(deg + u, (unsigned)__popc(peers));
                atomicAdd(deg + max(e.x, e.y), 1u);
            }
        }
        if (i >= m_in) continue;
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
            if (!(q.x < e.x || (q.x == e.x && q.y < e.y))) unsorted++;
        }
    }
    if (__any_sync(FULL, bad) && lane_id() == 0) atomicOr(&st->err, ERR_ENDPOINT);
    unsorted = warp_sum(unsorted);
    if (unsorted && lane_id() == 0) atomicAdd(&st->unsorted, unsorted);
}

void canon_keys(const uint32_t *pairs, uint64_t m_in, uint32_t n, uint64_t *keys, DevState *st, cudaStream_t s,
                uint32_t *deg)
{
    if (m_in == 0) return;
    const uint64_t blocks = std::min<uint64_t>(ceil_div(m_in, 256), 152ull * 16);
    if ((reinterpret_cast<uintptr_t>(pairs) & 7u) == 0)
        k_canon_keys<true><<<(unsigned)blocks, 256, 0, s>>>(pairs, m_in, n, keys, st, deg);
    else
        k_canon_keys<false><<<(unsigned)blocks, 256, 0, s>>>(pairs, m_in, n, keys, st, deg);
    note_launch();
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


