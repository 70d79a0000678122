// Device-side helpers shared by the libtc kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "tc.h"

namespace tcg {

constexpr unsigned FULL = 0xffffffffu;
constexpr int NUM_SMS_HINT = 152;

// ---------------------------------------------------------------- errors
// Bits of DevState::err raised by kernels; the host maps them to statuses.
enum : unsigned {
    ERR_ENDPOINT = 1u,   // an input endpoint >= n
    ERR_TIMEOUT = 2u,    // a bounded wait gave up
    ERR_OVERFLOW = 4u,   // an internal capacity was exceeded
};

// Per-graph device state: counters written by the kernels of one count.
struct DevState {
    unsigned long long m_sampled;  // kept edges m_p
    unsigned long long t_light;    // light-class triangles
    unsigned long long t_heavy;    // heavy-class triangles
    unsigned int n_heavy;          // heavy vertices
    unsigned int err;              // ERR_* bits
    unsigned int nlist[4];         // sizes of the source buckets
    unsigned int cursor[4];        // dynamic work cursors (one per kernel)
    unsigned long long src_elems;  // sum of d+(u) over intersected sources
    unsigned long long nbr_elems;  // list elements streamed through the tables
    unsigned long long partners;   // (owner, partner) pairs processed
    unsigned long long heavy_kchunks;  // 64-wide K chunks multiplied by the heavy contraction
    unsigned int dense;            // 1: the heavy class is counted by the dense tensor path
    unsigned int h_listed;         // heavy vertices listed for the dense path
    unsigned long long m_canon;    // canonical edges (create only)
    unsigned int unsorted;         // create: adjacent pairs out of order
    unsigned int light_lim;        // 1 + the largest light vertex with an edge (0: none); ids above are heavy
    unsigned long long t_core;     // triangles inside the dense core (all three ids >= the core base)
    unsigned int core_on;          // 1: the core block counts the triangles inside the core
    unsigned int heavy_below;      // heavy vertices below the core base
    unsigned int cursor_core;      // work cursor of the core contraction
    unsigned int cand_lo;          // single graph: rank ids below this cannot be heavy (see k_sample_keep)
    unsigned int cand_all;         // 1: the sample fell below the bound, every in-degree was counted
};

// A batch of independent graphs laid out as one disjoint union: graph g owns
// edges [eoff[g], eoff[g+1]) of the union's canonical key array and vertices
// [voff[g], voff[g+1]).  Keys hold union vertex ids; the sampling hash uses
// the graph-local key, so every graph draws the sample it would draw alone.
// k == 0 means a single graph (all per-graph arrays unused).
struct BatchView {
    uint32_t k = 0;
    const uint64_t *eoff = nullptr;      // [k + 1]
    const uint32_t *voff = nullptr;      // [k + 1]
    const uint64_t *thr = nullptr;       // [k] floor(p * 2^53)
    const uint64_t *seed_mix = nullptr;  // [k] splitmix64(seed)
    unsigned long long *m_p = nullptr;   // [k] kept edges
    unsigned int *n_heavy = nullptr;     // [k]
    unsigned long long *t_light = nullptr;
    unsigned long long *t_heavy = nullptr;
};

// Largest g in [0, k) with off[g] <= i (off non-decreasing, off[0] = 0).
template <typename T>
__device__ __forceinline__ uint32_t find_part(const T *off, uint32_t k, T i)
{
    uint32_t lo = 0, hi = k;
    while (hi - lo > 1) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(off + mid) <= i) lo = mid; else hi = mid;
    }
    return lo;
}

// find_part for 32 non-decreasing indices held by the lanes of a full warp:
// two searches for the end lanes, and per-lane searches only when the warp
// straddles a part boundary.
template <typename T>
__device__ __forceinline__ uint32_t find_part_warp(const T *off, uint32_t k, T i)
{
    const unsigned lane = threadIdx.x & 31u;
    uint32_t g = 0;
    if (lane == 0 || lane == 31) g = find_part(off, k, i);
    const uint32_t g0 = __shfl_sync(0xffffffffu, g, 0), g1 = __shfl_sync(0xffffffffu, g, 31);
    if (g0 == g1) return g0;
    return g0 + find_part(off + g0, g1 - g0 + 1, i);
}

// The same from a known part g_start <= the answer for lane 0 (parts are
// walked forward from it): for consecutive items that advance slowly.
template <typename T>
__device__ __forceinline__ uint32_t find_part_warp_from(const T *off, uint32_t k, T i, uint32_t g_start)
{
    const unsigned lane = threadIdx.x & 31u;
    uint32_t g = g_start;
    if (lane == 0 || lane == 31)
        while (g + 1 < k && off[g + 1] <= i) ++g;
    const uint32_t g0 = __shfl_sync(0xffffffffu, g, 0), g1 = __shfl_sync(0xffffffffu, g, 31);
    if (g0 == g1) return g0;
    return g0 + find_part(off + g0, g1 - g0 + 1, i);
}

// ---------------------------------------------------------------- splitmix64
// Steele, Lea and Flood's splitmix64 in the form Vigna published:
// z = x + golden gamma, then two xor-shift-multiply rounds and a final
// xor-shift, all modulo 2^64.
__host__ __device__ __forceinline__ uint64_t splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

// Section 3.1 edge sparsification as a counter-based draw: the canonical
// edge key (u << 32 | v), u < v, is kept iff its hash, reduced to 53 bits,
// falls below floor(p * 2^53).  seed_mix = splitmix64(seed).
__device__ __forceinline__ bool keep_edge(uint64_t key, uint64_t seed_mix, uint64_t thr)
{
    return (splitmix64(key ^ seed_mix) >> 11) < thr;
}

// ---------------------------------------------------------------- warp / block
__device__ __forceinline__ unsigned lane_id() { return threadIdx.x & 31u; }

__device__ __forceinline__ unsigned lanemask_lt()
{
    unsigned r;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(r));
    return r;
}

template <typename T>
__device__ __forceinline__ T warp_incl_scan(T x)
{
    const unsigned lane = lane_id();
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        T y = __shfl_up_sync(FULL, x, o);
        if (lane >= (unsigned)o) x += y;
    }
    return x;
}

template <typename T>
__device__ __forceinline__ T warp_sum(T x)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(FULL, x, o);
    return x;
}

// Exclusive scan of one value per thread across the block (blockDim.x a
// multiple of 32).  `warp_tot` is shared scratch of 33 entries.  Returns the
// exclusive prefix; *total receives the block sum.  Contains __syncthreads.
template <typename T>
__device__ __forceinline__ T block_excl_scan(T x, T *warp_tot, T *total)
{
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    T inc = warp_incl_scan(x);
    if (lane == 31) warp_tot[warp] = inc;
    __syncthreads();
    if (warp == 0) {
        T t = lane < nw ? warp_tot[lane] : T(0);
        T ti = warp_incl_scan(t);
        if (lane < nw) warp_tot[lane] = ti - t;
        if (lane == nw - 1) warp_tot[32] = ti;
    }
    __syncthreads();
    T res = inc - x + warp_tot[warp];
    *total = warp_tot[32];
    __syncthreads();
    return res;
}

template <typename T>
__device__ __forceinline__ T block_sum(T x, T *warp_tot)
{
    const unsigned lane = lane_id(), warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    x = warp_sum(x);
    if (lane == 0) warp_tot[warp] = x;
    __syncthreads();
    T r = T(0);
    if (warp == 0) {
        r = lane < nw ? warp_tot[lane] : T(0);
        r = warp_sum(r);
    }
    __syncthreads();
    return r;  // valid in thread 0 (and all of warp 0)
}

__device__ __forceinline__ uint64_t ld_stream_u64(const uint64_t *p)
{
    uint64_t r;
    asm volatile("ld.global.nc.L1::no_allocate.u64 %0, [%1];" : "=l"(r) : "l"(p));
    return r;
}

__device__ __forceinline__ ulonglong2 ld_stream_u64x2(const ulonglong2 *p)
{
    ulonglong2 r;
    asm volatile("ld.global.nc.L1::no_allocate.v2.u64 {%0, %1}, [%2];"
                 : "=l"(r.x), "=l"(r.y)
                 : "l"(p));
    return r;
}

}  // namespace tcg
