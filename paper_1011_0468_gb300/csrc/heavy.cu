// The heavy class on the tensor cores.
//
// Heavy vertices (deg_p^2 > m_p, Section 3.2) number at most 2 m_p^(1/2).
// Ordered by id (the graph is stored in rank order, csr.cu, and every kept
// edge points from the lower id to the higher) they give a strictly
// upper-triangular 0/1 matrix U, U[i][k] = 1 for every kept edge i -> k
// between heavy vertices.  Each all-heavy triangle a < b < c is exactly one
// term of
//     T_H = sum_{i < k} U[i][k] * (U U)[i][k],
// the matrix-product route of Alon, Yuster and Zwick that the paper builds
// on.  U and U^T are packed as fp8 e4m3 0/1 matrices (one byte per entry)
// and the product runs on tcgen05 (kind::f8f6f4, FP32 accumulation in tensor
// memory), exact because 0 and 1 are exact in e4m3 and every partial sum is
// an integer no larger than h < 2^24.  Only output tiles on or above the
// diagonal, and only the j-tiles between them, are multiplied; the epilogue
// masks D = U U with U and sums.
//
// sm_103a has no INT8 tcgen05 MMA (.kind::i8 is rejected for this target);
// fp8 has the same operand bytes and twice the bf16 rate.
#include <cuda.h>

#include "kernels.h"

namespace tcg {

// ======================================================================
// Ranking and packing
// ======================================================================

// Lists the heavy vertices.
__global__ void k_heavy_list(const uint8_t *__restrict__ heavy, uint32_t n, uint32_t *__restrict__ hlist,
                             uint32_t hlist_cap, DevState *st)
{
    const unsigned lane = lane_id();
    const uint64_t wstride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += wstride) {
        const uint64_t u = base + lane;
        const bool f = u < n && heavy[u];
        const unsigned mask = __ballot_sync(FULL, f);
        uint32_t off = 0;
        if (lane == 0 && mask) off = atomicAdd(&st->h_listed, (unsigned)__popc(mask));
        off = __shfl_sync(FULL, off, 0);
        if (f) {
            const uint32_t pos = off + __popc(mask & lanemask_lt());
            if (pos < hlist_cap) hlist[pos] = (uint32_t)u;
        }
    }
}

// Whether the dense path runs (2 <= h <= hcap, all listed) and whether the
// core block counts the top ranks (every heavy vertex inside the core:
// heavy_below, counted by the partition).  Decided right after the
// partition, so that the compaction already leaves out the pairs these
// blocks count.
__global__ void k_heavy_decide(uint32_t hcap, uint32_t hlist_cap, bool core, DevState *st)
{
    const uint32_t h = st->n_heavy;
    const bool dense = hcap != 0 && h >= 2 && h <= hcap && h <= hlist_cap;
    st->dense = dense ? 1u : 0u;
    st->core_on = (core && dense && st->heavy_below == 0) ? 1u : 0u;
}

void heavy_decide(const CountBuffers &b, const HeavyBuffers &hb, const CoreBuffers *core, cudaStream_t s)
{
    if (hb.hcap == 0 || hb.hlist_cap == 0 || b.n == 0) return;  // no dense block: DevState::dense stays 0
    k_heavy_decide<<<1, 1, 0, s>>>(hb.hcap, hb.hlist_cap, core && core->hb.hcap != 0, b.st);
    note_launch();
}

constexpr int HR_THREADS = 256;

// Dense index of each heavy vertex = the number of heavy vertices with a
// smaller id (O(h^2) comparisons, h <= 2 m_p^(1/2)), so that every edge
// between heavy vertices lands above the diagonal (only when the dense path
// runs).
__global__ void __launch_bounds__(HR_THREADS) k_heavy_rank(const uint32_t *__restrict__ hlist,
                                                           uint32_t *__restrict__ hidx, uint32_t hcap,
                                                           uint32_t hlist_cap, DevState *st)
{
    __shared__ unsigned long long s_key[HR_THREADS];
    const uint32_t h = st->n_heavy;
    const bool dense = st->dense != 0;  // k_heavy_decide
    if (!dense || blockIdx.x * HR_THREADS >= h) return;  // uniform per block
    const uint32_t i = blockIdx.x * HR_THREADS + threadIdx.x;
    unsigned long long mine = ~0ull;
    uint32_t v = 0;
    if (i < h) {
        v = hlist[i];
        mine = v;
    }
    uint32_t rank = 0;
    for (uint32_t j0 = 0; j0 < h; j0 += HR_THREADS) {
        const uint32_t j = j0 + threadIdx.x;
        s_key[threadIdx.x] = j < h ? (unsigned long long)hlist[j] : ~0ull;
        __syncthreads();
        const uint32_t cnt = min((uint32_t)HR_THREADS, h - j0);
        for (uint32_t q = 0; q < cnt; ++q) rank += s_key[q] < mine;
        __syncthreads();
    }
    if (i < h) hidx[v] = rank;
}

// Zero the used corner [0, hp) x [0, hp) of U and U^T, hp = h rounded up to 128.
__global__ void k_heavy_clear(uint8_t *__restrict__ U, uint8_t *__restrict__ UT, uint32_t hcap, DevState *st)
{
    if (!st->dense) return;
    const uint32_t hp = (st->n_heavy + 127) & ~127u;
    const uint64_t per_row = hp / 16;  // uint4 per row
    const uint64_t total = (uint64_t)hp * per_row;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total; t += stride) {
        const uint64_t r = t / per_row, c = t % per_row;
        reinterpret_cast<uint4 *>(U + r * hcap)[c] = make_uint4(0, 0, 0, 0);
        reinterpret_cast<uint4 *>(UT + r * hcap)[c] = make_uint4(0, 0, 0, 0);
    }
}

// One warp per heavy source: U[idx(v)][idx(w)] = U^T[idx(w)][idx(v)] = 1
// for every heavy out-neighbour w.
__global__ void k_heavy_pack(const uint32_t *__restrict__ ptrp, const uint32_t *__restrict__ col,
                             const uint8_t *__restrict__ heavy, const uint32_t *__restrict__ hlist,
                             const uint32_t *__restrict__ hidx, uint8_t *__restrict__ U, uint8_t *__restrict__ UT,
                             uint32_t hcap, DevState *st)
{
    if (!st->dense) return;
    const uint32_t h = st->n_heavy;
    const unsigned lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    constexpr uint8_t ONE = TC_ONE;
    for (uint32_t i = gw; i < h; i += nw) {
        const uint32_t v = hlist[i], r = hidx[v];
        const PaddedRow row = padded_row(ptrp, v);
        for (uint32_t q = row.beg + lane; q < row.beg + row.d; q += 32) {
            const uint32_t w = col[q];
            if (!heavy[w]) continue;  // an edge to a light vertex: not in U
            const uint32_t c = hidx[w];
            if (r >= hcap || c >= hcap) continue;
            U[(uint64_t)r * hcap + c] = ONE;
            UT[(uint64_t)c * hcap + r] = ONE;
        }
    }
}

// One warp per core row v (ids base .. base + hcap - 1 that exist): U[v - base][w - base] =
// U^T[w - base][v - base] = 1 for every out-neighbour w (all inside the core).
__global__ void k_core_pack(const uint32_t *__restrict__ ptrp, const uint32_t *__restrict__ col, uint32_t n,
                            uint32_t base, uint8_t *__restrict__ U, uint8_t *__restrict__ UT, uint32_t hcap,
                            DevState *st)
{
    if (!st->core_on) return;
    const unsigned lane = lane_id();
    const uint32_t gw = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, nw = (gridDim.x * blockDim.x) >> 5;
    constexpr uint8_t ONE = TC_ONE;
    for (uint32_t v = base + gw; v < n; v += nw) {
        const PaddedRow row = padded_row(ptrp, v);
        const uint32_t r = v - base;
        for (uint32_t q = row.beg + lane; q < row.beg + row.d; q += 32) {
            const uint32_t c = col[q] - base;  // col[q] > v >= base
            if (r >= hcap || c >= hcap) continue;
            U[(uint64_t)r * hcap + c] = ONE;
            UT[(uint64_t)c * hcap + r] = ONE;
        }
    }
}

// ======================================================================
// tcgen05 contraction
// ======================================================================

// Roles: warp 0 TMA producer, warp 1 TMEM owner and MMA issuer, warps 2-5
// epilogue (each reads the TMEM lane quarter warp % 4).
constexpr int TC_THREADS = 192;
constexpr int TC_STAGES = 4;
constexpr uint32_t TC_TILE = 128;                       // M = 128 rows of U (a row panel)
constexpr uint32_t TC_N = 256;                          // N = 256 columns (a column panel)
constexpr uint32_t TC_KC = 128;                         // fp8 elements per K chunk = one 128-B row
constexpr uint32_t TC_A_BYTES = TC_TILE * TC_KC;        // 16 KiB
constexpr uint32_t TC_B_BYTES = TC_N * TC_KC;           // 32 KiB
constexpr uint32_t TC_STAGE_BYTES = TC_A_BYTES + TC_B_BYTES;
constexpr uint32_t TC_SMEM = TC_STAGES * TC_STAGE_BYTES + 1024;  // + alignment slack
constexpr uint32_t TC_ACCS = 2;                         // accumulators: a tile's epilogue overlaps the next MMAs
constexpr uint32_t TC_TMEM_COLS = TC_ACCS * TC_N;       // 512: all of TMEM, one CTA per SM
constexpr uint32_t TC_RING = 4;                         // tile hand-over slots
constexpr uint32_t TC_NO_TILE = 0xffffffffu;
constexpr unsigned long long TC_WAIT_NS = 2000000000ull;  // bounded waits: 2 s

__device__ __forceinline__ uint32_t smem_u32(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long globaltimer()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}

__device__ __forceinline__ void mbar_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait until the phase of the given parity has completed; false after
// limit_ns (TC_WAIT_NS in the kernels) without completion.
__device__ __forceinline__ bool mbar_wait(uint64_t *bar, uint32_t parity, unsigned long long limit_ns = TC_WAIT_NS)
{
    if (mbar_try_wait(bar, parity)) return true;
    const unsigned long long t0 = globaltimer();
    for (;;) {
        if (mbar_try_wait(bar, parity)) return true;
        if (globaltimer() - t0 > limit_ns) return false;
    }
}

// The kernels' bounded wait on a barrier that nothing arrives at (phase 0
// of a fresh barrier with one expected arrival never completes): it must
// give up after limit_ns and say so (*gave_up = 1).
__global__ void k_wait_check(unsigned long long limit_ns, unsigned *gave_up)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        *gave_up = mbar_wait(&bar, 0u, limit_ns) ? 0u : 1u;
    }
}

__device__ __forceinline__ void tma_load_2d(uint32_t dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
            dst),
        "l"(map), "r"(x), "r"(y), "r"(smem_u32(bar))
        : "memory");
}

// Shared-memory matrix descriptor of a K-major operand tile stored with the
// 128-byte swizzle (rows of 128 B, 8-row groups 1024 B apart).
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr >> 4) & 0x3fffu);  // start address
    d |= (uint64_t)1 << 16;                   // leading byte offset (unused for this layout)
    d |= (uint64_t)(1024 >> 4) << 32;         // stride byte offset: 8-row groups
    d |= (uint64_t)1 << 46;                   // descriptor version for tcgen05
    d |= (uint64_t)2 << 61;                   // 128-byte swizzle
    return d;
}

// Instruction descriptor: D f32 (bits 4-5 = 1), A and B e4m3 (type fields at
// bits 7-9 and 10-12 = 0), both K-major, N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t TC_IDESC = (1u << 4) | ((TC_N >> 3) << 17) | ((TC_TILE >> 4) << 24);

// D (+)= A B^T over 32 fp8 elements of K (32 bytes of each operand row).
__device__ __forceinline__ void mma_fp8(uint32_t tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n}\n" ::"r"(
            tmem),
        "l"(a), "l"(b), "r"(TC_IDESC), "r"(accumulate)
        : "memory");
}

__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
                 : "memory");
}

__device__ __forceinline__ void mbar_arrive(uint64_t *bar)
{
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(bar)) : "memory");
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// 32 consecutive f32 columns of this warp's 32 TMEM lanes (no wait).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&r)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16,%17,%18,%19,"
        "%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]),
          "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]),
          "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]),
          "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
}

// Output tiles: row panel I (128 rows) by column panel P (256 columns),
// every pair with 2P + 1 >= I (the others lie below the diagonal, where U is
// zero); tile (I, P) multiplies the j-chunks [I, min(2P + 2, R)).  Tiles are
// handed out in groups of TC_GI row panels by TC_GP column panels, so that
// the CTAs running at the same time read the same few operand panels (a
// group's operands fit in L2).  Groups go column group by column group from
// the right (the longest tiles first), down each column group; inside a
// group, column panels from the right, row panels from the top.
constexpr int TC_GI = 16, TC_GP = 8;
constexpr int TC_MAX_GROUPS = 1024;  // order <= 65536: 32 row groups x 32 column groups

struct TileGrid {
    int R, C;    // row panels (of 128) and column panels (of 256)
    int Rg, Cg;  // row groups and column groups
    __device__ __forceinline__ uint32_t group_tiles(int gi, int gp) const
    {
        const int i0 = gi * TC_GI, i1 = min(i0 + TC_GI, R);
        uint32_t n = 0;
        for (int P = gp * TC_GP; P < min(gp * TC_GP + TC_GP, C); ++P) n += (uint32_t)max(0, min(i1, 2 * P + 2) - i0);
        return n;
    }
    // pre[k] = tiles of the groups before group k (k = 0 .. Rg Cg), one warp
    __device__ void prefix(uint32_t *pre, unsigned lane) const
    {
        const int G = Rg * Cg;
        uint32_t carry = 0;
        for (int k0 = 0; k0 < G; k0 += 32) {
            const int k = k0 + (int)lane;
            uint32_t x = k < G ? group_tiles(k % Rg, Cg - 1 - k / Rg) : 0u;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const uint32_t y = __shfl_up_sync(FULL, x, d);
                if ((int)lane >= d) x += y;
            }
            if (k < G) pre[k + 1] = carry + x;
            carry += __shfl_sync(FULL, x, 31);
        }
        if (lane == 0) pre[0] = 0;
    }
    // t-th tile (t < pre[Rg Cg]), packed as I << 16 | P
    __device__ uint32_t tile(const uint32_t *pre, uint32_t t) const
    {
        int lo = 0, hi = Rg * Cg;  // pre[lo] <= t < pre[hi]
        while (hi - lo > 1) {
            const int mid = (lo + hi) >> 1;
            if (pre[mid] <= t) lo = mid;
            else hi = mid;
        }
        t -= pre[lo];
        const int gi = lo % Rg, gp = Cg - 1 - lo / Rg;
        const int i0 = gi * TC_GI, i1 = min(i0 + TC_GI, R);
        for (int P = min(gp * TC_GP + TC_GP, C) - 1; P >= gp * TC_GP; --P) {
            const uint32_t cnt = (uint32_t)max(0, min(i1, 2 * P + 2) - i0);
            if (t < cnt) return (uint32_t)(i0 + (int)t) << 16 | (uint32_t)P;
            t -= cnt;
        }
        return TC_NO_TILE;
    }
};

// One contraction: which matrix order, which tile cursor and which output
// counter (the heavy block and the core block run the same kernel).
struct DenseJob {
    const unsigned *enable;      // runs iff *enable != 0
    const unsigned *h_dev;       // matrix order on the device, or NULL: h_host
    uint32_t h_host;
    unsigned *cursor;            // tile work cursor (zero on entry)
    unsigned long long *out;     // += sum_{i<k} U_ik (U U)_ik
};

// Persistent, warp-specialised: the producer takes tiles from the cursor
// (heaviest first) and hands each one to the MMA warp and the epilogue
// warps through a small ring; the MMA warp accumulates tile n in TMEM
// accumulator n % 2 while the epilogue warps read tile n - 1 from the other
// one.  Every wait is bounded: a stalled barrier sets ERR_TIMEOUT and the
// roles leave their loops; the CTA then waits (bounded) for its own
// outstanding copies and MMAs before it frees TMEM.
__global__ void __launch_bounds__(TC_THREADS, 1) k_heavy_tc(const __grid_constant__ CUtensorMap mapA,
                                                            const __grid_constant__ CUtensorMap mapB,
                                                            const uint8_t *__restrict__ U, uint32_t hcap,
                                                            DenseJob job, DevState *st)
{
    extern __shared__ uint8_t smem_raw[];
    __shared__ __align__(8) uint64_t full[TC_STAGES], empty[TC_STAGES];
    __shared__ __align__(8) uint64_t tfull[TC_RING], tempty[TC_RING], afull[TC_ACCS], aempty[TC_ACCS], drain;
    __shared__ uint32_t s_tile[TC_RING], s_pre[TC_MAX_GROUPS + 1];
    __shared__ uint32_t s_tmem, s_issued, s_consumed;
    __shared__ volatile uint32_t s_abort;
    if (!*job.enable) return;  // uniform: written before this launch
    const uint32_t h = job.h_dev ? *job.h_dev : job.h_host;
    const uint32_t hp = (h + TC_TILE - 1) / TC_TILE * TC_TILE;
    const int R = (int)(hp / TC_TILE), C = (R + 1) / 2;
    const TileGrid grid{R, C, (R + TC_GI - 1) / TC_GI, (C + TC_GP - 1) / TC_GP};
    if (grid.Rg * grid.Cg > TC_MAX_GROUPS) {  // an order above 65536 (the library never asks for one)
        if (threadIdx.x == 0) atomicOr(&st->err, ERR_OVERFLOW);
        return;
    }
    const unsigned warp = threadIdx.x >> 5, lane = lane_id();
    const uint32_t base = (smem_u32(smem_raw) + 1023u) & ~1023u;

    if (warp == 1) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(&s_tmem)),
                     "n"(TC_TMEM_COLS)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (threadIdx.x == 0) {
        for (int s = 0; s < TC_STAGES; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (uint32_t r = 0; r < TC_RING; ++r) {
            mbar_init(&tfull[r], 1);
            mbar_init(&tempty[r], 1 + 4);  // the MMA thread and the four epilogue warps
        }
        for (uint32_t a = 0; a < TC_ACCS; ++a) {
            mbar_init(&afull[a], 1);
            mbar_init(&aempty[a], 4);
        }
        mbar_init(&drain, 1);
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        s_abort = 0;
        s_issued = 0;
        s_consumed = 0;
    }
    if (warp == 0) grid.prefix(s_pre, lane);
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    const uint32_t tmem = s_tmem;

    if (warp == 0) {
        if (lane == 0) {  // TMA producer
            const uint32_t ntiles = s_pre[grid.Rg * grid.Cg];
            uint32_t it = 0;
            for (uint32_t n = 0;; ++n) {
                const uint32_t r = n % TC_RING, rph = (n / TC_RING) & 1u;
                if (!mbar_wait(&tempty[r], rph ^ 1u)) {
                    atomicOr(&st->err, ERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                const uint32_t t = s_abort ? ntiles : atomicAdd(job.cursor, 1u);
                const uint32_t tile = t < ntiles ? grid.tile(s_pre, t) : TC_NO_TILE;
                s_tile[r] = tile;
                mbar_arrive(&tfull[r]);
                if (tile == TC_NO_TILE) break;
                const uint32_t I = tile >> 16, P = tile & 0xffffu, c1 = min(2 * P + 2, (uint32_t)grid.R);
                bool ok = true;
                for (uint32_t c = I; c < c1; ++c, ++it) {
                    const uint32_t s = it % TC_STAGES, ph = (it / TC_STAGES) & 1u;
                    if (!mbar_wait(&empty[s], ph ^ 1u)) {
                        ok = false;
                        break;
                    }
                    mbar_expect_tx(&full[s], TC_STAGE_BYTES);
                    const uint32_t a = base + s * TC_STAGE_BYTES;
                    tma_load_2d(a, &mapA, &full[s], (int)(c * TC_KC), (int)(I * TC_TILE));
                    tma_load_2d(a + TC_A_BYTES, &mapB, &full[s], (int)(c * TC_KC), (int)(P * TC_N));
                }
                if (!ok) {
                    atomicOr(&st->err, ERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
            }
            s_issued = it;
        }
    } else if (warp == 1) {
        if (lane == 0) {  // MMA issuer
            uint32_t it = 0;
            unsigned long long kunits = 0;
            bool issued = false;
            for (uint32_t n = 0;; ++n) {
                const uint32_t r = n % TC_RING, rph = (n / TC_RING) & 1u;
                if (!mbar_wait(&tfull[r], rph)) {
                    atomicOr(&st->err, ERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                const uint32_t tile = s_tile[r];
                mbar_arrive(&tempty[r]);
                if (tile == TC_NO_TILE) break;
                const uint32_t I = tile >> 16, P = tile & 0xffffu, c1 = min(2 * P + 2, (uint32_t)grid.R);
                const uint32_t acc = n % TC_ACCS, aph = (n / TC_ACCS) & 1u;
                if (!mbar_wait(&aempty[acc], aph ^ 1u)) {  // the epilogue has read this accumulator
                    atomicOr(&st->err, ERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                const uint32_t d = tmem + acc * TC_N;
                bool ok = true;
                for (uint32_t c = I; c < c1; ++c, ++it) {
                    const uint32_t s = it % TC_STAGES, ph = (it / TC_STAGES) & 1u;
                    if (!mbar_wait(&full[s], ph)) {
                        ok = false;
                        break;
                    }
                    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
                    const uint32_t a = base + s * TC_STAGE_BYTES;
                    const uint64_t da = sw128_desc(a), db = sw128_desc(a + TC_A_BYTES);
#pragma unroll
                    for (uint32_t kk = 0; kk < TC_KC / 32; ++kk)  // 32 fp8 = 32 B per MMA
                        mma_fp8(d, da + 2 * kk, db + 2 * kk, (c > I || kk > 0) ? 1u : 0u);
                    issued = true;
                    mma_commit(&empty[s]);  // frees the stage once these MMAs have read it
                }
                if (!ok) {
                    atomicOr(&st->err, ERR_TIMEOUT);
                    s_abort = 1;
                    break;
                }
                mma_commit(&afull[acc]);  // accumulator complete
                kunits += (unsigned long long)(c1 - I) * (TC_N / TC_TILE) * (TC_KC / 64);  // 128x128x64 units
            }
            s_consumed = it;
            if (issued) {  // every MMA of this CTA has finished before TMEM is freed
                mma_commit(&drain);
                if (!mbar_wait(&drain, 0u)) atomicOr(&st->err, ERR_TIMEOUT);
            }
            if (kunits) atomicAdd(&st->heavy_kchunks, kunits);
        }
    } else {
        // epilogue: rows 32 (warp % 4) .. + 31 of each tile, D masked by U
        const uint32_t quarter = warp & 3u;
        unsigned long long total = 0;
        for (uint32_t n = 0;; ++n) {
            const uint32_t r = n % TC_RING, rph = (n / TC_RING) & 1u;
            if (!__all_sync(FULL, mbar_wait(&tfull[r], rph))) {
                if (lane == 0) atomicOr(&st->err, ERR_TIMEOUT);
                s_abort = 1;
                break;
            }
            const uint32_t tile = s_tile[r];
            __syncwarp();
            if (lane == 0) mbar_arrive(&tempty[r]);
            if (tile == TC_NO_TILE) break;
            const uint32_t I = tile >> 16, P = tile & 0xffffu;
            const uint32_t acc = n % TC_ACCS, aph = (n / TC_ACCS) & 1u;
            if (!__all_sync(FULL, mbar_wait(&afull[acc], aph))) {
                if (lane == 0) atomicOr(&st->err, ERR_TIMEOUT);
                s_abort = 1;
                break;
            }
            asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
            const uint32_t row = I * TC_TILE + quarter * 32 + lane;  // < hp <= hcap
            const uint8_t *urow = U + (uint64_t)row * hcap + (uint64_t)P * TC_N;
            const uint32_t ncols = min(TC_N, hp - P * TC_N);  // 128 or 256: columns below hp only
            const uint32_t taddr = tmem + ((quarter * 32u) << 16) + acc * TC_N;
            float fsum = 0.f;  // integers up to 2^24, exact: at most 256 terms of at most h <= 65536
#pragma unroll 1
            for (uint32_t q = 0; q < ncols / 32; ++q) {
                const uint4 *m4 = reinterpret_cast<const uint4 *>(urow + q * 32);
                const uint4 m0 = m4[0], m1 = m4[1];
                const bool any = (m0.x | m0.y | m0.z | m0.w | m1.x | m1.y | m1.z | m1.w) != 0;
                if (!__any_sync(FULL, any)) continue;  // warp-uniform: the load below is .sync.aligned
                uint32_t v[32];
                tmem_ld32(taddr + q * 32, v);
                tmem_wait_ld();
                const uint32_t w[8] = {m0.x, m0.y, m0.z, m0.w, m1.x, m1.y, m1.z, m1.w};
#pragma unroll
                for (int e = 0; e < 32; ++e)
                    if ((w[e >> 2] >> ((e & 3) * 8)) & 0xffu) fsum += __uint_as_float(v[e]);
            }
            total += (unsigned long long)fsum;
            asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
            __syncwarp();
            if (lane == 0) mbar_arrive(&aempty[acc]);  // the MMA warp may overwrite it
        }
        total = warp_sum(total);
        if (lane == 0 && total) atomicAdd(job.out, total);
    }
    __syncwarp();
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    if (threadIdx.x == 0 && s_abort) {
        // copies issued that no MMA consumed must land before the CTA exits
        for (uint32_t i = s_consumed; i < s_issued; ++i) mbar_wait(&full[i % TC_STAGES], (i / TC_STAGES) & 1u);
    }
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (warp == 1) {
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "n"(TC_TMEM_COLS)
                     : "memory");
    }
}

// ======================================================================
// Host side
// ======================================================================

typedef CUresult (*EncodeTiledFn)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                  const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn()
{
    static EncodeTiledFn fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
        cudaGetLastError();
    }
    return fn;
}

bool heavy_make_maps(HeavyBuffers &hb)
{
    EncodeTiledFn enc = encode_fn();
    if (!enc || !hb.U || !hb.UT || hb.hcap == 0) return false;
    const cuuint64_t dims[2] = {hb.hcap, hb.hcap};
    const cuuint64_t strides[1] = {(cuuint64_t)hb.hcap};
    const cuuint32_t boxes[2][2] = {{TC_KC, TC_TILE}, {TC_KC, TC_N}};  // A: 128 rows of U, B: 256 rows of U^T
    const cuuint32_t estr[2] = {1, 1};
    CUtensorMap *maps[2] = {reinterpret_cast<CUtensorMap *>(hb.mapA), reinterpret_cast<CUtensorMap *>(hb.mapB)};
    void *bufs[2] = {hb.U, hb.UT};
    for (int i = 0; i < 2; ++i) {
        if (enc(maps[i], CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, bufs[i], dims, strides, boxes[i], estr,
                CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) != CUDA_SUCCESS)
            return false;
    }
    return true;
}

void heavy_prepare(const CountBuffers &b, const HeavyBuffers &hb, const CoreBuffers *core, cudaStream_t s)
{
    if (hb.hcap == 0 || hb.hlist_cap == 0 || b.n == 0) return;  // no dense block: DevState::dense stays 0
    const bool with_core = core && core->hb.hcap != 0;
    k_heavy_list<<<grid_for(b.n, 256, 152 * 8), 256, 0, s>>>(b.heavy, b.n, hb.hlist, hb.hlist_cap, b.st);
    note_launch();
    k_heavy_rank<<<(unsigned)ceil_div(hb.hlist_cap, HR_THREADS), HR_THREADS, 0, s>>>(hb.hlist, hb.hidx, hb.hcap,
                                                                                   hb.hlist_cap, b.st);
    note_launch();
    k_heavy_clear<<<152 * 8, 256, 0, s>>>(hb.U, hb.UT, hb.hcap, b.st);
    note_launch();
    k_heavy_pack<<<152 * 4, 256, 0, s>>>(b.ptrp, b.col, b.heavy, hb.hlist, hb.hidx, hb.U, hb.UT, hb.hcap, b.st);
    note_launch();
    if (with_core) {  // the rows of the core this count uses (its order may be below hcap)
        const uint64_t order = std::min<uint64_t>(core->hb.hcap, b.n - core->base);
        const uint64_t bytes = order * core->hb.hcap;
        cudaMemsetAsync(core->hb.U, 0, bytes, s);
        cudaMemsetAsync(core->hb.UT, 0, bytes, s);
        k_core_pack<<<152 * 8, 256, 0, s>>>(b.ptrp, b.col, b.n, core->base, core->hb.U, core->hb.UT, core->hb.hcap,
                                            b.st);
        note_launch();
    }
}

int wait_check(uint32_t limit_us)
{
    unsigned *flag = nullptr, host = 2;
    if (cudaMalloc(&flag, sizeof(unsigned)) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    k_wait_check<<<1, 32>>>((unsigned long long)limit_us * 1000ull, flag);
    note_launch();
    const bool ok = cudaMemcpy(&host, flag, sizeof(unsigned), cudaMemcpyDeviceToHost) == cudaSuccess;
    cudaFree(flag);
    if (!ok) {
        cudaGetLastError();
        return -1;
    }
    return (int)host;
}

void heavy_contract(const CountBuffers &b, const HeavyBuffers &hb, const CoreBuffers *core, cudaStream_t s)
{
    cudaFuncSetAttribute(k_heavy_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, TC_SMEM);
    const CUtensorMap *ma = reinterpret_cast<const CUtensorMap *>(hb.mapA);
    const CUtensorMap *mb = reinterpret_cast<const CUtensorMap *>(hb.mapB);
    const DenseJob heavy_job{&b.st->dense, &b.st->n_heavy, 0, &b.st->cursor[3], &b.st->t_heavy};
    k_heavy_tc<<<152, TC_THREADS, TC_SMEM, s>>>(*ma, *mb, hb.U, hb.hcap, heavy_job, b.st);
    note_launch();
    if (core && core->hb.hcap != 0) {
        const CUtensorMap *ca = reinterpret_cast<const CUtensorMap *>(core->hb.mapA);
        const CUtensorMap *cb = reinterpret_cast<const CUtensorMap *>(core->hb.mapB);
        const uint32_t order = std::min<uint32_t>(core->hb.hcap, b.n - core->base);
        const DenseJob core_job{&b.st->core_on, nullptr, order, &b.st->cursor_core, &b.st->t_core};
        k_heavy_tc<<<152, TC_THREADS, TC_SMEM, s>>>(*ca, *cb, core->hb.U, core->hb.hcap, core_job, b.st);
        note_launch();
    }
}

}  // namespace tcg
