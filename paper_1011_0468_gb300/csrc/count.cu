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
// Owner work items.
//
// Every oriented pair (a -> b) closes |N+(a) n N+(b)| triangles.  The pair
// is handled by the endpoint with the LONGER out-list as the "owner": its
// list is put into a shared-memory hash table and the shorter list is
// streamed through it, so each pair reads min(d+(a), d+(b)) list elements.
//   owner x, partner v in N+(x) with d+(v) <= d+(x)   (class of x)
//   owner x, partner u in in-list(x): d+(u) < d+(x)   (class of u)
// The class of a triangle is the class of its lowest vertex, which is the
// source of the pair: x in the first case, u in the second.
//
// An item is (segment << 32 | owner); segment s covers partners
// [s * SEG, (s + 1) * SEG) of the owner's partner sequence (its d+(x)
// out-neighbours, then its in-list).  Owners are bucketed by d+(x), which
// sizes their table: 2..32 (one warp), 33..1024 (one block, static table),
// > 1024 (one block, dynamic table).  Owners with d+ < 2 close nothing.
// ======================================================================

constexpr uint32_t SEG = 256;
constexpr uint32_t WARP_MAX = 32, MID_MAX = 1024;
constexpr uint32_t EMPTY = 0xffffffffu;

uint64_t items_capacity(uint32_t n, uint64_t m)
{
    // warp + mid items: <= owners + (m_p + in-list) / SEG; large items after
    const uint64_t wm = (uint64_t)n + 2 * m / SEG + 64;
    const uint64_t large = m / MID_MAX + 2 * m / SEG + 64;
    return wm + large;
}

static uint64_t wm_capacity(uint32_t n, uint64_t m) { return (uint64_t)n + 2 * m / SEG + 64; }

__device__ __forceinline__ uint32_t bucket_of(uint32_t d) { return d <= WARP_MAX ? 0u : (d <= MID_MAX ? 1u : 2u); }

__global__ void k_items(const uint32_t *__restrict__ rowptr, const uint32_t *__restrict__ inptr, uint32_t n,
                        uint64_t *__restrict__ items, uint64_t wm_cap, uint64_t cap, DevState *st)
{
    const unsigned lane = lane_id();
    const uint64_t wstride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += wstride) {
        const uint64_t x = base + lane;
        uint32_t d = 0, np = 0;
        if (x < n) {
            d = rowptr[x + 1] - rowptr[x];
            if (d >= 2) np = d + (inptr[x + 1] - inptr[x]);
        }
        const uint32_t nseg = (np + SEG - 1) / SEG, b = bucket_of(d);
#pragma unroll
        for (uint32_t bb = 0; bb < 3; ++bb) {
            const uint32_t c = b == bb ? nseg : 0u;
            const uint32_t inc = warp_incl_scan(c);
            uint32_t off = 0;
            if (lane == 31 && inc) off = atomicAdd(&st->nlist[bb], inc);
            off = __shfl_sync(FULL, off, 31) + inc - c;
            for (uint32_t s = 0; s < c; ++s) {
                const uint64_t idx = (uint64_t)off + s;
                const uint64_t pos = bb == 0 ? idx : (bb == 1 ? wm_cap - 1 - idx : wm_cap + idx);
                const bool ok = bb == 2 ? pos < cap : idx < wm_cap;
                if (ok)
                    items[pos] = ((uint64_t)s << 32) | (uint32_t)x;
                else
                    atomicOr(&st->err, ERR_OVERFLOW);
            }
        }
    }
}

void build_items(const CountBuffers &b, cudaStream_t s)
{
    const uint64_t wm = wm_capacity(b.n, b.m);
    k_items<<<grid_for(b.n, 256, 152 * 8), 256, 0, s>>>(b.rowptr, b.inptr, b.n, b.items, wm, b.items_cap, b.st); note_launch();
}

// ======================================================================
// Shared-memory hash set of an out-list (open addressing, linear probing,
// at most half full, so every probe sequence meets an empty slot).
// ======================================================================

__device__ __forceinline__ uint32_t tab_hash(uint32_t y, uint32_t shift) { return (y * 0x9e3779b1u) >> shift; }

// Both loops visit at most every slot once (the table is never more than half
// full, so they normally stop after one or two slots).
__device__ __forceinline__ void tab_insert(uint32_t *tab, uint32_t mask, uint32_t shift, uint32_t y)
{
    uint32_t h = tab_hash(y, shift);
    for (uint32_t it = 0; it <= mask; ++it) {
        const uint32_t prev = atomicCAS(tab + h, EMPTY, y);
        if (prev == EMPTY || prev == y) return;
        h = (h + 1) & mask;
    }
}

__device__ __forceinline__ bool tab_probe(const uint32_t *tab, uint32_t mask, uint32_t shift, uint32_t y)
{
    uint32_t h = tab_hash(y, shift);
    for (uint32_t it = 0; it <= mask; ++it) {
        const uint32_t k = tab[h];
        if (k == y) return true;
        if (k == EMPTY) return false;
        h = (h + 1) & mask;
    }
    return false;
}

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
__device__ __forceinline__ bool sorted_contains(const uint32_t *a, uint32_t len, uint32_t w)
{
    uint32_t lo = 0, hi = len;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (__ldg(a + mid) < w) lo = mid + 1; else hi = mid;
    }
    return lo < len && __ldg(a + lo) == w;
}

struct Tally {
    unsigned long long light = 0, heavy = 0, table = 0, stream = 0, partners = 0;
};

__device__ __forceinline__ void flush_tally(Tally t, unsigned long long *red /* 33 */, DevState *st)
{
    unsigned long long v[5] = {t.light, t.heavy, t.table, t.stream, t.partners};
    unsigned long long *dst[5] = {&st->t_light, &st->t_heavy, &st->src_elems, &st->nbr_elems, &st->partners};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const unsigned long long s = block_sum(v[i], red);
        if (threadIdx.x == 0 && s) atomicAdd(dst[i], s);
    }
}

// Partner j of owner x (j < d: out-neighbour, else in-list entry): the
// start and length of the list to stream and the class of the pair's
// triangles; len = 0 when the pair is handled elsewhere or closes nothing.
__device__ __forceinline__ void partner(const uint32_t *__restrict__ rowptr, const uint32_t *__restrict__ inlist,
                                        const uint8_t *__restrict__ heavy, uint32_t d, uint32_t ib, uint8_t hx,
                                        uint32_t j, uint32_t y, bool is_out, uint32_t &start, uint32_t &len,
                                        uint32_t &cls)
{
    (void)j;
    (void)inlist;
    const uint32_t yb = rowptr[y], dy = rowptr[y + 1] - yb;
    start = yb;
    if (is_out) {
        len = (dy >= 1 && dy <= d) ? dy : 0u;
        cls = hx;
    } else {
        len = dy >= 2 ? dy : 0u;
        cls = len ? heavy[y] : 0u;
    }
    (void)ib;
}

// ---------------------------------------------------------------- warp items

constexpr int PW_THREADS = 256;
constexpr int PW_WARPS = PW_THREADS / 32;
constexpr uint32_t WTAB = 64;  // table slots for d+ <= 32

__global__ void __launch_bounds__(PW_THREADS) k_probe_warp(const uint32_t *__restrict__ rowptr,
                                                           const uint32_t *__restrict__ col,
                                                           const uint32_t *__restrict__ inptr,
                                                           const uint32_t *__restrict__ inlist,
                                                           const uint64_t *__restrict__ items, uint64_t wm_cap,
                                                           const uint8_t *__restrict__ heavy, DevState *st)
{
    __shared__ uint32_t s_tab[PW_WARPS][WTAB];
    __shared__ uint32_t s_pre[PW_WARPS][32];
    __shared__ uint32_t s_beg[PW_WARPS][32];
    __shared__ unsigned long long red[33];
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const uint32_t nitems = (uint32_t)min((unsigned long long)st->nlist[0], (unsigned long long)wm_cap);
    constexpr uint32_t shift = 32 - 6;  // log2(WTAB) = 6
    Tally t;
    for (;;) {
        uint32_t idx = 0;
        if (lane == 0) idx = atomicAdd(&st->cursor[0], 1u);
        idx = __shfl_sync(FULL, idx, 0);
        if (idx >= nitems) break;
        const uint64_t item = items[idx];
        const uint32_t x = (uint32_t)item, seg = (uint32_t)(item >> 32);
        const uint32_t beg = rowptr[x], d = rowptr[x + 1] - beg;
        if (d > WARP_MAX) {  // cannot happen unless the item list overflowed
            if (lane == 0) atomicOr(&st->err, ERR_OVERFLOW);
            continue;
        }
        const uint8_t hx = heavy[x];
        s_tab[w][lane] = EMPTY;
        s_tab[w][lane + 32] = EMPTY;
        __syncwarp();
        uint32_t own = 0;
        if (lane < d) {
            own = col[beg + lane];
            tab_insert(s_tab[w], WTAB - 1, shift, own);
        }
        __syncwarp();
        if (seg == 0) t.table += d;
        const uint32_t ib = inptr[x], np = d + (inptr[x + 1] - ib);
        const uint32_t p0 = seg * SEG, p1 = min(np, p0 + SEG);
        for (uint32_t c0 = p0; c0 < p1; c0 += 32) {
            const uint32_t j = c0 + lane;
            uint32_t start = 0, len = 0, cls = 0;
            if (j < p1) {
                // out-partners only occur in the first chunk (d <= 32), where j == lane
                const bool is_out = j < d;
                const uint32_t y = is_out ? own : inlist[ib + j - d];
                partner(rowptr, inlist, heavy, d, ib, hx, j, y, is_out, start, len, cls);
            }
            const uint32_t inc = warp_incl_scan(len);
            const uint32_t W = __shfl_sync(FULL, inc, 31);
            const unsigned clsmask = __ballot_sync(FULL, cls != 0);
            const unsigned live = __ballot_sync(FULL, len != 0);
            if (lane == 0) t.partners += __popc(live);
            s_pre[w][lane] = inc - len;
            s_beg[w][lane] = start;
            __syncwarp();
            for (uint32_t e = lane; e < W; e += 32) {
                const uint32_t i = seg_of(s_pre[w], 32, e);
                const uint32_t y = col[s_beg[w][i] + (e - s_pre[w][i])];
                if (tab_probe(s_tab[w], WTAB - 1, shift, y)) {
                    if ((clsmask >> i) & 1u) ++t.heavy; else ++t.light;
                }
            }
            if (lane == 0) t.stream += W;
            __syncwarp();
        }
    }
    if (lane != 0) t.table = 0;  // counted once per warp
    flush_tally(t, red, st);
}

// ---------------------------------------------------------------- block items

constexpr int PB_THREADS = 256;
constexpr uint32_t MID_TAB = 2048;  // slots, >= 2 * MID_MAX

template <bool DYN>
__global__ void __launch_bounds__(PB_THREADS) k_probe_block(const uint32_t *__restrict__ rowptr,
                                                            const uint32_t *__restrict__ col,
                                                            const uint32_t *__restrict__ inptr,
                                                            const uint32_t *__restrict__ inlist,
                                                            const uint64_t *__restrict__ items, uint64_t wm_cap,
                                                            const uint8_t *__restrict__ heavy, DevState *st,
                                                            uint32_t tab_slots, uint64_t cap)
{
    extern __shared__ uint32_t s_dyn[];
    __shared__ uint32_t s_static[DYN ? 1 : MID_TAB];
    uint32_t *tab = DYN ? s_dyn : s_static;
    __shared__ uint32_t s_pre[PB_THREADS];
    __shared__ uint32_t s_beg[PB_THREADS];
    __shared__ uint8_t s_cls[PB_THREADS];
    __shared__ uint32_t wt[33];
    __shared__ unsigned long long red[33];
    __shared__ uint32_t s_idx;
    const uint32_t b = DYN ? 2 : 1;
    const uint32_t nitems =
        (uint32_t)min((unsigned long long)st->nlist[b], (unsigned long long)(DYN ? cap - wm_cap : wm_cap));
    Tally t;
    for (;;) {
        if (threadIdx.x == 0) s_idx = atomicAdd(&st->cursor[b], 1u);
        __syncthreads();
        const uint32_t idx = s_idx;
        if (idx >= nitems) break;
        const uint64_t item = DYN ? items[wm_cap + idx] : items[wm_cap - 1 - idx];
        const uint32_t x = (uint32_t)item, seg = (uint32_t)(item >> 32);
        const uint32_t beg = rowptr[x], d = rowptr[x + 1] - beg;
        const uint8_t hx = heavy[x];
        // table size: a power of two >= 2 d; fall back to a binary search of
        // the sorted row when it does not fit
        uint32_t slots = 64;
        while (slots < 2 * d && slots < (1u << 30)) slots <<= 1;
        const bool use_tab = slots <= tab_slots && (uint64_t)slots >= 2ull * d;
        const uint32_t shift = 32 - (31 - __clz(slots));
        if (use_tab) {
            for (uint32_t i = threadIdx.x; i < slots; i += PB_THREADS) tab[i] = EMPTY;
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < d; i += PB_THREADS) tab_insert(tab, slots - 1, shift, col[beg + i]);
        }
        if (seg == 0 && threadIdx.x == 0) t.table += d;
        const uint32_t ib = inptr[x], np = d + (inptr[x + 1] - ib);
        const uint32_t p0 = seg * SEG, p1 = min(np, p0 + SEG);
        const uint32_t j = p0 + threadIdx.x;
        uint32_t start = 0, len = 0, cls = 0;
        if (j < p1) {
            const bool is_out = j < d;
            const uint32_t y = is_out ? col[beg + j] : inlist[ib + j - d];
            partner(rowptr, inlist, heavy, d, ib, hx, j, y, is_out, start, len, cls);
        }
        t.partners += len != 0;
        uint32_t W;
        const uint32_t ex = block_excl_scan(len, wt, &W);  // also orders the table build
        s_pre[threadIdx.x] = ex;
        s_beg[threadIdx.x] = start;
        s_cls[threadIdx.x] = (uint8_t)cls;
        __syncthreads();
        for (uint32_t e = threadIdx.x; e < W; e += PB_THREADS) {
            const uint32_t i = seg_of(s_pre, PB_THREADS, e);
            const uint32_t y = col[s_beg[i] + (e - s_pre[i])];
            const bool hit = use_tab ? tab_probe(tab, slots - 1, shift, y) : sorted_contains(col + beg, d, y);
            if (hit) {
                if (s_cls[i]) ++t.heavy; else ++t.light;
            }
        }
        if (threadIdx.x == 0) t.stream += W;
        __syncthreads();  // s_idx, the table and the chunk arrays are rewritten next
    }
    flush_tally(t, red, st);
}

void intersect(const CountBuffers &b, int dyn_smem_bytes, cudaStream_t s)
{
    if (b.n == 0 || b.m == 0) return;
    const uint64_t wm = wm_capacity(b.n, b.m);
    k_probe_warp<<<152 * 8, PW_THREADS, 0, s>>>(b.rowptr, b.col, b.inptr, b.inlist, b.items, wm, b.heavy, b.st); note_launch();
    k_probe_block<false><<<152 * 6, PB_THREADS, 0, s>>>(b.rowptr, b.col, b.inptr, b.inlist, b.items, wm, b.heavy,
                                                         b.st, MID_TAB, b.items_cap); note_launch();
    if (dyn_smem_bytes > 48 * 1024)
        cudaFuncSetAttribute(k_probe_block<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem_bytes);
    k_probe_block<true><<<152, PB_THREADS, dyn_smem_bytes, s>>>(b.rowptr, b.col, b.inptr, b.inlist, b.items, wm,
                                                                b.heavy, b.st, (uint32_t)(dyn_smem_bytes / 4),
                                                                b.items_cap); note_launch();
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
    for (int i = 0; i < 8; ++i) out->ms[i] = 0.0f;
}

void finalize(const CountBuffers &b, double p, tc_result *out_dev, cudaStream_t s)
{
    k_finalize<<<1, 1, 0, s>>>(b.st, b.m, b.n, p, out_dev); note_launch();
}

}  // namespace tcg
