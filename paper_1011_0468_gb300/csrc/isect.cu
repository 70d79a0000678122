// Counting kernels of libtc, part 2: the exact triangle counts of the light
// and heavy classes (Section 3.2) on the degree-oriented CSR.
//
// Every kept edge is directed from the endpoint of lower (deg_p, id) to the
// higher one, so each triangle {a, b, c} with rank(a) < rank(b) < rank(c) is
// seen exactly once: for the pair (a -> b) as the common out-neighbour c of
// a and b.  Light vertices have lower degree than heavy ones, so a triangle
// has a light vertex iff its lowest vertex a is light.
//
// A pair (a -> b) is resolved by the endpoint with the LONGER out-list, the
// "owner": its list is put into a shared-memory hash set and the shorter
// list is streamed through it, so each pair reads min(d+(a), d+(b))
// elements:
//   owner x, partner v in N+(x) with d+(v) <= d+(x)  (triangle class of x)
//   owner x, partner u in in-list(x), d+(u) < d+(x)  (triangle class of u)
//
// Work items are (segment << 32 | owner); a segment is a run of the owner's
// partner sequence (its d+(x) out-neighbours, then its in-list).  Owners
// are bucketed by d+(x), which sizes their hash set: 2..256 (one warp per
// item), 257..1024 (one block, static table), > 1024 (one block, dynamic
// table, or a binary search of the sorted row when even that is too
// small).  Owners with d+ < 2 close no triangle.
#include "kernels.h"

namespace tcg {

constexpr uint32_t SEG_B = 2048;     // largest partners per block item (IsectConfig::seg_b)
constexpr uint32_t WARP_MAX = 256;   // largest warp-owner out-degree (IsectConfig::warp_max)
constexpr uint32_t MID_MAX = 1024;
constexpr uint32_t EMPTY = 0xffffffffu;
constexpr uint32_t GRAB = 8;  // warp items taken per work-cursor atomic

// warp + mid items <= owners + (m_p + in-list entries) / SEG_MIN, for any
// schedule
static uint64_t wm_capacity(uint32_t n, uint64_t m) { return (uint64_t)n + 2 * m / SEG_MIN + 64; }

uint64_t items_capacity(uint32_t n, uint64_t m)
{
    // large items (d+ > MID_MAX, at most m / MID_MAX owners) after the rest
    return wm_capacity(n, m) + m / MID_MAX + 2 * m / 256 + 64;
}

__device__ __forceinline__ uint32_t bucket_of(uint32_t d, uint32_t warp_max)
{
    return d <= warp_max ? 0u : (d <= MID_MAX ? 1u : 2u);
}

// Item layout: owner in bits 0..31; single graph: segment in bits 32..63;
// batch union: segment in bits 32..47 and the owner's graph in bits 48..63.
__device__ __forceinline__ uint64_t make_item(uint32_t x, uint32_t seg, uint32_t g, bool batch)
{
    return batch ? (((uint64_t)g << 48) | ((uint64_t)seg << 32) | x) : (((uint64_t)seg << 32) | x);
}

__device__ __forceinline__ void split_item(uint64_t item, bool batch, uint32_t &x, uint32_t &seg, uint32_t &g)
{
    x = (uint32_t)item;
    seg = batch ? (uint32_t)((item >> 32) & 0xffffu) : (uint32_t)(item >> 32);
    g = batch ? (uint32_t)(item >> 48) : 0u;
}

__global__ void k_items(const uint32_t *__restrict__ rowptr, const uint32_t *__restrict__ inptr, uint32_t n,
                        uint64_t *__restrict__ items, uint64_t wm_cap, uint64_t cap, DevState *st, BatchView bv,
                        IsectConfig cfg)
{
    const bool batch = bv.k != 0;
    const unsigned lane = lane_id();
    const uint64_t wstride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < n; base += wstride) {
        const uint64_t x = base + lane;
        uint32_t d = 0, np = 0;
        if (x < n) {
            d = rowptr[x + 1] - rowptr[x];
            if (d >= 2) np = d + (inptr[x + 1] - inptr[x]);
        }
        const uint32_t gx = batch ? find_part_warp(bv.voff, bv.k, (uint32_t)(x < n ? x : n - 1)) : 0u;
        const uint32_t b = bucket_of(d, cfg.warp_max), seg = b == 0 ? cfg.seg_w : cfg.seg_b;
        uint32_t nseg = (np + seg - 1) / seg;
        if (batch && nseg > 0x10000u) {  // segment index must fit 16 bits
            atomicOr(&st->err, ERR_OVERFLOW);
            nseg = 0x10000u;
        }
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
                    items[pos] = make_item((uint32_t)x, s, gx, batch);
                else
                    atomicOr(&st->err, ERR_OVERFLOW);
            }
        }
    }
}

void build_items(const CountBuffers &b, cudaStream_t s)
{
    const uint64_t wm = wm_capacity(b.n, b.m);
    k_items<<<grid_for(b.n, 256, 152 * 8), 256, 0, s>>>(b.rowptr, b.inptr, b.n, b.items, wm, b.items_cap, b.st,
                                                          b.bv, b.cfg);
    note_launch();
}

// ======================================================================
// Shared-memory hash set of an out-list: open addressing with linear
// probing, at most a quarter full, so a probe sequence meets an empty slot
// after ~1.4 slots on average.  Both loops are bounded by the table size.
// ======================================================================

__device__ __forceinline__ uint32_t tab_hash(uint32_t y, uint32_t shift) { return (y * 0x9e3779b1u) >> shift; }

__device__ __forceinline__ void tab_insert(uint32_t *tab, uint32_t mask, uint32_t shift, uint32_t y)
{
    uint32_t h = tab_hash(y, shift);
    for (uint32_t it = 0; it <= mask; ++it) {
        const uint32_t prev = atomicCAS(tab + h, EMPTY, y);
        if (prev == EMPTY || prev == y) return;
        h = (h + 1) & mask;
    }
}

struct HashSet {
    const uint32_t *tab;
    uint32_t mask, shift;
    __device__ __forceinline__ bool contains(uint32_t y) const
    {
        uint32_t h = tab_hash(y, shift);
        uint32_t k = tab[h];
        for (uint32_t it = 0; k != y && k != EMPTY && it < mask; ++it) {
            h = (h + 1) & mask;
            k = tab[h];
        }
        return k == y;
    }
};

// Fallback for rows whose hash set does not fit on chip: binary search of
// the sorted row in global memory.
struct SortedRow {
    const uint32_t *a;
    uint32_t len;
    __device__ __forceinline__ bool contains(uint32_t w) const
    {
        uint32_t lo = 0, hi = len;
        while (lo < hi) {
            const uint32_t mid = (lo + hi) >> 1;
            if (__ldg(a + mid) < w) lo = mid + 1; else hi = mid;
        }
        return lo < len && __ldg(a + lo) == w;
    }
};

struct Tally {
    unsigned long long light = 0, heavy = 0, table = 0, stream = 0, partners = 0;
};

// Batch unions: move this warp's class counts into graph g's counters.
__device__ __forceinline__ void flush_graph_counts(Tally &t, const BatchView &bv, uint32_t g)
{
    const unsigned long long l = warp_sum(t.light), h = warp_sum(t.heavy);
    if (lane_id() == 0) {
        if (l) atomicAdd(bv.t_light + g, l);
        if (h) atomicAdd(bv.t_heavy + g, h);
    }
    t.light = t.heavy = 0;
}

__device__ __forceinline__ void flush_tally(const Tally &t, unsigned long long *red /* 33 */, DevState *st)
{
    const unsigned long long v[5] = {t.light, t.heavy, t.table, t.stream, t.partners};
    unsigned long long *dst[5] = {&st->t_light, &st->t_heavy, &st->src_elems, &st->nbr_elems, &st->partners};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        const unsigned long long s = block_sum(v[i], red);
        if (threadIdx.x == 0 && s) atomicAdd(dst[i], s);
    }
}

// Partner y of owner x: where its out-list starts, how many elements to
// stream (0 when the pair is resolved by the other endpoint, closes no
// triangle, or is heavy-class while the dense tensor path counts that class)
// and the class of the pair's triangles.
__device__ __forceinline__ void partner_of(const uint32_t *__restrict__ rowptr, const uint8_t *__restrict__ heavy,
                                           uint32_t d, uint8_t hx, uint32_t y, bool is_out, bool skip_heavy,
                                           uint32_t &start, uint32_t &len, uint32_t &cls)
{
    const uint32_t yb = rowptr[y], dy = rowptr[y + 1] - yb;
    start = yb;
    if (is_out) {
        len = (dy >= 1 && dy <= d) ? dy : 0u;
        cls = hx;
    } else {
        len = dy >= 2 ? dy : 0u;
        cls = len ? heavy[y] : 0u;
    }
    if (cls && skip_heavy) len = 0;  // the dense tensor path counts this class
}

// Streams the out-lists of up to 32 partners (one per lane: start, len, cls)
// through the owner's set, 32 elements per step.  The partner of element e
// is found in O(1): a bitmask of the partners whose lists start inside the
// current 32-element window, plus the count of those that started before.
// s_beg / s_pre: this warp's 32-entry shared scratch.
template <class Set>
__device__ __forceinline__ void stream_group(const uint32_t *__restrict__ col, const Set &set, uint32_t start,
                                             uint32_t len, uint32_t cls, uint32_t *s_beg, uint32_t *s_pre, Tally &t,
                                             bool account = true)
{
    const unsigned lane = lane_id();
    const unsigned live = __ballot_sync(FULL, len != 0);
    if (!live) return;
    const uint32_t inc = warp_incl_scan(len);
    const uint32_t pre = inc - len;
    const uint32_t W = __shfl_sync(FULL, inc, 31);
    const uint32_t r = __popc(live & lanemask_lt());  // rank among live partners
    const unsigned heavy_bits = __reduce_or_sync(FULL, (len != 0 && cls != 0) ? (1u << r) : 0u);
    if (len) {
        s_beg[r] = start;
        s_pre[r] = pre;
    }
    __syncwarp();
    const unsigned upto = 0xffffffffu >> (31 - lane);  // bits 0..lane
    uint32_t before = 0;  // live partners starting before the window
    for (uint32_t wb = 0; wb < W; wb += 32) {
        const bool here = len != 0 && pre >= wb && pre - wb < 32;
        const unsigned starts = __reduce_or_sync(FULL, here ? (1u << (pre - wb)) : 0u);
        const uint32_t e = wb + lane;
        if (e < W) {
            const uint32_t k = before + __popc(starts & upto) - 1;
            const uint32_t y = __ldg(col + s_beg[k] + (e - s_pre[k]));
            const uint32_t hit = set.contains(y);
            const uint32_t hc = (heavy_bits >> k) & 1u;
            t.heavy += hit & hc;
            t.light += hit & (hc ^ 1u);
        }
        before += __popc(starts);
    }
    if (account && lane == 0) {
        t.stream += W;
        t.partners += __popc(live);
    }
    __syncwarp();
}

// ---------------------------------------------------------------- list streaming

// A partner list of at least LONG_LIST elements is streamed by one warp,
// consecutive lanes on consecutive elements, two elements in flight per lane.
constexpr uint32_t LONG_LIST = 32;

template <class Set>
__device__ __forceinline__ void stream_list(const uint32_t *__restrict__ col, const Set &set, uint32_t beg,
                                            uint32_t len, uint32_t cls, Tally &t)
{
    const unsigned lane = lane_id();
    uint32_t hits = 0;
    uint32_t e = lane;
    for (; e + 32 < len; e += 64) {
        const uint32_t y0 = __ldg(col + beg + e), y1 = __ldg(col + beg + e + 32);
        hits += set.contains(y0);
        hits += set.contains(y1);
    }
    if (e < len) hits += set.contains(__ldg(col + beg + e));
    if (cls) t.heavy += hits; else t.light += hits;
}

// Streams one warp's 32 partners (one per lane): the long lists one after the
// other with the whole warp, the short ones packed through stream_group.
template <class Set>
__device__ __forceinline__ void stream_partners(const uint32_t *__restrict__ col, const Set &set, uint32_t start,
                                                uint32_t len, uint32_t cls, uint32_t *s_beg, uint32_t *s_pre,
                                                Tally &t)
{
    const bool is_long = len >= LONG_LIST;
    if (len) {
        t.stream += len;
        t.partners += 1;
    }
    unsigned lm = __ballot_sync(FULL, is_long);
    while (lm) {
        const int k = __ffs(lm) - 1;
        lm &= lm - 1;
        stream_list(col, set, __shfl_sync(FULL, start, k), __shfl_sync(FULL, len, k), __shfl_sync(FULL, cls, k), t);
    }
    stream_group(col, set, start, is_long ? 0u : len, cls, s_beg, s_pre, t, false);
}

// ---------------------------------------------------------------- warp items

constexpr int PW_THREADS = 256;
constexpr int PW_WARPS = PW_THREADS / 32;
constexpr uint32_t WTAB = 1024;  // per-warp table slots, >= 4 * WARP_MAX

__global__ void __launch_bounds__(PW_THREADS, 5) k_probe_warp(const uint32_t *__restrict__ rowptr,
                                                           const uint32_t *__restrict__ col,
                                                           const uint32_t *__restrict__ inptr,
                                                           const uint32_t *__restrict__ inlist,
                                                           const uint64_t *__restrict__ items, uint64_t wm_cap,
                                                           const uint8_t *__restrict__ heavy, DevState *st,
                                                           BatchView bv, IsectConfig cfg)
{
    __shared__ uint32_t s_tab[PW_WARPS][WTAB];
    __shared__ uint32_t s_pre[PW_WARPS][32];
    __shared__ uint32_t s_beg[PW_WARPS][32];
    __shared__ unsigned long long red[33];
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const uint32_t nitems = (uint32_t)min((unsigned long long)st->nlist[0], (unsigned long long)wm_cap);
    const bool skip_heavy = st->dense != 0;
    uint32_t *tab = s_tab[w];
    const bool batch = bv.k != 0;
    uint32_t cur_g = 0;  // graph whose counts this warp holds (batch)
    Tally t;
    for (;;) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(&st->cursor[0], GRAB);
        first = __shfl_sync(FULL, first, 0);
        if (first >= nitems) break;
        const uint32_t last = min(first + GRAB, nitems);
        for (uint32_t idx = first; idx < last; ++idx) {
            uint32_t x, seg, g;
            split_item(items[idx], batch, x, seg, g);
            if (batch && g != cur_g) {
                flush_graph_counts(t, bv, cur_g);
                cur_g = g;
            }
            const uint32_t beg = rowptr[x], d = rowptr[x + 1] - beg;
            if (d > cfg.warp_max || d > WARP_MAX) {  // cannot happen unless the item list overflowed
                if (lane == 0) atomicOr(&st->err, ERR_OVERFLOW);
                continue;
            }
            const uint8_t hx = heavy[x];
            uint32_t slots = 64;
            while (slots < 4 * d) slots <<= 1;  // <= WTAB since d <= WARP_MAX
            const uint32_t shift = 32 - (31 - __clz(slots));
            const HashSet set{tab, slots - 1, shift};
            for (uint32_t i = lane; i < slots; i += 32) tab[i] = EMPTY;
            __syncwarp();
            for (uint32_t i = lane; i < d; i += 32) tab_insert(tab, slots - 1, shift, __ldg(col + beg + i));
            __syncwarp();
            if (seg == 0 && lane == 0) t.table += d;
            const uint32_t ib = inptr[x], np = d + (inptr[x + 1] - ib);
            const uint32_t p0 = seg * cfg.seg_w, p1 = min(np, p0 + cfg.seg_w);
            for (uint32_t c0 = p0; c0 < p1; c0 += 32) {
                const uint32_t j = c0 + lane;
                uint32_t start = 0, len = 0, cls = 0;
                if (j < p1) {
                    const bool is_out = j < d;
                    const uint32_t y = is_out ? __ldg(col + beg + j) : __ldg(inlist + ib + j - d);
                    partner_of(rowptr, heavy, d, hx, y, is_out, skip_heavy, start, len, cls);
                }
                stream_partners(col, set, start, len, cls, s_beg[w], s_pre[w], t);
            }
            __syncwarp();  // the table is rewritten by the next item
        }
    }
    if (batch) flush_graph_counts(t, bv, cur_g);
    flush_tally(t, red, st);
}

// ---------------------------------------------------------------- block items

constexpr int PB_THREADS = 256;
constexpr int PB_WARPS = PB_THREADS / 32;
constexpr uint32_t PB_PER_THREAD = SEG_B / PB_THREADS;  // partner slots set up per thread (at most)
constexpr uint32_t MID_TAB = 4096;                      // >= 4 * MID_MAX slots

// One block resolves one item: up to SEG_B partners of one owner.  Partner
// lists of at least 32 elements are streamed by one warp each, consecutive
// lanes on consecutive elements (two in flight per lane); shorter lists are
// packed 32 partners at a time through stream_group.  Warps take long lists
// first, then short groups, from shared counters, so they finish within one
// list of each other.
template <bool DYN>
__global__ void __launch_bounds__(PB_THREADS, 4) k_probe_block(const uint32_t *__restrict__ rowptr,
                                                            const uint32_t *__restrict__ col,
                                                            const uint32_t *__restrict__ inptr,
                                                            const uint32_t *__restrict__ inlist,
                                                            const uint64_t *__restrict__ items, uint64_t wm_cap,
                                                            const uint8_t *__restrict__ heavy, DevState *st,
                                                            uint32_t tab_slots, uint64_t cap, BatchView bv,
                                                            IsectConfig cfg)
{
    extern __shared__ uint32_t s_dyn[];
    __shared__ uint32_t s_static[DYN ? 1 : MID_TAB];
    uint32_t *tab = DYN ? s_dyn : s_static;
    // partners: long lists from the front, short ones from the back
    __shared__ uint32_t s_pbeg[SEG_B];
    __shared__ uint32_t s_plen[SEG_B];
    __shared__ uint8_t s_pcls[SEG_B];
    __shared__ uint32_t s_pre[PB_WARPS][32];
    __shared__ uint32_t s_beg[PB_WARPS][32];
    __shared__ uint32_t wt[33];
    __shared__ unsigned long long red[33];
    __shared__ uint32_t s_idx, s_next_long, s_next_short;
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const uint32_t b = DYN ? 2 : 1;
    const uint32_t nitems =
        (uint32_t)min((unsigned long long)st->nlist[b], (unsigned long long)(DYN ? cap - wm_cap : wm_cap));
    const bool skip_heavy = st->dense != 0;
    Tally t;
    for (;;) {
        if (threadIdx.x == 0) {
            s_idx = atomicAdd(&st->cursor[b], 1u);
            s_next_long = 0;
            s_next_short = 0;
        }
        __syncthreads();
        const uint32_t idx = s_idx;
        if (idx >= nitems) break;
        uint32_t x, seg, g;
        split_item(DYN ? items[wm_cap + idx] : items[wm_cap - 1 - idx], bv.k != 0, x, seg, g);
        const uint32_t beg = rowptr[x], d = rowptr[x + 1] - beg;
        const uint8_t hx = heavy[x];
        // a power of two >= 4 d slots, when that fits
        uint32_t slots = 64;
        while (slots < 4 * d && slots < (1u << 30)) slots <<= 1;
        const bool use_tab = slots <= tab_slots && (uint64_t)slots >= 4ull * d;
        const uint32_t shift = 32 - (31 - __clz(slots));
        if (use_tab) {
            for (uint32_t i = threadIdx.x; i < slots; i += PB_THREADS) tab[i] = EMPTY;
            __syncthreads();
            for (uint32_t i = threadIdx.x; i < d; i += PB_THREADS) tab_insert(tab, slots - 1, shift, __ldg(col + beg + i));
        }
        if (seg == 0 && threadIdx.x == 0) t.table += d;
        const uint32_t ib = inptr[x], np = d + (inptr[x + 1] - ib);
        const uint32_t p0 = seg * cfg.seg_b, p1 = min(np, p0 + cfg.seg_b);
        const uint32_t per = cfg.seg_b / PB_THREADS;  // <= PB_PER_THREAD
        // set up this thread's PB_PER_THREAD consecutive partners
        uint32_t pstart[PB_PER_THREAD], plen[PB_PER_THREAD], pcls[PB_PER_THREAD];
        uint32_t mine = 0;  // (long count << 16) | short count
#pragma unroll
        for (uint32_t q = 0; q < PB_PER_THREAD; ++q) {
            const uint32_t j = p0 + threadIdx.x * per + q;
            pstart[q] = 0;
            plen[q] = 0;
            pcls[q] = 0;
            if (q < per && j < p1) {
                const bool is_out = j < d;
                const uint32_t y = is_out ? __ldg(col + beg + j) : __ldg(inlist + ib + j - d);
                partner_of(rowptr, heavy, d, hx, y, is_out, skip_heavy, pstart[q], plen[q], pcls[q]);
            }
            if (plen[q]) {
                mine += plen[q] >= LONG_LIST ? (1u << 16) : 1u;
                t.stream += plen[q];
                t.partners += 1;
            }
        }
        uint32_t tot;
        const uint32_t ex = block_excl_scan(mine, wt, &tot);  // also orders the set build
        uint32_t rl = ex >> 16, rs = SEG_B - 1 - (ex & 0xffffu);
#pragma unroll
        for (uint32_t q = 0; q < PB_PER_THREAD; ++q) {
            if (plen[q]) {
                const uint32_t r = plen[q] >= LONG_LIST ? rl++ : rs--;
                s_pbeg[r] = pstart[q];
                s_plen[r] = plen[q];
                s_pcls[r] = (uint8_t)pcls[q];
            }
        }
        const uint32_t nlong = tot >> 16, nshort = tot & 0xffffu;
        const uint32_t nshort_groups = (nshort + 31) / 32;
        __syncthreads();  // partners and set are complete
        for (;;) {
            uint32_t k = 0;
            if (lane == 0) k = atomicAdd(&s_next_long, 1u);
            k = __shfl_sync(FULL, k, 0);
            if (k >= nlong) break;
            if (use_tab)
                stream_list(col, HashSet{tab, slots - 1, shift}, s_pbeg[k], s_plen[k], s_pcls[k], t);
            else
                stream_list(col, SortedRow{col + beg, d}, s_pbeg[k], s_plen[k], s_pcls[k], t);
        }
        for (;;) {
            uint32_t g = 0;
            if (lane == 0) g = atomicAdd(&s_next_short, 1u);
            g = __shfl_sync(FULL, g, 0);
            if (g >= nshort_groups) break;
            const uint32_t i = g * 32 + lane;
            uint32_t start = 0, len = 0, cls = 0;
            if (i < nshort) {
                const uint32_t r = SEG_B - 1 - i;
                start = s_pbeg[r];
                len = s_plen[r];
                cls = s_pcls[r];
            }
            if (use_tab)
                stream_group(col, HashSet{tab, slots - 1, shift}, start, len, cls, s_beg[w], s_pre[w], t, false);
            else
                stream_group(col, SortedRow{col + beg, d}, start, len, cls, s_beg[w], s_pre[w], t, false);
        }
        if (bv.k != 0) flush_graph_counts(t, bv, g);
        __syncthreads();  // every warp is done with this owner
    }
    flush_tally(t, red, st);
}

// Static + dynamic shared memory of the large-owner kernel must fit the
// function's opt-in limit, which starts at 48 KiB in every process: raise it
// once per process and device to the largest size requested so far.
void intersect_prepare(int dyn_smem_bytes)
{
    static int set_bytes[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    if (dev < 0 || dev >= 64 || dyn_smem_bytes > set_bytes[dev]) {
        if (cudaFuncSetAttribute(k_probe_block<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn_smem_bytes) ==
                cudaSuccess &&
            dev >= 0 && dev < 64)
            set_bytes[dev] = dyn_smem_bytes;
    }
}

void intersect(const CountBuffers &b, int dyn_smem_bytes, cudaStream_t s)
{
    if (b.n == 0 || b.m == 0) return;
    const uint64_t wm = wm_capacity(b.n, b.m);
    k_probe_warp<<<152 * 8, PW_THREADS, 0, s>>>(b.rowptr, b.col, b.inptr, b.inlist, b.items, wm, b.heavy, b.st,
                                                b.bv, b.cfg);
    note_launch();
    k_probe_block<false><<<152 * 8, PB_THREADS, 0, s>>>(b.rowptr, b.col, b.inptr, b.inlist, b.items, wm, b.heavy,
                                                         b.st, MID_TAB, b.items_cap, b.bv, b.cfg);
    note_launch();
    intersect_prepare(dyn_smem_bytes);
    k_probe_block<true><<<152, PB_THREADS, dyn_smem_bytes, s>>>(b.rowptr, b.col, b.inptr, b.inlist, b.items, wm,
                                                                b.heavy, b.st, (uint32_t)(dyn_smem_bytes / 4),
                                                                b.items_cap, b.bv, b.cfg);
    note_launch();
}

}  // namespace tcg
