// Counting kernels of libtc, part 2: the exact triangle counts of the light
// and heavy classes (Section 3.2) on the degree-oriented CSR.
//
// Every kept edge is directed from the endpoint of lower rank (csr.cu), so
// each triangle {a, b, c} with rank(a) < rank(b) < rank(c) is seen exactly
// once: for the pair (a -> b) as the common out-neighbour c of a and b.  A
// triangle is heavy iff all three vertices are heavy; a pair with a light
// endpoint closes light triangles only, and only the (rare) pairs of two
// heavy vertices look at the third vertex (ids at or above
// DevState::light_lim are heavy, the rest are looked up).
//
// A pair (a -> b) is resolved by the endpoint with the LONGER out-list, the
// "owner": its list is put into a shared-memory set (a hash set, or for the
// block kernels a bitmap of its rank window) and the shorter list is
// streamed through it:
//   owner x, partner v in N+(x) with d+(v) <= d+(x): stream N+(v)
//   owner x, partner u in in-list(x), d+(u) < d+(x): stream the part of
//     N+(u) ranked above x (rows are sorted by rank and the in-list entry
//     holds the position of x in N+(u))
// so each pair reads at most min(d+(a), d+(b)) entries.  The compaction
// (csr.cu) hands every pair that can close a triangle to its owner: the
// out-list of x holds its out-partners, the in-list its in-partners.
//
// Work items are (segment << 32 | owner); a segment is a run of the owner's
// partner sequence (its out-list, then its in-list).  Owners are bucketed
// by d+(x), which sizes their set: 2..256 (one warp per item), 257..1024
// (one 128-thread block, 4096-slot table, eight blocks per SM so that one
// block's item setup overlaps the others' streaming), > 1024 (one
// 1024-thread block, larger table, or a binary search of the sorted row
// when even that is too small); the cutoffs and the set of each block
// kernel follow the schedule (IsectConfig).  Owners with d+ < 2 close no
// triangle.  Rows are stored padded to 16 bytes (kernels.h), so the
// partners' lists stream as uint4 chunks.
#include <algorithm>

#include "kernels.h"

namespace tcg {

constexpr uint32_t SEG_B = 512;      // largest partners per mid-owner item (IsectConfig::seg_b is capped here)
constexpr uint32_t SEG_L = 4096;     // largest partners per large-owner item (IsectConfig::seg_l)
constexpr uint32_t WARP_MAX = 256;   // largest warp-owner out-degree (IsectConfig::warp_max)
constexpr uint32_t MID_MAX = 1024;
constexpr uint32_t MID_MIN = 512;    // smallest IsectConfig::mid_max
constexpr uint32_t EMPTY = 0xffffffffu;
constexpr uint32_t GRAB = 8;  // warp items taken per work-cursor atomic (at most 32)
constexpr int NWIN = 2;  // 32-chunk windows in flight per warp step

// warp + mid items <= owners + (m_p + in-list entries) / SEG_MIN, for any
// schedule
static uint64_t wm_capacity(uint32_t n, uint64_t m) { return (uint64_t)n + 2 * m / SEG_MIN + 64; }

uint64_t items_capacity(uint32_t n, uint64_t m)
{
    // large items (d+ > mid_max >= MID_MIN, at most m / MID_MIN owners) after the rest
    return wm_capacity(n, m) + m / MID_MIN + 2 * m / 256 + 64;
}

__device__ __forceinline__ uint32_t bucket_of(uint32_t d, const IsectConfig &cfg)
{
    return d <= cfg.warp_max ? 0u : (d <= min(max(cfg.mid_max, MID_MIN), MID_MAX) ? 1u : 2u);
}

// Partners per item of an owner of out-degree d in bucket b (see IsectConfig).
__device__ __forceinline__ uint32_t seg_len(uint32_t d, uint32_t b, const IsectConfig &cfg)
{
    const uint32_t floor = b == 0 ? SEG_MIN : 256u;
    const uint32_t work = b == 0 ? cfg.work_w : (b == 1 ? cfg.work_b : cfg.work_l);
    uint32_t s = b == 0 ? cfg.seg_w : (b == 1 ? min(cfg.seg_b, SEG_B) : min(cfg.seg_l, SEG_L));
    while (s > floor && (uint64_t)s * d > work) s >>= 1;
    return s;
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

__global__ void k_items(const uint32_t *__restrict__ rowptr, const uint32_t *__restrict__ inptr,
                        const uint32_t *__restrict__ inend, const uint32_t *__restrict__ ocnt, uint32_t n,
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
            if (d >= 2) np = ocnt[x] + (inend[x] - inptr[x]);
        }
        const uint32_t gx = batch ? find_part_warp(bv.voff, bv.k, (uint32_t)(x < n ? x : n - 1)) : 0u;
        const uint32_t b = bucket_of(d, cfg), seg = seg_len(d, b, cfg);
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
    k_items<<<grid_for(b.n, 256, 152 * 8), 256, 0, s>>>(b.rowptr, b.inptr, b.inend, b.ocnt, b.n, b.items, wm, b.items_cap,
                                                          b.st, b.bv, b.cfg);
    note_launch();
}

// ======================================================================
// Shared-memory hash set of an out-list: buckets of two slots (one 8-byte
// load per lookup), filled in slot order, with linear probing over buckets.
// At most an eighth of the slots are used where the table fits (a quarter
// otherwise), so a lookup almost always ends at its first bucket.  A full
// bucket holds its two keys in increasing order, or in decreasing order once
// some key has overflowed from it into the following buckets: a lookup that
// misses in a full bucket goes on only then, and ends at the first bucket
// with a free slot.  (A full bucket is common: about 9% of the buckets at a
// quarter of the slots used; one that overflowed is rare.)  Every change to
// a bucket is one 8-byte compare-and-swap; a bucket changes at most three
// times (empty, one key, two keys in order, swapped), which bounds the retry
// loops.  The probe loops are bounded by the table size.
// ======================================================================

__device__ __forceinline__ uint32_t bucket_hash(uint32_t y, uint32_t shift) { return (y * 0x9e3779b1u) >> shift; }

__device__ __forceinline__ unsigned long long bucket_pack(uint32_t lo, uint32_t hi)
{
    return ((unsigned long long)hi << 32) | lo;
}

// nb = 2^k buckets: mask = nb - 1, shift = 32 - k.
__device__ __forceinline__ void bucket_insert(uint2 *tab, uint32_t mask, uint32_t shift, uint32_t y)
{
    unsigned long long *t64 = reinterpret_cast<unsigned long long *>(tab);
    const uint32_t home = bucket_hash(y, shift);
    uint32_t b = home;
    for (uint32_t it = 0; it <= mask; ++it) {
        unsigned long long cur = ~0ull;  // first guess: empty
        for (int tries = 0; tries < 8; ++tries) {
            const uint32_t k0 = (uint32_t)cur, k1 = (uint32_t)(cur >> 32);
            if (k0 == y || k1 == y) return;
            if (k1 != EMPTY) break;  // full: probe on
            const unsigned long long want =
                k0 == EMPTY ? bucket_pack(y, EMPTY) : (k0 < y ? bucket_pack(k0, y) : bucket_pack(y, k0));
            const unsigned long long prev = atomicCAS(t64 + b, cur, want);
            if (prev == cur) {
                if (b != home) {  // overflowed: the (full) home bucket takes the decreasing order
                    unsigned long long h = atomicOr(t64 + home, 0ull);
                    for (int t2 = 0; t2 < 4 && (uint32_t)h < (uint32_t)(h >> 32); ++t2) {
                        const unsigned long long p2 = atomicCAS(t64 + home, h, bucket_pack((uint32_t)(h >> 32), (uint32_t)h));
                        if (p2 == h) break;
                        h = p2;
                    }
                }
                return;
            }
            cur = prev;
        }
        b = (b + 1) & mask;
    }
}

struct BucketSet {
    const uint2 *tab;
    uint32_t mask, shift;
    __device__ __forceinline__ uint32_t contains(uint32_t y) const
    {
        uint32_t b = bucket_hash(y, shift);
        uint2 v = tab[b];
        bool hit = v.x == y || v.y == y;
        // a hit, a free slot (EMPTY is the largest value; an empty bucket has
        // v.x == v.y) or a full bucket without overflow
        if (hit || v.x <= v.y) return hit;
        for (uint32_t it = 0; !hit && v.y != EMPTY && it < mask; ++it) {
            b = (b + 1) & mask;
            v = tab[b];
            hit = v.x == y || v.y == y;
        }
        return hit;
    }
};

// Table size (slots) for an owner of out-degree d: a power of two >= 8 d,
// at most cap; 0 when even 4 d slots do not fit.
__device__ __forceinline__ uint32_t table_slots(uint32_t d, uint32_t cap)
{
    uint32_t slots = 64;
    while (slots < 8 * d && slots < cap) slots <<= 1;
    return (slots <= cap && (uint64_t)slots >= 4ull * d) ? slots : 0u;
}

// Shift of the bucket hash for a table of `slots` slots (slots / 2 buckets).
__device__ __forceinline__ uint32_t bucket_shift(uint32_t slots) { return 32u - (31u - __clz(slots >> 1)); }

// Bitmap of an owner's list over its rank window: vertex base + i is in the
// set iff bit i of bm is set (i < bits).  The rows are sorted by rank, so an
// owner x with largest out-neighbour `last` needs last - x bits from base =
// x + 1; every streamed entry is ranked above x (or is SENT, or an entry of
// an in-partner's row before x, which all fall outside the window).  One
// 4-byte shared load and no probe loop per lookup.
struct BitmapSet {
    const uint32_t *bm;
    uint32_t base, bits;
    __device__ __forceinline__ uint32_t contains(uint32_t y) const
    {
        const uint32_t o = y - base;
        return o < bits ? (bm[o >> 5] >> (o & 31u)) & 1u : 0u;
    }
};

// Fallback for rows whose hash set does not fit on chip: binary search of
// the sorted row in global memory.
struct SortedRow {
    const uint32_t *a;
    uint32_t len;
    __device__ __forceinline__ uint32_t contains(uint32_t w) const
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

// Pair classes and what the kernels need to finish them.
struct PairCtx {
    const uint8_t *heavy;
    uint32_t lim;      // DevState::light_lim
    bool dense;        // the tensor path counts the all-heavy triangles
    uint32_t core_lo;  // pairs whose lower endpoint is at or above this id are the core block's
};

// Partner of owner x (heavy flag hx): the chunk range of the part of the
// partner's padded out-list to stream and whether both endpoints of the pair
// are heavy (hh), from its list entry e (csr.cu).  Out-list partner y: e.x = y
// (its padded row starts at ptrp[y]), e.y = d+(y) with y's heavy flag in bit 31.
// In-list partner: e.x is the padded position of x in the partner's row, e.y
// the number of entries after it (>= 1), with the partner's heavy flag in
// bit 31.  The range is empty when the pair is
// resolved by the other endpoint, closes no triangle, or (dense) can close
// no triangle with a light vertex.  Also counts the streamed list entries
// into the tally.
__device__ __forceinline__ void partner_of(const uint32_t *__restrict__ ptrp, const PairCtx &pc, uint32_t hx,
                                           uint32_t x, bool is_out, uint2 e, uint32_t &c0, uint32_t &nc, uint32_t &hh,
                                           Tally &t)
{
    uint32_t len, b;
    if (is_out) {  // pair (x -> y): e.x = y, e.y = d+(y) | y's heavy flag << 31
        // (the compaction appended it only for 1 <= d+(y) <= d+(x) and a row of
        // x that goes on past y, and never a pair both of whose ends the dense
        // block counts)
        len = x < pc.core_lo ? e.y & 0x7fffffffu : 0u;
        c0 = (__ldg(ptrp + e.x) & ~3u) >> 2;
        nc = (len + 3) >> 2;
        b = 0;
        hh = hx ? e.y >> 31 : 0u;
    } else {  // pair (partner -> x): the entries of the partner's row after x
        // the compaction appended it only for 2 <= d+(partner) < d, a row
        // that goes on past x and a partner below the core
        len = e.y & 0x7fffffffu;
        c0 = (e.x + 1) >> 2;
        nc = ((e.x + 1 + len + 3) >> 2) - c0;
        b = x;
        hh = hx ? e.y >> 31 : 0u;
    }
    if (hh && pc.dense && b >= pc.lim) len = nc = 0;  // every third vertex would be heavy
    t.stream += len;
    t.partners += len != 0;
}

// Looks up the 4 entries of a chunk; hits go to hl (light triangles), or for
// a pair of two heavy vertices to hl / hv by the third vertex's class.
template <class Set>
__device__ __forceinline__ void probe4(const Set &set, const uint4 &q, bool hh, const PairCtx &pc, uint32_t &hl,
                                       uint32_t &hv)
{
    // the lookups are the same for every pair (no divergence between the
    // lanes of heavy-heavy pairs and the others); only the hits of a
    // heavy-heavy pair look at the third vertex's class
    const uint32_t y[4] = {q.x, q.y, q.z, q.w};
    uint32_t h[4];
#pragma unroll
    for (int i = 0; i < 4; ++i) h[i] = set.contains(y[i]);
    if (!hh) {
        hl += h[0] + h[1] + h[2] + h[3];
        return;
    }
#pragma unroll
    for (int i = 0; i < 4; ++i) {
        if (h[i]) {
            if (y[i] >= pc.lim || __ldg(pc.heavy + y[i])) ++hv; else ++hl;
        }
    }
}

__device__ __forceinline__ void add_hits(Tally &t, const PairCtx &pc, uint32_t hl, uint32_t hv)
{
    t.light += hl;
    if (!pc.dense) t.heavy += hv;  // else counted by the tensor path
}

// Lanes [a, b) of the warp hold consecutive parts with cnt >= 1 entries
// each (other lanes cnt = 0), laid end to end at exclusive offsets pre.
// Returns the lane of the part that holds entry `e` (< the total), given
// `starts`, the bitmask of the parts beginning inside e's 32-entry window,
// and `before`, the parts that began before it.
__device__ __forceinline__ uint32_t part_lane(uint32_t a, uint32_t before, unsigned starts, unsigned upto)
{
    return (a + before + __popc(starts & upto) - 1) & 31u;
}

// Streams the padded out-lists of up to 32 partners (one per lane: chunks
// [c0, c0 + nc) of the uint4 view of the columns; hh: both endpoints heavy)
// through the owners' sets.  The partners' chunks are laid end to end and
// every step hands each lane one 16-byte chunk (4 list entries; the SENT
// padding never matches).  A lane finds the partner of its chunk in O(1):
// a bitmask of the partners whose chunks start inside the current 32-chunk
// window, plus the count of those that started before it.  NWIN windows are
// in flight per step.  MULTI: each partner looks up its own owner's set in
// the warp's table (tinfo = first bucket | shift << 16); else all use set.
// s_base / s_tinfo: this warp's 32-entry shared scratch.
template <bool MULTI, class Set>
__device__ __forceinline__ void stream_chunks(const uint4 *__restrict__ col4, const Set &set, const uint2 *wtab,
                                              uint32_t c0, uint32_t nc, uint32_t hh, uint32_t tinfo,
                                              uint32_t *s_base, uint32_t *s_tinfo, const PairCtx &pc, Tally &t)
{
    const unsigned lane = lane_id();
    const unsigned live = __ballot_sync(FULL, nc != 0);
    if (!live) return;
    const uint32_t inc = warp_incl_scan(nc);
    const uint32_t pre = inc - nc;  // first chunk of this partner in the window sequence
    const uint32_t W = __shfl_sync(FULL, inc, 31);
    const uint32_t r = __popc(live & lanemask_lt());  // rank among live partners
    const unsigned hh_bits = __reduce_or_sync(FULL, (nc != 0 && hh != 0) ? (1u << r) : 0u);
    if (nc) {
        s_base[r] = c0 - pre;  // chunk of sequence position e: s_base[rank] + e
        if (MULTI) s_tinfo[r] = tinfo;
    }
    __syncwarp();
    const unsigned upto = 0xffffffffu >> (31 - lane);  // bits 0..lane
    uint32_t before = 0;  // live partners starting before the window
    uint32_t hl = 0, hv = 0;
    for (uint32_t wb = 0; wb < W; wb += 32 * NWIN) {
        uint32_t e[NWIN], k[NWIN];
        uint4 q[NWIN];
#pragma unroll
        for (int i = 0; i < NWIN; ++i) {
            const uint32_t off = pre - wb - 32u * i;
            const unsigned sti = __reduce_or_sync(FULL, (nc != 0 && off < 32u) ? (1u << off) : 0u);
            e[i] = wb + 32u * i + lane;
            k[i] = before + __popc(sti & upto) - 1;
            before += __popc(sti);
        }
#pragma unroll
        for (int i = 0; i < NWIN; ++i)
            if (e[i] < W) q[i] = __ldg(col4 + (s_base[k[i]] + e[i]));
#pragma unroll
        for (int i = 0; i < NWIN; ++i) {
            if (e[i] < W) {
                const bool h2 = (hh_bits >> k[i]) & 1u;
                if (MULTI) {
                    const uint32_t ti = s_tinfo[k[i]], sh = ti >> 16;
                    const BucketSet ms{wtab + (ti & 0xffffu), (1u << (32u - sh)) - 1u, sh};
                    probe4(ms, q[i], h2, pc, hl, hv);
                } else {
                    probe4(set, q[i], h2, pc, hl, hv);
                }
            }
        }
    }
    add_hits(t, pc, hl, hv);
    __syncwarp();  // s_base / s_tinfo are rewritten by the next call
}

// ---------------------------------------------------------------- warp items

constexpr int PW_THREADS = 256;
constexpr int PW_WARPS = PW_THREADS / 32;
constexpr uint32_t WTAB = 1024;  // per-warp table slots, >= 4 * WARP_MAX

// A warp takes 32 warp items at a time (one per lane) and resolves them in
// packs: runs of consecutive items of one graph whose hash sets fit the
// warp's table together (sum of slots <= WTAB).  A pack's out-lists are
// inserted, and its partners set up and streamed, as single flattened
// sequences, so a pack of many small owners costs about what one owner with
// the same number of partners and list entries costs.
__global__ void __launch_bounds__(PW_THREADS, 4) k_probe_warp(const uint32_t *__restrict__ ptrp,
                                                           const uint32_t *__restrict__ col,
                                                           const uint32_t *__restrict__ rowptr,
                                                           const uint2 *__restrict__ olist,
                                                           const uint32_t *__restrict__ ocnt,
                                                           const uint32_t *__restrict__ inptr,
                                                           const uint32_t *__restrict__ inend,
                                                           const uint2 *__restrict__ inlist,
                                                           const uint64_t *__restrict__ items, uint64_t wm_cap,
                                                           const uint8_t *__restrict__ heavy, DevState *st,
                                                           BatchView bv, IsectConfig cfg, uint32_t core_base)
{
    __shared__ uint2 s_tab[PW_WARPS][WTAB / 2];
    __shared__ uint32_t s_base[PW_WARPS][32];
    __shared__ uint32_t s_tinfo[PW_WARPS][32];
    // the 32 items of the current grab, by lane: row start, out-list start
    // and length, in-list start, first partner, owner, and out-degree |
    // heavy flag << 31
    __shared__ uint32_t s_beg[PW_WARPS][32], s_ob[PW_WARPS][32], s_oc[PW_WARPS][32], s_ib[PW_WARPS][32];
    __shared__ uint32_t s_p0[PW_WARPS][32], s_dh[PW_WARPS][32], s_x[PW_WARPS][32];
    __shared__ uint32_t s_ti[PW_WARPS][32], s_pre[PW_WARPS][32];  // table info; prefix within the pack
    __shared__ unsigned long long red[33];
    const unsigned lane = lane_id(), w = threadIdx.x >> 5;
    const unsigned upto = 0xffffffffu >> (31 - lane);
    const uint32_t nitems = (uint32_t)min((unsigned long long)st->nlist[0], (unsigned long long)wm_cap);
    const PairCtx pc{heavy, st->light_lim, st->dense != 0, st->core_on ? core_base : 0xffffffffu};
    const uint4 *col4 = reinterpret_cast<const uint4 *>(col);
    uint2 *tab = s_tab[w];
    const bool batch = bv.k != 0;
    uint32_t cur_g = 0;  // graph whose counts this warp holds (batch)
    uint32_t table_of = 0xffffffffu;  // owner whose set the table holds (single-item packs), else ~0
    Tally t;
    for (;;) {
        uint32_t first = 0;
        if (lane == 0) first = atomicAdd(&st->cursor[0], GRAB);
        first = __shfl_sync(FULL, first, 0);
        if (first >= nitems) break;
        const uint32_t got = min(GRAB, nitems - first);
        // lane i: item first + i
        uint32_t g = 0, d = 0, slots = 0, npart = 0;
        if (lane < got) {
            uint32_t x, seg;
            split_item(items[first + lane], batch, x, seg, g);
            const PaddedRow row = padded_row(ptrp, x);
            d = row.d;
            slots = d <= cfg.warp_max && d <= WARP_MAX ? table_slots(d, WTAB) : 0u;
            uint32_t hx = 0, ob = 0, oc = 0, ib = 0, p0 = 0;
            if (slots && d >= 2) {
                hx = heavy[x];
                ob = rowptr[x];
                oc = ocnt[x];
                ib = inptr[x];
                const uint32_t np = oc + (inend[x] - ib);
                const uint32_t sl = seg_len(d, 0, cfg);
                p0 = seg * sl;
                npart = np > p0 ? min(np - p0, sl) : 0u;
                if (seg == 0) t.table += d;
            }
            if (!slots || d < 2 || !npart) {  // only if the item list overflowed
                atomicOr(&st->err, ERR_OVERFLOW);
                slots = 0;
            }
            s_beg[w][lane] = row.beg;
            s_ob[w][lane] = ob;
            s_oc[w][lane] = oc;
            s_ib[w][lane] = ib;
            s_p0[w][lane] = p0;
            s_dh[w][lane] = d | (hx << 31);
            s_x[w][lane] = x;
        }
        const bool good = slots != 0;
        uint32_t a = 0;
        while (a < got) {
            if (!__shfl_sync(FULL, good, a)) {  // skip a bad item
                ++a;
                continue;
            }
            // the pack: lanes [a, b), one graph, sum of slots <= WTAB
            const uint32_t ga = __shfl_sync(FULL, g, a);
            const uint32_t sl = lane >= a && lane < got ? slots : 0u;
            const uint32_t inc = warp_incl_scan(sl);
            const bool ok = lane >= a && lane < got && good && inc <= WTAB && (!batch || g == ga);
            const unsigned notok = ~__ballot_sync(FULL, ok) & (0xffffffffu << a);
            const uint32_t b = notok ? min((uint32_t)__ffs(notok) - 1, got) : got;
            const bool in_pack = lane >= a && lane < b;
            const uint32_t total_buckets = __shfl_sync(FULL, inc, b - 1) >> 1;
            if (in_pack) s_ti[w][lane] = ((inc - sl) >> 1) | (bucket_shift(slots) << 16);  // first bucket | shift
            if (batch && ga != cur_g) {
                flush_graph_counts(t, bv, cur_g);
                cur_g = ga;
            }
            // consecutive segments of one owner reuse its set
            const uint32_t xa = __shfl_sync(FULL, s_x[w][lane], a);
            const bool reuse = b == a + 1 && xa == table_of;
            table_of = b == a + 1 ? xa : 0xffffffffu;
            if (!reuse)
                for (uint32_t i = lane; i < total_buckets; i += 32) tab[i] = make_uint2(EMPTY, EMPTY);
            // insert the pack's out-lists, one entry per lane per step
            if (!reuse) {
                const uint32_t c = in_pack ? d : 0u;
                const uint32_t ic = warp_incl_scan(c), tot = __shfl_sync(FULL, ic, 31);
                s_pre[w][lane] = ic - c;
                __syncwarp();
                const uint32_t pcs = ic - c;
                uint32_t before = 0;
                for (uint32_t wb = 0; wb < tot; wb += 32) {
                    const unsigned sts = __reduce_or_sync(FULL, (c != 0 && pcs - wb < 32u) ? (1u << (pcs - wb)) : 0u);
                    const uint32_t L = part_lane(a, before, sts, upto);
                    const uint32_t e = wb + lane;
                    if (e < tot) {
                        const uint32_t ti = s_ti[w][L], sh = ti >> 16;
                        bucket_insert(tab + (ti & 0xffffu), (1u << (32u - sh)) - 1u, sh,
                                      __ldg(col + s_beg[w][L] + (e - s_pre[w][L])));
                    }
                    before += __popc(sts);
                }
                __syncwarp();
            }
            // partners, 32 per step, each streamed through its owner's set
            {
                const uint32_t c = in_pack ? npart : 0u;
                const uint32_t ic = warp_incl_scan(c), tot = __shfl_sync(FULL, ic, 31);
                s_pre[w][lane] = ic - c;
                __syncwarp();
                const uint32_t pcs = ic - c;
                uint32_t before = 0;
                for (uint32_t wb = 0; wb < tot; wb += 32) {
                    const unsigned sts = __reduce_or_sync(FULL, (c != 0 && pcs - wb < 32u) ? (1u << (pcs - wb)) : 0u);
                    const uint32_t L = part_lane(a, before, sts, upto);
                    const uint32_t q = wb + lane;
                    uint32_t c0 = 0, nc = 0, hh = 0, ti = 0;
                    if (q < tot) {
                        const uint32_t dh = s_dh[w][L];
                        const uint32_t j = s_p0[w][L] + (q - s_pre[w][L]), oc = s_oc[w][L];
                        const bool is_out = j < oc;
                        const uint2 e = is_out ? __ldg(olist + s_ob[w][L] + j) : __ldg(inlist + s_ib[w][L] + j - oc);
                        ti = s_ti[w][L];
                        partner_of(ptrp, pc, dh >> 31, s_x[w][L], is_out, e, c0, nc, hh, t);
                    }
                    stream_chunks<true>(col4, BucketSet{tab, 0, 0}, tab, c0, nc, hh, ti, s_base[w], s_tinfo[w], pc, t);
                    before += __popc(sts);
                }
            }
            __syncwarp();  // the table and the pack arrays are rewritten next
            a = b;
        }
    }
    if (batch) flush_graph_counts(t, bv, cur_g);
    flush_tally(t, red, st);
}

// ---------------------------------------------------------------- block items

constexpr int PB_THREADS = 128;       // mid owners: eight CTAs per SM, one small table each
constexpr int PB_DYN_THREADS = 1024;  // large owners: one CTA per SM around one table of up to 128 KiB
constexpr uint32_t MID_TAB = 4096;                      // >= 4 * MID_MAX slots (dynamic shared memory)
constexpr uint32_t UNIT = 128;                          // chunks per unit of block streaming
constexpr int NWIN_MID = 2;                             // windows in flight per warp step: mid owners
constexpr int NWIN_DYN = 2;                             // and large owners
constexpr uint32_t PRE_CLS = 0x80000000u;               // class bit beside a partner's chunk prefix

// Streams chunks [wb0, min(wb0 + UNIT, total)) of an item's partner sequence
// through set.  Live partner k has its chunks at s_c0[k] .. and begins at
// position s_pre[k] & ~PRE_CLS of the sequence (increasing in k); the warp
// finds the partner covering wb0 by a 32-way search and then maps chunks to
// partners window by window as stream_chunks does, except that a window
// lying inside one partner (a long list) reads that partner's chunks
// directly.
template <int WIN, class Set>
__device__ __forceinline__ void stream_unit(const uint4 *__restrict__ col4, const Set &set, const uint32_t *s_c0,
                                            const uint32_t *s_pre, uint32_t nlive, uint32_t total, uint32_t wb0,
                                            const PairCtx &pc, Tally &t)
{
    const unsigned lane = lane_id();
    const unsigned upto = 0xffffffffu >> (31 - lane);
    // largest k with pre[k] <= wb0 (pre[0] = 0)
    uint32_t lo = 0, hi = nlive;
    while (hi - lo > 1) {
        const uint32_t step = (hi - lo + 31) / 32;
        const uint32_t k = lo + lane * step;
        const bool ok = k < hi && (s_pre[k] & ~PRE_CLS) <= wb0;
        const unsigned m = __ballot_sync(FULL, ok);  // lanes 0 .. j
        const uint32_t j = 31 - __clz(m);
        lo += j * step;
        hi = min(hi, lo + step);
    }
    uint32_t before = lo + ((s_pre[lo] & ~PRE_CLS) < wb0 ? 1u : 0u);  // partners beginning before the window
    const uint32_t end = min(total, wb0 + UNIT);
    uint32_t hl = 0, hv = 0;
    // the partner that covers the window start (before - 1) and where the
    // next one begins: a window that lies inside one partner needs no mapping
    uint32_t cur = before ? before - 1 : 0u, cur_pk = s_pre[cur], cur_c0 = s_c0[cur];
    uint32_t nxt = before < nlive ? s_pre[before] & ~PRE_CLS : total;
    for (uint32_t wb = wb0; wb < end; wb += 32 * WIN) {
        uint32_t e[WIN], pk[WIN];
        uint4 q[WIN];
#pragma unroll
        for (int i = 0; i < WIN; ++i) {
            const uint32_t w0 = wb + 32u * i;
            e[i] = w0 + lane;
            if (before != 0 && w0 + 32u <= nxt) {  // warp-uniform: the whole window is in partner cur
                pk[i] = cur_pk;
                if (e[i] < end) q[i] = __ldg(col4 + (cur_c0 + (e[i] - (cur_pk & ~PRE_CLS))));
                continue;
            }
            const uint32_t kk = before + lane;
            const uint32_t pre = kk < nlive ? (s_pre[kk] & ~PRE_CLS) : 0xffffffffu;
            const unsigned sti = __reduce_or_sync(FULL, pre - w0 < 32u ? (1u << (pre - w0)) : 0u);
            const uint32_t k = before + __popc(sti & upto) - 1;
            before += __popc(sti);
            if (e[i] < end) {
                pk[i] = s_pre[k];
                q[i] = __ldg(col4 + (s_c0[k] + (e[i] - (pk[i] & ~PRE_CLS))));
            }
            cur = before - 1;  // covers the next window's start
            cur_pk = s_pre[cur];
            cur_c0 = s_c0[cur];
            nxt = before < nlive ? s_pre[before] & ~PRE_CLS : total;
        }
#pragma unroll
        for (int i = 0; i < WIN; ++i) {
            if (e[i] < end) probe4(set, q[i], (pk[i] & PRE_CLS) != 0, pc, hl, hv);
        }
    }
    add_hits(t, pc, hl, hv);
}

// One block resolves one item: up to seg_b partners of one owner.  Every
// thread sets up its share of the partners; the live ones are compacted
// into shared memory with the prefix of their chunk counts, and the warps
// take the item's chunk sequence UNIT chunks at a time from a shared
// counter, so they finish within one unit of each other.  The owner's set
// sits in dynamic shared memory (tab_slots 4-byte slots): a hash set, or
// where it does not fit or the schedule asks for it a binary search of the
// owner's sorted row (!BM); a bitmap of its rank window, or where that does
// not fit the hash set (BM, mid owners: their set always fits) or the
// binary search (BM, large owners).  A kernel holds two of the three
// lookups: with all three inlined into the streaming loop the 64-register
// budget spills.
template <bool DYN, bool BM>
__global__ void __launch_bounds__(DYN ? PB_DYN_THREADS : PB_THREADS, DYN ? 1 : 8) k_probe_block(const uint32_t *__restrict__ ptrp,
                                                                      const uint32_t *__restrict__ col,
                                                                      const uint32_t *__restrict__ rowptr,
                                                                      const uint2 *__restrict__ olist,
                                                                      const uint32_t *__restrict__ ocnt,
                                                                      const uint32_t *__restrict__ inptr,
                                                                      const uint32_t *__restrict__ inend,
                                                                      const uint2 *__restrict__ inlist,
                                                                      const uint64_t *__restrict__ items,
                                                                      uint64_t wm_cap,
                                                                      const uint8_t *__restrict__ heavy,
                                                                      DevState *st, uint32_t tab_slots,
                                                                      uint64_t cap, BatchView bv, IsectConfig cfg,
                                                                      uint32_t core_base)
{
    constexpr uint32_t NT = DYN ? PB_DYN_THREADS : PB_THREADS;
    constexpr uint32_t SEG = DYN ? SEG_L : SEG_B;        // partners per item (at most)
    constexpr uint32_t PER_MAX = (SEG + NT - 1) / NT;    // partner slots set up per thread (at most)
    // dynamic shared memory: the owner's set (tab_slots 4-byte slots), then
    // the live partners of the current item (seg_cap of each array)
    extern __shared__ uint2 tab[];
    const uint32_t seg_cap = DYN ? min(cfg.seg_l, SEG_L) : min(cfg.seg_b, SEG_B);
    uint32_t *s_c0 = reinterpret_cast<uint32_t *>(tab) + tab_slots;
    uint32_t *s_pre = s_c0 + seg_cap;  // chunk prefix | PRE_CLS (both endpoints heavy)
    __shared__ unsigned long long wt[33];
    __shared__ unsigned long long red[33];
    __shared__ uint32_t s_idx, s_next, s_left, s_built;
    const unsigned lane = lane_id();
    const uint32_t b = DYN ? 2 : 1;
    const uint32_t nitems =
        (uint32_t)min((unsigned long long)st->nlist[b], (unsigned long long)(DYN ? cap - wm_cap : wm_cap));
    // a block takes consecutive items per grab (large owners up to 8, mid
    // owners up to cfg.run_b, at least 8 grabs per block): an owner's items
    // are consecutive, and the table is rebuilt only when the owner changes
    const uint32_t run = max(1u, min(DYN ? 8u : min(cfg.run_b, 8u), nitems / (gridDim.x * 8u)));
    if (threadIdx.x == 0) {
        s_left = 0;
        s_built = 0xffffffffu;  // owner whose set the table holds
    }
    const PairCtx pc{heavy, st->light_lim, st->dense != 0, st->core_on ? core_base : 0xffffffffu};
    const uint4 *col4 = reinterpret_cast<const uint4 *>(col);
    Tally t;
    for (;;) {
        if (threadIdx.x == 0) {
            if (s_left == 0) {
                s_idx = atomicAdd(&st->cursor[b], run);
                s_left = run;
            } else {
                ++s_idx;
            }
            --s_left;
            s_next = 0;
        }
        __syncthreads();
        const uint32_t idx = s_idx;
        if (idx >= nitems) break;
        uint32_t x, seg, g;
        split_item(DYN ? items[wm_cap + idx] : items[wm_cap - 1 - idx], bv.k != 0, x, seg, g);
        const PaddedRow row = padded_row(ptrp, x);
        const uint32_t d = row.d;
        const uint32_t hx = heavy[x];
        // the owner's set (BM kernels run only without the schedule's
        // binary-search bit)
        constexpr bool HASH = !BM || !DYN, SORTED = !BM || DYN;
        const bool bsearch = !BM && ((cfg.lookup >> (DYN ? 1 : 0)) & 1u);
        uint32_t bits = 0;
        if (BM) {
            bits = __ldg(col + row.beg + d - 1) - x;  // up to the largest out-neighbour (d >= 2)
            if (bits > tab_slots * 32u || (uint64_t)x + 1 + bits > (uint64_t)SENT) bits = 0;
        }
        const bool bitmap = bits != 0;
        const uint32_t slots = !HASH || bitmap || bsearch ? 0u : table_slots(d, tab_slots);
        if (!SORTED && !bitmap && !slots && threadIdx.x == 0) atomicOr(&st->err, ERR_OVERFLOW);  // never: see above
        const BucketSet set{tab, slots ? (slots >> 1) - 1 : 0u, slots ? bucket_shift(slots) : 0u};
        uint32_t *bm = reinterpret_cast<uint32_t *>(tab);
        if ((slots || bitmap) && s_built != x) {
            if (bitmap) {
                for (uint32_t i = threadIdx.x; i < (bits + 31) / 32; i += NT) bm[i] = 0u;
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < d; i += NT) {
                    const uint32_t o = __ldg(col + row.beg + i) - (x + 1);
                    atomicOr(bm + (o >> 5), 1u << (o & 31u));
                }
            } else {
                for (uint32_t i = threadIdx.x; i < (slots >> 1); i += NT) tab[i] = make_uint2(EMPTY, EMPTY);
                __syncthreads();
                for (uint32_t i = threadIdx.x; i < d; i += NT)
                    bucket_insert(tab, set.mask, set.shift, __ldg(col + row.beg + i));
            }
        }
        if (seg == 0 && threadIdx.x == 0) t.table += d;
        const uint32_t ob = rowptr[x], oc = ocnt[x], ib = inptr[x], np = oc + (inend[x] - ib);
        const uint32_t sl = seg_len(d, DYN ? 2 : 1, cfg);
        const uint32_t p0 = seg * sl, p1 = min(np, p0 + sl);
        const uint32_t per = (sl + NT - 1) / NT;  // <= PER_MAX
        // set up this thread's `per` consecutive partners
        uint32_t pc0[PER_MAX], pncc[PER_MAX];
        unsigned long long mine = 0;  // live partners << 32 | their chunks
#pragma unroll
        for (uint32_t q = 0; q < PER_MAX; ++q) {
            const uint32_t j = p0 + threadIdx.x * per + q;
            uint32_t c0 = 0, nc = 0, hh = 0;
            if (q < per && j < p1) {
                const bool is_out = j < oc;
                const uint2 e = is_out ? __ldg(olist + ob + j) : __ldg(inlist + ib + j - oc);
                partner_of(ptrp, pc, hx, x, is_out, e, c0, nc, hh, t);
            }
            pc0[q] = c0;
            pncc[q] = (nc << 1) | hh;
            if (nc) mine += (1ull << 32) | nc;
        }
        unsigned long long tot;
        const unsigned long long ex = block_excl_scan(mine, wt, &tot);  // also orders the set build
        uint32_t r = (uint32_t)(ex >> 32), pre = (uint32_t)ex;
#pragma unroll
        for (uint32_t q = 0; q < PER_MAX; ++q) {
            const uint32_t nc = pncc[q] >> 1;
            if (nc) {
                s_c0[r] = pc0[q];
                s_pre[r] = pre | (pncc[q] & 1u ? PRE_CLS : 0u);
                ++r;
                pre += nc;
            }
        }
        const uint32_t nlive = (uint32_t)(tot >> 32), total = (uint32_t)tot;
        __syncthreads();  // partners and set are complete
        for (;;) {
            uint32_t u = 0;
            if (lane == 0) u = atomicAdd(&s_next, 1u);
            u = __shfl_sync(FULL, u, 0);
            if (u * UNIT >= total) break;
            if (BM && bitmap) {
                stream_unit<DYN ? NWIN_DYN : NWIN_MID>(col4, BitmapSet{bm, x + 1, bits}, s_c0, s_pre, nlive, total,
                                                   u * UNIT, pc, t);
            } else if (HASH && slots) {
                stream_unit<DYN ? NWIN_DYN : NWIN_MID>(col4, set, s_c0, s_pre, nlive, total, u * UNIT, pc, t);
            } else if constexpr (SORTED) {
                stream_unit<DYN ? NWIN_DYN : NWIN_MID>(col4, SortedRow{col + row.beg, d}, s_c0, s_pre, nlive, total,
                                                   u * UNIT, pc, t);
            }
        }
        if (bv.k != 0) flush_graph_counts(t, bv, g);
        __syncthreads();  // every warp is done with this owner
        if (threadIdx.x == 0) s_built = slots || bitmap ? x : 0xffffffffu;
    }
    flush_tally(t, red, st);
}

// Static + dynamic shared memory of the block kernels must fit the
// function's opt-in limit, which starts at 48 KiB in every process: raise it
// once per process and device (to the largest size requested so far for the
// large-owner kernel).
void intersect_prepare(int dyn_smem_bytes)
{
    static int set_bytes[64] = {};
    static bool mid_set[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    const bool known = dev >= 0 && dev < 64;
    if (!known || !mid_set[dev]) {
        const int mid = (int)(MID_TAB * 4 + 2 * SEG_B * 4);
        if (cudaFuncSetAttribute(k_probe_block<false, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, mid) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_probe_block<false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, mid) ==
                cudaSuccess &&
            known)
            mid_set[dev] = true;
    }
    const int dyn = dyn_smem_bytes + (int)(2 * SEG_L * 4);
    if (!known || dyn > set_bytes[dev]) {
        if (cudaFuncSetAttribute(k_probe_block<true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) ==
                cudaSuccess &&
            cudaFuncSetAttribute(k_probe_block<true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, dyn) ==
                cudaSuccess &&
            known)
            set_bytes[dev] = dyn;
    }
}

void intersect(const CountBuffers &b, int dyn_smem_bytes, cudaStream_t s)
{
    if (b.n == 0 || b.m == 0) return;
    const uint64_t wm = wm_capacity(b.n, b.m);
    intersect_prepare(dyn_smem_bytes);
    k_probe_warp<<<152 * 4, PW_THREADS, 0, s>>>(b.ptrp, b.col, b.rowptr, b.olist, b.ocnt, b.inptr, b.inend, b.inlist,
                                                b.items, wm, b.heavy, b.st, b.bv, b.cfg, b.core_base);
    note_launch();
    const uint32_t seg_b = std::min(b.cfg.seg_b, SEG_B), seg_l = std::min(b.cfg.seg_l, SEG_L);
    auto kmid = (b.cfg.lookup & 5u) == 4u ? k_probe_block<false, true> : k_probe_block<false, false>;
    kmid<<<152 * 8, PB_THREADS, MID_TAB * 4 + 2 * seg_b * 4, s>>>(b.ptrp, b.col, b.rowptr, b.olist, b.ocnt, b.inptr,
                                                                 b.inend, b.inlist, b.items, wm, b.heavy, b.st, MID_TAB,
                                                                 b.items_cap, b.bv, b.cfg, b.core_base);
    note_launch();
    auto klarge = (b.cfg.lookup & 10u) == 8u ? k_probe_block<true, true> : k_probe_block<true, false>;
    klarge<<<152, PB_DYN_THREADS, dyn_smem_bytes + 2 * seg_l * 4, s>>>(b.ptrp, b.col, b.rowptr, b.olist, b.ocnt,
                                                                      b.inptr, b.inend, b.inlist, b.items, wm, b.heavy,
                                                                      b.st, (uint32_t)(dyn_smem_bytes / 4),
                                                                      b.items_cap, b.bv, b.cfg, b.core_base);
    note_launch();
}

}  // namespace tcg
