// Host-side launchers of the libtc device kernels (internal interface).
#pragma once

#include <cstdint>
#include <vector>
#include <cuda_runtime.h>

#include "common.cuh"

namespace tcg {

// ---------------------------------------------------------------- prims.cu
constexpr int RX_THREADS = 256;                  // 8 warps per tile
constexpr int RX_ITEMS = 16;                     // items per thread
constexpr int RX_TILE = RX_THREADS * RX_ITEMS;   // 4096 items per tile
constexpr int RX_MAX_BITS = 8;                   // digit width limit
constexpr int RX_BINS = 1 << RX_MAX_BITS;
constexpr int SC_CHUNK = 4096;                   // scan elements per block

inline uint64_t ceil_div(uint64_t a, uint64_t b) { return (a + b - 1) / b; }

// Process-wide count of kernel launches made by the library (api.cu);
// add_launches accounts for the kernels of a replayed CUDA graph.
void note_launch();
void add_launches(unsigned long long n);

// Blocks for `work` items at `threads` per block, at most `cap` (count.cu).
unsigned grid_for(uint64_t work, int threads, unsigned cap);

// Scratch (uint32 entries) needed by scan_excl_u32 for `len` elements.
uint64_t scan_scratch_elems(uint64_t len);

// In-place exclusive prefix sum of a[0, len).  If total is non-NULL the
// sum of all elements is written there (device pointer).  scratch holds
// scan_scratch_elems(len) uint32.
void scan_excl_u32(uint32_t *a, uint64_t len, uint32_t *total, uint32_t *scratch, cudaStream_t s);
// The same over 64-bit values; scratch holds ceil(len / SC_CHUNK) + 1 of them.
void scan_excl_u64(unsigned long long *a, uint64_t len, unsigned long long *total, unsigned long long *scratch,
                   cudaStream_t s);
// Exclusive prefix sums of a[0, len) and b[0, len) in one pass; the sum of b
// must stay below 2^32.  scratch as for scan_excl_u32.
void scan_excl_pair(uint32_t *a, uint32_t *b, uint64_t len, uint32_t *scratch, cudaStream_t s);

// One stable LSD radix pass over the n 64-bit items of `in` on bits
// [shift, shift + width), width <= 8, into out.  hist holds
// (1 << width) * ceil(n / RX_TILE) uint32; scan_scratch as for
// scan_excl_u32 on that many.
void radix_pass(const uint64_t *in, uint64_t n, int shift, int width, uint32_t *hist, uint32_t *scan_scratch,
                uint64_t *out, cudaStream_t s);

// Padded rows.  The column array of the counting kernels stores every row
// from a 16-byte boundary, padded with SENT up to a multiple of 4 entries,
// so that rows stream as aligned uint4 chunks.  ptrp[x] (x <= n) holds the
// padded start of row x (a multiple of 4) with the row's pad count
// (0..3) in its low two bits; ptrp[n] is the padded total.
constexpr uint32_t SENT = 0xfffffffeu;  // never a vertex id (ids < 2^32 - 2)
// Capacity (uint32 entries) of the padded column array for n, m.
inline uint64_t colp_capacity(uint32_t n, uint64_t m) { return m + 3 * (m < n ? m : (uint64_t)n) + 4; }
struct PaddedRow {
    uint32_t beg;  // padded start (multiple of 4)
    uint32_t d;    // out-degree
};
__device__ __forceinline__ PaddedRow padded_row(const uint32_t *__restrict__ ptrp, uint32_t x)
{
    const uint32_t a = __ldg(ptrp + x), b = __ldg(ptrp + x + 1);
    return PaddedRow{a & ~3u, (b & ~3u) - (a & ~3u) - (a & 3u)};
}

// Canonical keys from raw pairs: (min << 32 | max), self-loops become
// ~0ull; endpoints >= n raise ERR_ENDPOINT; pairs that are not strictly
// increasing in order are counted into st->unsorted.  With deg (zeroed, [n]),
// also counts the endpoints of the valid pairs: the full degrees when
// st->unsorted stays 0.
void canon_keys(const uint32_t *pairs, uint64_t m_in, uint32_t n, uint64_t *keys, DevState *st, cudaStream_t s,
                uint32_t *deg = nullptr);

// Stable removal of repeats and ~0ull from sorted keys; the count goes to
// st->m_canon.  tile_cnt holds ceil(m_in / RX_TILE) + 1 uint32.
void unique_keys(const uint64_t *keys, uint64_t m_in, uint64_t *out, uint32_t *tile_cnt,
                 uint32_t *scan_scratch, DevState *st, cudaStream_t s);

// ---------------------------------------------------------------- csr.cu
// Rank relabeling at graph creation (see csr.cu).  rank = (full degree, id)
// within the vertex's graph (batch unions: degree capped at 65535 for the
// rank, and every graph keeps its id range).
struct Relabeled {
    uint64_t *rel;   // [m] canonical keys in rank ids, sorted
    uint64_t *orig;  // [m] the original canonical key of each rel key
    uint32_t *perm;  // [n] original id of each rank id
    uint32_t *rank;  // [n] rank id of each original id
};
struct RelabelScratch {
    uint64_t *kA, *kB;  // [m] each
    uint64_t *vA, *vB;  // [n] each
    uint32_t *deg;      // [n]
    uint32_t *hist;     // radix histograms for max(m, n) items
    uint32_t *scan;     // scan scratch for those
};
// voff / k: batch union offsets (k = 0: one graph).  deg_ready: sc.deg
// already holds the full degrees (from canon_keys).  Returns out.rel.
uint64_t *relabel(const uint64_t *ekey, uint64_t m, uint32_t n, const uint32_t *voff, uint32_t k,
                  const Relabeled &out, const RelabelScratch &sc, cudaStream_t s, bool deg_ready = false);

// The sampled, oriented CSR of one count (single graph or batch union).
struct RowsArgs {
    const uint64_t *rel, *orig;  // relabeled keys and their original keys [m]
    uint64_t m;
    uint32_t n;
    uint64_t seed_mix, thr;      // single graph
    BatchView bv;                // batch union (bv.k > 0)
    uint32_t *deg;               // [n] sampled degrees
    uint32_t *rowptr;            // [n + 1] kept out-degrees, then row offsets
    uint32_t *inptr;             // [n + 1] in-list starts
    uint32_t *inend;             // [n] in-list ends: the in-list of v is inlist[inptr[v] .. inend[v])
    uint32_t *ptrp;              // [n + 2] padded row pointers (see SENT)
    uint32_t *colp;              // [colp_capacity(n, m)] padded columns
    uint2 *inlist;               // [m] in-list entries (source, padded position of the edge in its row)
    uint2 *olist;                // [m] out-lists: the live out-partners v of x at olist[rowptr[x] ..], each
                                 // as (v, d+(v) | v's heavy flag << 31 when x is heavy)
    uint32_t *ocnt;              // [n] their number
    uint32_t *keepw;             // [ceil(m / 32)] keep bits
    uint32_t *tile_cnt;          // [ceil(m / RX_TILE) + 1]
    uint32_t *scan;              // scan scratch for max(n + 1, tiles)
    uint32_t *spread;            // [hot_size(n)] per-vertex counters in hot_index order
    DevState *st;
    // single graph: the static rows (csr.cu static_rows; inptr then holds the
    // static in-list reservations) and the lower bound on m_p that picks the
    // vertices whose in-degrees are counted; nullptr: union path
    const uint32_t *frow = nullptr;
    uint64_t m_lo = 0;
    // heavy flags (partition); the in-list entries carry the source's flag.
    // Pairs the dense blocks count (DevState::dense / core_on) are left out of
    // the owners' lists: both ends heavy with the upper end at or above
    // light_lim, or the lower end at or above core_base
    const uint8_t *heavy = nullptr;
    uint32_t core_base = 0xffffffffu;
    // tiles with more than half their edges kept: scatter four edges of a
    // thread at a time (pays where nearly every tile is full, p >= 0.75; it
    // costs occupancy, 54 registers against 40, where most tiles are sparse)
    bool scatter4 = false;
};
// Rank-order rows (relabel) of up to ROW_MID keys are sorted by one warp in
// registers; longer rows by a block, with global scratch beyond shared memory.
constexpr uint32_t ROW_MID = 1024;
// Static rows of a single graph at creation: frow[0..n] (row offsets of rel)
// and inres[0..n] (in-list reservation offsets: full in-degrees).  perm and
// deg_orig: rank -> original id and the full degree by original id.
// *out = the number of v < n with deg[v] > thr.
void count_above(const uint32_t *deg, uint32_t n, uint32_t thr, unsigned long long *out, cudaStream_t s);
void static_rows(const uint64_t *rel, uint64_t m, uint32_t n, const uint32_t *perm, const uint32_t *deg_orig,
                 uint32_t *frow, uint32_t *inres, uint32_t *scan, cudaStream_t s);

// Dense-core candidates: w[k] (k < levels <= CORE_LEVELS_MAX, device) = the
// entries the p = 1 intersections stream for the pairs (not both heavy)
// whose lower end lies in the top core_min << k ranks but not in the top
// core_min << (k - 1).  inres: the full in-degree offsets (static rows).
constexpr int CORE_LEVELS_MAX = 4;
void core_work(const uint64_t *rel, const uint32_t *frow, const uint32_t *inres, uint32_t n, uint64_t m,
               uint32_t core_min, int levels, unsigned long long *w, cudaStream_t s);
// Counters that every edge bumps at its target (in-degrees, in-list
// cursors) are kept at hot_index(v): the id rotated within hot_bits(n) bits,
// so that consecutive ids (the hubs are the top ranks) land 4 KiB apart in
// different L2 slices instead of all on a few.
inline int hot_bits(uint32_t n)
{
    int b = 1;
    while (b < 32 && (1ull << b) < n) ++b;
    return b;
}
inline uint64_t hot_size(uint32_t n) { return 1ull << hot_bits(n); }
__host__ __device__ __forceinline__ uint32_t hot_index(uint32_t v, int bits)
{
    const int r = bits < 10 ? bits : 10;
    const uint32_t mask = bits >= 32 ? 0xffffffffu : (1u << bits) - 1u;
    return r == bits ? v : (((v << r) | (v >> (bits - r))) & mask);
}
// Sampling (Section 3.1), sampled degrees, kept out-degrees, keep bits.
void sample_rows(const RowsArgs &a, cudaStream_t s);
// After sample_rows (and the partition): the padded CSR and the in-lists.
void build_rows(const RowsArgs &a, cudaStream_t s);

// ---------------------------------------------------------------- count.cu
// Schedule of the intersection kernels (isect.cu); any choice gives the same
// counts.  warp_max: owners with 2 <= d+ <= warp_max are resolved by one warp
// (32 .. 256); seg_w / seg_b / seg_l: most partners per work item of the warp
// kernel, the mid-owner blocks (warp_max < d+ <= 1024) and the large-owner
// blocks (d+ > 1024) (seg_w in [SEG_MIN, 1024], seg_b in [256, 512], seg_l in
// [256, 4096], powers of two); work_w / work_b / work_l: an owner of
// out-degree d gets items of the largest power of two <= seg (of its kernel)
// partners with partners * d <= work, but at least SEG_MIN (warp) or 256
// (blocks), which bounds the list entries an item streams; run_b: items a
// mid-owner block takes per work-cursor grab (1 .. 8; consecutive items of
// one owner then share its hash set); mid_max: owners with warp_max < d+ <=
// mid_max go to the 128-thread blocks, larger ones to the 1024-thread blocks
// (512 .. 1024); lookup: how the block kernels test membership in the
// owner's list, bits 0 and 2 for the mid-owner blocks, bits 1 and 3 for the
// large-owner blocks: bit 0 / 1 a binary search of the owner's sorted row;
// else bit 2 / 3 a shared-memory bitmap of the owner's rank window, where
// the window does not fit the table's memory the hash set (mid owners) or
// the binary search (large owners); else a shared-memory hash set, or the
// binary search where it does not fit.  A graph's default sets bit 3 when
// no large owner's window can exceed the table (LOOKUP_BITMAP_LARGE,
// tc_graph_create).
constexpr uint32_t SEG_MIN = 64;
constexpr uint32_t LOOKUP_DEFAULT = 0;
constexpr uint32_t LOOKUP_BITMAP_LARGE = 8;
struct IsectConfig {
    uint32_t warp_max = 256;
    uint32_t seg_w = 512;
    uint32_t seg_b = 512;
    uint32_t work_w = 1u << 14;
    uint32_t work_b = 1u << 19;
    uint32_t seg_l = 4096;
    uint32_t work_l = 1u << 25;
    uint32_t run_b = 1;
    uint32_t mid_max = 1024;
    uint32_t lookup = LOOKUP_DEFAULT;
};

// The membership test of block kernel k (0: mid owners, 1: large owners)
// under lookup, for the schedule descriptions; and the lookup field with
// kernel k's bits set to v (0 hash set, 1 binary search, 4 bitmap).
inline const char *lookup_name(uint32_t lookup, int k)
{
    const uint32_t m = lookup >> k;
    return (m & 1u) ? "binary search"
                    : ((m & 4u) ? (k ? "rank-window bitmap, else binary search" : "rank-window bitmap, else hash set")
                                : "hash set");
}
inline uint32_t lookup_with(uint32_t lookup, int k, uint32_t v) { return (lookup & ~(5u << k)) | (v << k); }

struct CountBuffers {
    const uint64_t *ekey;   // canonical keys [m]
    uint64_t m;
    uint32_t n;
    uint32_t *deg;          // [n]
    uint8_t *heavy;         // [n]
    uint32_t *rowptr;       // [n + 1]
    uint32_t *col;          // padded CSR columns (see SENT / ptrp)
    uint32_t *ptrp;         // [n + 2] padded row pointers
    uint32_t *inptr;        // [n + 1] in-list starts
    uint32_t *inend;        // [n] in-list ends
    const uint2 *inlist;    // in-list entries (source, padded position of the edge)
    const uint2 *olist;     // out-lists (RowsArgs::olist)
    const uint32_t *ocnt;   // [n]
    uint64_t *items;        // owner work items [items_cap]
    uint64_t items_cap;
    DevState *st;
    BatchView bv;           // k > 0: the graph is a batch union
    IsectConfig cfg;        // intersection schedule
    uint32_t core_base = 0xffffffffu;  // base of the dense core of this count (see CoreBuffers), or none
    // single graph with static rows: kept out-degrees sit in rowptr, in-degrees
    // of the candidates in spread (or static when all_kept), inptr the static
    // reservations
    bool static_rows = false, all_kept = false;
    uint32_t *spread = nullptr;
    // single graph: partition on the whole graph's degrees (deg^2 > m_orig)
    // when frow is set, else on the sample's
    const uint32_t *frow = nullptr;
    uint64_t m_orig = 0;
};

void partition(const CountBuffers &b, cudaStream_t s);
// Capacity (entries) of the owner work-item array for a graph of n, m.
uint64_t items_capacity(uint32_t n, uint64_t m);
void build_items(const CountBuffers &b, cudaStream_t s);
// dyn_smem_bytes: shared memory of the hash table for owners with d+ > 1024
void intersect(const CountBuffers &b, int dyn_smem_bytes, cudaStream_t s);
// Raise the launch limit that intersect needs (called by intersect; call it
// ahead of a stream capture so that the capture contains stream work only).
void intersect_prepare(int dyn_smem_bytes);
void finalize(const CountBuffers &b, double p, tc_result *out_dev, cudaStream_t s);
// batch union: one tc_result per graph, p_dev[k] the graphs' sampling rates
void finalize_batch(const CountBuffers &b, const double *p_dev, tc_result *out_dev, cudaStream_t s);

// ---------------------------------------------------------------- batch.cu
// Device buffers of one batched count over a union of up to m_cap edges,
// n_cap vertices and k_cap graphs (batch.cu, server.cu).
struct UnionScratch {
    uint64_t m_cap = 0;
    uint32_t n_cap = 0, k_cap = 0;
    uint64_t *rel = nullptr, *orig = nullptr;  // union keys in rank ids (sorted) and their original keys
    uint2 *inlist = nullptr;
    uint2 *olist = nullptr;
    uint32_t *ocnt = nullptr;
    uint64_t *items = nullptr;
    uint64_t items_cap = 0;
    uint32_t *deg = nullptr, *rowptr = nullptr, *inptr = nullptr, *hist = nullptr, *scan = nullptr;
    uint32_t *colp = nullptr, *ptrp = nullptr, *keepw = nullptr, *tile_cnt = nullptr, *spread = nullptr;
    uint32_t *inend = nullptr;
    uint8_t *heavy = nullptr;
    DevState *st = nullptr;
    uint64_t *eoff = nullptr, *thr = nullptr, *seed_mix = nullptr;
    uint32_t *voff = nullptr;
    double *p = nullptr;
    unsigned long long *counters = nullptr;  // m_p[k_cap], t_light[k_cap], t_heavy[k_cap], n_heavy[k_cap] (u32)
    tc_result *res_dev = nullptr;
    int smem_bytes = 0;
};
// Allocates every buffer (cudaMalloc); false on failure (allocs keeps what
// was allocated, bytes the total).
bool union_scratch_alloc(UnionScratch &u, uint64_t m_cap, uint32_t n_cap, uint32_t k_cap, std::vector<void *> &allocs,
                         uint64_t &bytes);
// Union of resident graphs: rel / orig [m] <- graph g's rank-order keys
// rel_src[g] and original keys orig_src[g] (device pointer arrays, k
// entries), shifted by voff[g]; eoff / voff as for BatchView.
void gather_graphs(const uint64_t *const *rel_src, const uint64_t *const *orig_src, const uint64_t *eoff,
                   const uint32_t *voff, uint32_t k, uint64_t m, uint64_t *rel, uint64_t *orig, cudaStream_t s);
// The count of k graphs whose union (m edges, n vertices) sits in u.rel /
// u.orig (rank order, see csr.cu), with u.eoff / u.voff / u.thr /
// u.seed_mix / u.p filled: per-graph results land in u.res_dev.
void union_count(UnionScratch &u, uint64_t m, uint32_t n, uint32_t k, const IsectConfig &cfg, cudaStream_t s);

// ---------------------------------------------------------------- heavy.cu
// Dense heavy block: U and U^T (hcap x hcap fp8, row stride hcap), the
// heavy vertex list and each heavy vertex's dense index, and the TMA
// descriptors of U and U^T (CUtensorMap storage).  hcap == 0 disables the
// dense path (the intersection kernels then count the heavy class).
// U and U^T hold 0 and 1 as fp8 e4m3 bytes (1.0 = 0x38): the tensor cores
// multiply them exactly (fp32 sums of at most 65536 ones: hcap <= 32768 for
// the heavy block, <= 65536 for the core).
constexpr uint8_t TC_ONE = 0x38;
struct HeavyBuffers {
    uint8_t *U = nullptr;
    uint8_t *UT = nullptr;
    uint32_t hcap = 0;
    uint32_t *hlist = nullptr;
    uint32_t hlist_cap = 0;
    uint32_t *hidx = nullptr;  // [n]
    alignas(64) unsigned char mapA[128];
    alignas(64) unsigned char mapB[128];
};

bool heavy_make_maps(HeavyBuffers &hb);
// The dense core: the vertices with the top n - base ids (ranks), at most
// hcap of them (a count may use fewer than the graph allocated); U (row
// stride hcap) is their strictly upper 0/1 matrix, U[v - base][w - base] = 1
// for every kept edge v -> w inside the core.  Every triangle whose lowest
// vertex is in the core lies in the core, so when the core block runs
// (DevState::core_on) the intersection kernels skip the pairs whose lower
// endpoint is in it and the contraction counts those triangles (t_core).
struct CoreBuffers {
    HeavyBuffers hb;  // hlist / hidx unused; hcap = core size
    uint32_t base = 0;
};
// after the CSR: list, rank and pack the heavy vertices; sets DevState::dense,
// and DevState::core_on when core (may be NULL) is to run for this count
// Decides DevState::dense and core_on right after the partition (before the
// compaction, which leaves out the pairs these blocks count).
void heavy_decide(const CountBuffers &b, const HeavyBuffers &hb, const CoreBuffers *core, cudaStream_t s);
// Runs the tensor kernels' bounded mbarrier wait on a barrier nothing
// arrives at, for limit_us: 1 when it gave up (as it must), 0 when it
// completed, -1 on a CUDA error.
int wait_check(uint32_t limit_us);
void heavy_prepare(const CountBuffers &b, const HeavyBuffers &hb, const CoreBuffers *core, cudaStream_t s);
// T_H += sum_{i<k} U_ik (U U)_ik on tcgen05 (no-op unless DevState::dense),
// and t_core likewise over the core matrix when DevState::core_on
void heavy_contract(const CountBuffers &b, const HeavyBuffers &hb, const CoreBuffers *core, cudaStream_t s);

// ---------------------------------------------------------------- triples.cu
// Triple sampling (Sections 3.2-3.3) over the symmetric adjacency of a graph
// in its original ids (see triples.cu for U and the estimator).
struct TripleDev {
    unsigned long long m_p, universe, samples, closed_wedge, closed_path;
    unsigned int n_heavy, nlist, err, pad;
};
struct TripleBuffers {
    uint32_t n = 0;
    uint64_t m = 0;
    uint32_t *soff = nullptr;   // [n + 1] the whole graph: row offsets of the symmetric adjacency
    uint32_t *snbr = nullptr;   // [2 m] neighbours, every row sorted by id
    uint32_t *off_p = nullptr;  // [n + 1] the same for the sample of a count (p < 1)
    uint32_t *nbr_p = nullptr;  // [2 m]
    uint32_t *qpre = nullptr;   // [2 m] heavy rows: 2-paths through the earlier neighbours
    unsigned long long *cnt = nullptr;     // [n + 1] triples per vertex, then their exclusive prefix
    unsigned long long *scan64 = nullptr;  // scan scratch for n + 1 (64-bit)
    uint32_t *scan32 = nullptr;            // scan scratch for n + 1 (32-bit)
    uint32_t *hlist = nullptr;  // heavy vertices of a count [hcap]
    uint32_t hcap = 0;          // > the number of heavy vertices of any sample (2 m^(1/2) + 2)
    TripleDev *dev = nullptr;
    tc_triple_result *res = nullptr;
};
// soff / snbr from the m original keys (any order); tmpA / tmpB hold 2 m
// keys each, hist / scan the radix scratch for 2 m items; nbits covers n.
void triples_build(const uint64_t *orig, uint64_t m, uint32_t n, int nbits, TripleBuffers &tb, uint64_t *tmpA,
                   uint64_t *tmpB, uint32_t *hist, uint32_t *scan, cudaStream_t s);
// One triple-sampling count into *out_dev (thr >= 2^53: every edge kept).
void triples_count(const TripleBuffers &tb, uint64_t seed_mix, uint64_t thr, uint64_t seed, uint64_t samples,
                   bool hybrid, double p, tc_triple_result *out_dev, cudaStream_t s);

// ---------------------------------------------------------------- stream.cu
// Section 5.2's three passes over a host-resident adjacency stream (see
// stream.cu); res receives everything but ms.  Blocks.
tc_status stream_count(const uint64_t *off_host, const uint32_t *adj_host, uint32_t n, uint64_t seed,
                       uint64_t samples, double c, uint64_t chunk_entries, cudaStream_t s, tc_stream_result *res);

}  // namespace tcg
