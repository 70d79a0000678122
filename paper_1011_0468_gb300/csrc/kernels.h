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
// scan_scratch_elems(len) uint32.  With dyn_items non-NULL only the first
// dyn_bins * ceil(*dyn_items / RX_TILE) elements (at most len) are scanned:
// the digit histograms of a radix pass over a device-counted item list.
void scan_excl_u32(uint32_t *a, uint64_t len, uint32_t *total, uint32_t *scratch, cudaStream_t s,
                   const unsigned long long *dyn_items = nullptr, uint32_t dyn_bins = 0);

// Source of the items of a radix pass.
struct ItemSource {
    // PLAIN: items as they are; SAMPLE_ORIENT: canonical keys, kept ones
    // oriented; ORIENT: canonical keys already sampled, all oriented
    enum Kind { PLAIN = 0, SAMPLE_ORIENT = 1, ORIENT = 2 } kind;
    const uint64_t *in;                 // PLAIN: items; SAMPLE_ORIENT / ORIENT: canonical keys
    uint64_t n_host;                    // item count when n_dev is NULL
    const unsigned long long *n_dev;    // device item count (e.g. m_p), or NULL
    const uint32_t *deg;                // SAMPLE_ORIENT / ORIENT: sampled degrees
    uint64_t seed_mix, thr;             // SAMPLE_ORIENT: keep test (single graph)
    BatchView bv;                       // SAMPLE_ORIENT over a batch union (bv.k > 0)
};

// Optional by-product of the last radix pass over oriented edges
// (src << 32 | dst): the in-lists, every pair appended to its dst's list.  P
// has n + 2 entries; on entry P[0] = 0 and P[1 + v] = the start of v's
// in-list; afterwards the in-list of vertex v is inlist[P[v] .. P[v + 1])
// (in no particular order).
struct InListArgs {
    uint32_t *P;
    uint32_t *inlist;
    uint32_t n;
};

// One stable LSD radix pass over 64-bit items on bits [shift, shift+width),
// width <= 8.  Tiles of RX_TILE items; hist holds (1 << width) * ntiles
// uint32 (digit-major), ntiles = ceil(n_max / RX_TILE).  If dplus is
// non-NULL the count kernel also histograms (item >> 32) into it.  The
// scatter writes the full items to out, or when out_low32 is non-NULL only
// their low 32 bits there, at position + padoff[item >> 32] when padoff is
// non-NULL.  With `in` non-NULL the scatter also fills the in-lists
// described above.
void radix_pass(const ItemSource &src, uint64_t n_max, int shift, int width, uint32_t *hist,
                uint32_t *scan_scratch, uint32_t *dplus, uint64_t *out, uint32_t *out_low32,
                const InListArgs *in, cudaStream_t s, const uint32_t *padoff = nullptr);

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

// Degree-oriented CSR of the sampled graph (single graph or batch union):
// stable LSD radix sort of (src << 32 | dst) on the src bits (at least two
// passes), the first pass sampling and orienting the canonical keys, the
// last one also filling the in-lists (every kept edge, under its dst; their
// sizes deg - d+ are known after the first pass) and writing the columns
// straight into the padded layout.  rowptr [n + 1] and inptr [n + 2] are zeroed here;
// *col = colp (padded columns, colp_capacity entries), ptrp [n + 2] its row
// pointers, and the in-lists are placed in bufA / bufB.
struct CsrArgs {
    const uint64_t *ekey;
    uint64_t m;
    uint32_t n;
    int nbits;  // bits of a vertex id
    const uint32_t *deg;
    uint64_t seed_mix, thr;  // single graph
    BatchView bv;            // batch union (bv.k > 0)
    const unsigned long long *m_sampled_dev;
    uint64_t *bufA, *bufB;
    uint32_t *rowptr, *inptr, *hist, *scan;
    uint32_t *colp, *ptrp;
    // NULL, or the kept keys already compacted in canonical order
    // (m_sampled_dev of them, not in bufA): the first pass then only orients
    const uint64_t *kept = nullptr;
};
void csr_build(const CsrArgs &a, uint32_t **col, uint32_t **inlist, cudaStream_t s);

// Canonical keys from raw pairs: (min << 32 | max), self-loops become
// ~0ull; endpoints >= n raise ERR_ENDPOINT; pairs that are not strictly
// increasing in order are counted into st->unsorted.
void canon_keys(const uint32_t *pairs, uint64_t m_in, uint32_t n, uint64_t *keys, DevState *st,
                cudaStream_t s);

// Stable removal of repeats and ~0ull from sorted keys; the count goes to
// st->m_canon.  tile_cnt holds ceil(m_in / RX_TILE) + 1 uint32.
void unique_keys(const uint64_t *keys, uint64_t m_in, uint64_t *out, uint32_t *tile_cnt,
                 uint32_t *scan_scratch, DevState *st, cudaStream_t s);

// ---------------------------------------------------------------- count.cu
// Schedule of the intersection kernels (isect.cu); any choice gives the same
// counts.  warp_max: owners with 2 <= d+ <= warp_max are resolved by one warp
// (32 .. 256); seg_w / seg_b: most partners per work item of the warp / block
// kernels (seg_w in [SEG_MIN, 1024], seg_b in [256, 2048], powers of two);
// work_w / work_b: an owner of out-degree d gets items of the largest power
// of two <= seg_w (seg_b) partners with partners * d <= work_w (work_b), but
// at least SEG_MIN (256), which bounds the list entries an item streams.
constexpr uint32_t SEG_MIN = 64;
struct IsectConfig {
    uint32_t warp_max = 256;
    uint32_t seg_w = 512;
    uint32_t seg_b = 2048;
    uint32_t work_w = 1u << 14;
    uint32_t work_b = 1u << 19;
};

struct CountBuffers {
    const uint64_t *ekey;   // canonical keys [m]
    uint64_t m;
    uint32_t n;
    uint32_t *deg;          // [n]
    uint8_t *heavy;         // [n]
    uint32_t *rowptr;       // [n + 1]
    uint32_t *col;          // padded CSR columns (see SENT / ptrp)
    uint32_t *ptrp;         // [n + 2] padded row pointers
    uint32_t *inptr;        // [n + 2] in-list offsets
    uint32_t *inlist;       // in-lists
    uint64_t *items;        // owner work items [items_cap]
    uint64_t items_cap;
    DevState *st;
    BatchView bv;           // k > 0: the graph is a batch union
    IsectConfig cfg;        // intersection schedule
};

// Sampling and sampled degrees.  With tile_cnt non-NULL (single graph only)
// the kept edges of every RX_TILE-key tile are also counted there.
void sample_degree(const CountBuffers &b, uint64_t seed_mix, uint64_t thr, cudaStream_t s,
                   uint32_t *tile_cnt = nullptr);
// After sample_degree with tile_cnt: the kept keys, in canonical order, to
// out (tile_cnt is scanned in place; scan_scratch as for scan_excl_u32).
void kept_scatter(const CountBuffers &b, uint64_t seed_mix, uint64_t thr, uint64_t *out, uint32_t *tile_cnt,
                  uint32_t *scan_scratch, cudaStream_t s);
void partition(const CountBuffers &b, cudaStream_t s);
void compact_kept(const CountBuffers &b, uint64_t seed_mix, uint64_t thr, uint64_t *out,
                  uint32_t *tile_cnt, uint32_t *scan_scratch, cudaStream_t s);
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
    uint64_t *ekey = nullptr, *bufA = nullptr, *bufB = nullptr, *items = nullptr;
    uint64_t items_cap = 0;
    uint32_t *deg = nullptr, *rowptr = nullptr, *inptr = nullptr, *hist = nullptr, *scan = nullptr;
    uint32_t *colp = nullptr, *ptrp = nullptr;
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
// The count of k graphs whose union (m edges, n vertices) sits in u.ekey,
// with u.eoff / u.voff / u.thr / u.seed_mix / u.p filled: per-graph results
// land in u.res_dev.
void union_count(UnionScratch &u, uint64_t m, uint32_t n, uint32_t k, const IsectConfig &cfg, cudaStream_t s);

// ---------------------------------------------------------------- heavy.cu
// Dense heavy block: U and U^T (hcap x hcap bf16, row stride hcap), the
// heavy vertex list and each heavy vertex's dense index, and the TMA
// descriptors of U and U^T (CUtensorMap storage).  hcap == 0 disables the
// dense path (the intersection kernels then count the heavy class).
struct HeavyBuffers {
    uint16_t *U = nullptr;
    uint16_t *UT = nullptr;
    uint32_t hcap = 0;
    uint32_t *hlist = nullptr;
    uint32_t hlist_cap = 0;
    uint32_t *hidx = nullptr;  // [n]
    alignas(64) unsigned char mapA[128];
    alignas(64) unsigned char mapB[128];
};

bool heavy_make_maps(HeavyBuffers &hb);
// after the CSR: list, rank and pack the heavy vertices; sets DevState::dense
void heavy_prepare(const CountBuffers &b, const HeavyBuffers &hb, cudaStream_t s);
// T_H += sum_{i<k} U_ik (U U)_ik on tcgen05 (no-op unless DevState::dense)
void heavy_contract(const CountBuffers &b, const HeavyBuffers &hb, cudaStream_t s);

}  // namespace tcg
