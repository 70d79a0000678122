// tc_count_noalloc: the whole count for small graphs without any device
// allocation.
//
// Some callers cannot call cudaMalloc: a host framework whose memory pool
// already owns the device memory (a second allocator would fragment it or
// fail), code that runs where a device allocation would synchronise the GPU
// or is simply not permitted (latency-critical loops, plugin hosts that only
// hand out buffers).  For them this entry point keeps all its scratch in one
// file-scope __device__ array of fixed size, which every GPU that loads the
// library holds until the process exits.  The caller passes the edge list
// (device memory) and receives the result in host memory.
//
// The array is shared by all calls: each call clears what must start at
// zero, and calls that overlap on the GPU (different streams or host
// threads) race on it.
#include <mutex>
#include <utility>

#include "kernels.h"

namespace {

using namespace tcg;

constexpr uint64_t NA_M = TC_NOALLOC_MAX_EDGES;
constexpr uint64_t NA_N = TC_NOALLOC_MAX_VERTICES;
constexpr uint64_t NA_ALIGN = 256;
constexpr uint64_t na_round(uint64_t b) { return (b + NA_ALIGN - 1) / NA_ALIGN * NA_ALIGN; }
constexpr uint64_t NA_TILES = (NA_M + RX_TILE - 1) / RX_TILE;
constexpr uint64_t NA_HIST = NA_TILES << RX_MAX_BITS;  // uint32 entries
constexpr uint64_t NA_SCAN = 2 * ((NA_HIST > NA_N + 2 ? NA_HIST : NA_N + 2) / SC_CHUNK + 2);
constexpr uint64_t NA_ITEMS = NA_N + 2 * NA_M / SEG_MIN + NA_M / 512 + 2 * NA_M / 256 + 256;  // >= items_capacity(N, M)
constexpr uint64_t NA_COLP = NA_M + 3 * NA_M + 4;  // >= colp_capacity(N, M)
static_assert(NA_N <= NA_M, "the vertex sort reuses the key buffers");
// A rank-order row (out-degree d of the degree order) has d(d - 1) / 2 <= m,
// so with m <= NA_M every row has fewer than NA_DMAX keys: at most ROW_MID,
// the rows one warp sorts in registers.  The long-row path of the relabeling
// (which would use RelabelScratch::kB as global scratch, here the same
// memory as other buffers) is therefore never taken.
constexpr uint64_t NA_DMAX = 725;
static_assert(NA_DMAX * (NA_DMAX - 1) / 2 > NA_M, "rows stay below NA_DMAX keys");
static_assert(NA_DMAX <= ROW_MID, "every row is sorted by the warp path");
constexpr uint64_t NA_BYTES = 4 * na_round(8 * NA_M)                     // ekey (then rel), orig, bufA, bufB
                              + 5 * na_round(4 * NA_N)                   // perm, rank, spread, inend, ocnt
                              + na_round(4 * (NA_M / 32 + 1)) + na_round(4 * (NA_TILES + 1))  // keepw, tile_cnt
                              + na_round(4 * NA_HIST) + na_round(4 * NA_SCAN)
                              + 2 * na_round(4 * (NA_N + 2))             // deg, rowptr
                              + na_round(NA_N)                           // heavy
                              + na_round(4 * (NA_N + 2))                 // inptr
                              + na_round(4 * NA_COLP) + na_round(4 * (NA_N + 2))  // colp, ptrp
                              + na_round(8 * NA_ITEMS) + na_round(sizeof(DevState)) + na_round(sizeof(tc_result));

static __device__ __align__(256) unsigned char g_na_scratch[NA_BYTES];

// Device address of g_na_scratch per device, looked up once per device (the
// host-side symbol is only a stand-in, never a device address).
std::mutex g_na_mutex;
void *g_na_addr[64] = {};

tc_status na_scratch(void **out)
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    std::lock_guard<std::mutex> lock(g_na_mutex);
    if (!g_na_addr[dev]) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_na_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return TC_ECUDA;
        }
        g_na_addr[dev] = p;
    }
    *out = g_na_addr[dev];
    return TC_OK;
}

struct Carver {
    unsigned char *p;
    uint64_t used = 0;
    template <typename T>
    T *take(uint64_t count)
    {
        T *r = reinterpret_cast<T *>(p + used);
        used += na_round(count * sizeof(T));
        return r;
    }
};

int na_bits(uint32_t n)
{
    int b = 1;
    while (b < 32 && (1ull << b) < n) ++b;
    return b;
}

// Digit widths of the radix passes over `bits` bits (at most 8 each, as even
// as possible).  Returns the pass count.
int na_widths(int bits, int w[4])
{
    const int P = (bits + RX_MAX_BITS - 1) / RX_MAX_BITS;
    for (int i = 0; i < P; ++i) w[i] = bits / P + (i < bits % P ? 1 : 0);
    return P;
}

}  // namespace

extern "C" tc_status tc_count_noalloc(const uint32_t *edges_dev, uint64_t m_in, uint32_t n, double p, uint64_t seed,
                                      tc_result *out_host, void *cuda_stream)
{
    if (!out_host || n == 0 || (m_in > 0 && !edges_dev) || !(p > 0.0 && p <= 1.0)) return TC_EINVAL;
    if (m_in > NA_M || n > NA_N) return TC_EINVAL;
    void *base = nullptr;
    tc_status status = na_scratch(&base);
    if (status != TC_OK) return status;
    cudaStream_t s = (cudaStream_t)cuda_stream;

    Carver c{(unsigned char *)base};
    uint64_t *ekey = c.take<uint64_t>(NA_M);
    uint64_t *orig = c.take<uint64_t>(NA_M);
    uint32_t *perm = c.take<uint32_t>(NA_N);
    uint32_t *rank = c.take<uint32_t>(NA_N);
    uint32_t *spread = c.take<uint32_t>(NA_N);  // hot_size(n) <= NA_N
    uint32_t *inend = c.take<uint32_t>(NA_N);
    uint32_t *ocnt = c.take<uint32_t>(NA_N);
    uint32_t *keepw = c.take<uint32_t>(NA_M / 32 + 1);
    uint32_t *tile_cnt = c.take<uint32_t>(NA_TILES + 1);
    uint64_t *bufA = c.take<uint64_t>(NA_M);
    uint64_t *bufB = c.take<uint64_t>(NA_M);
    uint32_t *hist = c.take<uint32_t>(NA_HIST);
    uint32_t *scan = c.take<uint32_t>(NA_SCAN);
    uint32_t *deg = c.take<uint32_t>(NA_N + 2);
    uint32_t *rowptr = c.take<uint32_t>(NA_N + 2);
    uint8_t *heavy = c.take<uint8_t>(NA_N);
    uint32_t *inptr = c.take<uint32_t>(NA_N + 2);
    uint32_t *colp = c.take<uint32_t>(NA_COLP);
    uint32_t *ptrp = c.take<uint32_t>(NA_N + 2);
    uint64_t *items = c.take<uint64_t>(NA_ITEMS);
    DevState *st = c.take<DevState>(1);
    tc_result *res = c.take<tc_result>(1);
    if (c.used > NA_BYTES || items_capacity(n, m_in) > NA_ITEMS || colp_capacity(n, m_in) > NA_COLP) return TC_ECUDA;

    // ---- canonical keys: (min, max), no self-loops or repeats, sorted
    cudaMemsetAsync(st, 0, sizeof(DevState), s);
    DevState hs;
    uint64_t m = 0;
    if (m_in > 0) {
        canon_keys(edges_dev, m_in, n, bufA, st, s);
        uint64_t *a = bufA, *b = bufB;
        const int nbits = na_bits(n);
        for (int half = 0; half < 2; ++half) {
            int shift = half ? 32 : 0;
            int wd[4];
            const int np = na_widths(nbits, wd);
            for (int k = 0; k < np; ++k) {
                const int w = wd[k];
                radix_pass(a, m_in, shift, w, hist, scan, b, s);
                std::swap(a, b);
                shift += w;
            }
        }
        unique_keys(a, m_in, ekey, hist, scan, st, s);
        if (cudaMemcpyAsync(&hs, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
            cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            return TC_ECUDA;
        }
        if (hs.err & ERR_ENDPOINT) return TC_EINVAL;
        m = hs.m_canon;
    }

    // ---- rank relabeling (csr.cu): rel keys replace the canonical keys; the
    // vertex sort and the key sort both ping-pong between bufA and bufB.  The
    // long-row scratch (kB = bufB) is never touched: see NA_DMAX.
    relabel(ekey, m, n, nullptr, 0, Relabeled{ekey, orig, perm, rank},
            RelabelScratch{bufA, bufB, bufA, bufB, deg, hist, scan}, s);

    // ---- the count (Sections 3.1-3.2), every buffer inside the array
    const uint64_t seed_mix = splitmix64(seed), thr = (uint64_t)(p * 9007199254740992.0);
    CountBuffers cb;
    cb.ekey = ekey;
    cb.m = m;
    cb.n = n;
    cb.deg = deg;
    cb.heavy = heavy;
    cb.rowptr = rowptr;
    cb.col = colp;
    cb.ptrp = ptrp;
    cb.inptr = inptr;
    cb.inend = inend;
    cb.inlist = reinterpret_cast<uint2 *>(bufA);
    cb.olist = reinterpret_cast<uint2 *>(bufB);  // free after the sorts; m <= NA_M entries of 8 bytes
    cb.ocnt = ocnt;
    cb.items = items;
    cb.items_cap = items_capacity(n, m);
    cb.st = st;
    RowsArgs ra;
    ra.rel = ekey;
    ra.orig = orig;
    ra.m = m;
    ra.n = n;
    ra.seed_mix = seed_mix;
    ra.thr = thr;
    ra.deg = deg;
    ra.rowptr = rowptr;
    ra.inptr = inptr;
    ra.inend = inend;
    ra.ptrp = ptrp;
    ra.colp = colp;
    ra.inlist = reinterpret_cast<uint2 *>(bufA);
    ra.olist = reinterpret_cast<uint2 *>(bufB);
    ra.ocnt = ocnt;
    ra.heavy = heavy;
    ra.keepw = keepw;
    ra.tile_cnt = tile_cnt;
    ra.scan = scan;
    ra.spread = spread;
    ra.st = st;
    cudaMemsetAsync(st, 0, sizeof(DevState), s);
    sample_rows(ra, s);
    partition(cb, s);
    if (m > 0) {
        build_rows(ra, s);
        build_items(cb, s);
        // every out-degree is at most sqrt(2 m) <= 725 here: the smallest
        // table of the large-owner kernel (8192 slots) always suffices
        intersect(cb, 8192 * 4, s);
    }
    finalize(cb, p, res, s);
    if (cudaGetLastError() != cudaSuccess) return TC_ECUDA;  // a launch was rejected
    if (cudaMemcpyAsync(out_host, res, sizeof(tc_result), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaMemcpyAsync(&hs, st, sizeof(DevState), cudaMemcpyDeviceToHost, s) != cudaSuccess ||
        cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    if (hs.err & ERR_ENDPOINT) return TC_EINVAL;
    if (hs.err) return TC_ECUDA;
    return TC_OK;
}
