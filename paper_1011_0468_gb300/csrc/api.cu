// C ABI of libtc (declared in include/tc.h): graph objects, the order of the
// device phases of one count, and the inspection entry points.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>
#include <vector>

#include "kernels.h"

using namespace tcg;

namespace {

tc_alloc_fn g_alloc = nullptr;
tc_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;

void *dev_alloc(uint64_t bytes, cudaStream_t s)
{
    bytes = std::max<uint64_t>(bytes, 256);
    if (g_alloc) return g_alloc(bytes, s, g_alloc_ctx);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(void *p, cudaStream_t s)
{
    if (!p) return;
    if (g_free)
        g_free(p, s, g_alloc_ctx);
    else
        cudaFree(p);
}

int bits_for(uint32_t n)
{
    int b = 1;
    while (b < 32 && (1ull << b) < n) ++b;
    return b;
}

// Split `bits` into the fewest passes of at most RX_MAX_BITS, as even as
// possible.
std::vector<int> pass_widths(int bits)
{
    const int P = (bits + RX_MAX_BITS - 1) / RX_MAX_BITS;
    std::vector<int> w(P, bits / P);
    for (int i = 0; i < bits % P; ++i) w[i]++;
    return w;
}

constexpr int NUM_EVENTS = 6;

std::atomic<unsigned long long> g_launches{0};

}  // namespace

void tcg::note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
void tcg::add_launches(unsigned long long n) { g_launches.fetch_add(n, std::memory_order_relaxed); }

struct tc_graph {
    uint32_t n = 0;
    uint64_t m = 0;
    int nbits = 1;
    cudaStream_t stream = nullptr;
    int timing = 0;
    int smem_bytes = 0;
    uint64_t bytes = 0;
    // device
    uint64_t *ekey = nullptr;   // canonical keys (u << 32 | v), sorted [m]
    uint64_t *bufA = nullptr;   // radix ping-pong [m]
    uint64_t *bufB = nullptr;   // radix ping-pong [m]
    uint32_t *deg = nullptr;    // [n]
    uint32_t *rowptr = nullptr; // [n + 1]
    uint8_t *heavy = nullptr;   // [n]
    uint32_t *inptr = nullptr;  // [n + 2] in-list offsets (see InListArgs)
    uint32_t *col = nullptr;    // padded CSR columns (= colp)
    uint32_t *inlist = nullptr; // in-lists (inside bufA or bufB)
    uint32_t *colp = nullptr;   // [colp_capacity(n, m)] rows padded to 16 bytes
    uint32_t *ptrp = nullptr;   // [n + 2] padded row pointers
    uint64_t *items = nullptr;  // owner work items, all buckets [items_cap]
    uint64_t items_cap = 0;
    uint32_t *hist = nullptr;   // [RX_BINS * ntiles(m)]
    uint32_t *scan = nullptr;   // scan scratch
    HeavyBuffers hb;            // dense heavy block (hb.hcap == 0: not used)
    DevState *st = nullptr;
    tc_result *res_dev = nullptr;
    // pinned host
    tc_result *res_host = nullptr;
    DevState *st_host = nullptr;
    // phase-timing ring: TC_TIMING_RING slots of NUM_EVENTS events
    std::vector<cudaEvent_t> ring;
    uint64_t ring_head = 0;  // next slot to record
    uint64_t ring_tail = 0;  // oldest undrained count
    std::vector<void *> allocs;

    void *alloc(uint64_t b)
    {
        void *p = dev_alloc(b, stream);
        if (p) {
            allocs.push_back(p);
            bytes += b;
        }
        return p;
    }
    void release(void *p)
    {
        auto it = std::find(allocs.begin(), allocs.end(), p);
        if (it != allocs.end()) {
            allocs.erase(it);
            dev_free(p, stream);
        }
    }
};

namespace {

void free_graph(tc_graph *g)
{
    if (!g) return;
    cudaStreamSynchronize(g->stream);
    for (void *p : g->allocs) dev_free(p, g->stream);
    g->allocs.clear();
    if (g->res_host) cudaFreeHost(g->res_host);
    if (g->st_host) cudaFreeHost(g->st_host);
    for (auto &e : g->ring) cudaEventDestroy(e);
    cudaGetLastError();
    delete g;
}

tc_status status_of_err(unsigned err)
{
    if (err & ERR_ENDPOINT) return TC_EINVAL;
    if (err & ERR_TIMEOUT) return TC_ETIMEOUT;
    if (err & ERR_OVERFLOW) return TC_ECUDA;
    return TC_OK;
}

bool bad_p(double p) { return !(p > 0.0 && p <= 1.0); }

uint64_t threshold_of(double p) { return (uint64_t)(p * 9007199254740992.0); }

CountBuffers buffers_of(tc_graph *g);

// At sampling rates up to this, the kept edges are compacted first and the
// radix passes run over them alone; above it the first pass samples the
// whole edge list itself.
constexpr double COMPACT_P = 0.5;

// Sampling, degrees and partition (Sections 3.1-3.2) into g->deg/heavy/st;
// with `compact`, also the per-tile kept counts in g->hist.
void enqueue_sample(tc_graph *g, uint64_t seed_mix, uint64_t thr, const CountBuffers &b, bool compact = false)
{
    cudaMemsetAsync(g->st, 0, sizeof(DevState), g->stream);
    cudaMemsetAsync(g->deg, 0, (size_t)g->n * 4, g->stream);
    sample_degree(b, seed_mix, thr, g->stream, compact ? g->hist : nullptr);
    partition(b, g->stream);
}

// Degree-oriented CSR of the sampled graph by stable LSD radix sort of
// (src << 32 | dst) on the src bits, plus the in-lists.  With `compact`
// (after enqueue_sample with compact) the kept keys are gathered into bufB
// first.  Fills g->col / g->inlist / g->inptr.
void enqueue_csr(tc_graph *g, uint64_t seed_mix, uint64_t thr, bool compact = false)
{
    CsrArgs a;
    a.ekey = g->ekey;
    a.m = g->m;
    a.n = g->n;
    a.nbits = g->nbits;
    a.deg = g->deg;
    a.seed_mix = seed_mix;
    a.thr = thr;
    a.m_sampled_dev = &g->st->m_sampled;
    a.bufA = g->bufA;
    a.bufB = g->bufB;
    a.rowptr = g->rowptr;
    a.inptr = g->inptr;
    a.hist = g->hist;
    a.scan = g->scan;
    a.colp = g->colp;
    a.ptrp = g->ptrp;
    if (compact) {
        kept_scatter(buffers_of(g), seed_mix, thr, g->bufB, g->hist, g->scan, g->stream);
        a.kept = g->bufB;
    }
    csr_build(a, &g->col, &g->inlist, g->stream);
}

CountBuffers buffers_of(tc_graph *g)
{
    CountBuffers b;
    b.ekey = g->ekey;
    b.m = g->m;
    b.n = g->n;
    b.deg = g->deg;
    b.heavy = g->heavy;
    b.rowptr = g->rowptr;
    b.col = g->col;
    b.ptrp = g->ptrp;
    b.inptr = g->inptr;
    b.inlist = g->inlist;
    b.items = g->items;
    b.items_cap = g->items_cap;
    b.st = g->st;
    return b;
}

cudaEvent_t &ring_event(tc_graph *g, uint64_t count, int i)
{
    return g->ring[(count % TC_TIMING_RING) * NUM_EVENTS + i];
}

void record(tc_graph *g, bool timing, int i)
{
    if (timing) cudaEventRecord(ring_event(g, g->ring_head, i), g->stream);
}

// Phase times of one recorded count, layout of tc_result.ms.
void ring_times(tc_graph *g, uint64_t count, float *ms)
{
    const int pairs[5][2] = {{0, 1}, {1, 2}, {2, 3}, {3, 4}, {0, 5}};
    for (int i = 0; i < 8; ++i) ms[i] = 0.0f;
    for (int i = 0; i < 5; ++i) {
        float t;
        if (cudaEventElapsedTime(&t, ring_event(g, count, pairs[i][0]), ring_event(g, count, pairs[i][1])) ==
            cudaSuccess)
            ms[i] = t;
    }
    cudaGetLastError();
}

tc_status enqueue_count(tc_graph *g, double p, uint64_t seed, tc_result *dst, bool timing)
{
    const uint64_t seed_mix = splitmix64(seed), thr = threshold_of(p);
    const bool compact = p <= COMPACT_P;
    CountBuffers b = buffers_of(g);
    record(g, timing, 0);
    enqueue_sample(g, seed_mix, thr, b, compact);
    record(g, timing, 1);
    if (g->m > 0) {
        enqueue_csr(g, seed_mix, thr, compact);
        b = buffers_of(g);
        if (g->hb.hcap) heavy_prepare(b, g->hb, g->stream);
        build_items(b, g->stream);
    }
    record(g, timing, 2);
    if (g->m > 0) intersect(b, g->smem_bytes, g->stream);
    record(g, timing, 3);
    if (g->m > 0 && g->hb.hcap) heavy_contract(b, g->hb, g->stream);
    record(g, timing, 4);
    finalize(b, p, g->res_dev, g->stream);
    record(g, timing, 5);
    if (timing) {
        g->ring_head++;
        if (g->ring_head - g->ring_tail > TC_TIMING_RING) g->ring_tail = g->ring_head - TC_TIMING_RING;
    }
    cudaMemcpyAsync(dst, g->res_dev, sizeof(tc_result), cudaMemcpyDeviceToHost, g->stream);
    cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream);
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ECUDA;
}

tc_status sync_graph(tc_graph *g)
{
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    return status_of_err(g->st_host->err);
}

}  // namespace

extern "C" {

void tc_set_allocator(tc_alloc_fn alloc, tc_free_fn free_fn, void *ctx)
{
    if (alloc && free_fn) {
        g_alloc = alloc;
        g_free = free_fn;
        g_alloc_ctx = ctx;
    } else {
        g_alloc = nullptr;
        g_free = nullptr;
        g_alloc_ctx = nullptr;
    }
}

const char *tc_status_str(tc_status s)
{
    switch (s) {
    case TC_OK: return "ok";
    case TC_EINVAL: return "invalid argument";
    case TC_ENOMEM: return "out of memory";
    case TC_ECUDA: return "CUDA error";
    case TC_ETIMEOUT: return "device wait timed out";
    case TC_EBUSY: return "busy";
    }
    return "unknown status";
}

int tc_version(void) { return 100; }

uint64_t tc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

tc_status tc_graph_create(const uint32_t *edges, uint64_t m_in, uint32_t n, int edges_on_device,
                          void *cuda_stream, tc_graph **out)
{
    if (!out) return TC_EINVAL;
    *out = nullptr;
    if (n == 0 || n == 0xffffffffu || (m_in > 0 && !edges) || m_in > 0xfffffffeull) return TC_EINVAL;

    tc_graph *g = new (std::nothrow) tc_graph;
    if (!g) return TC_ENOMEM;
    g->n = n;
    g->nbits = bits_for(n);
    g->stream = (cudaStream_t)cuda_stream;
    cudaStream_t s = g->stream;

    if (cudaMallocHost((void **)&g->res_host, sizeof(tc_result)) != cudaSuccess ||
        cudaMallocHost((void **)&g->st_host, sizeof(DevState)) != cudaSuccess) {
        cudaGetLastError();
        free_graph(g);
        return TC_ENOMEM;
    }
    g->st = (DevState *)g->alloc(sizeof(DevState));
    g->res_dev = (tc_result *)g->alloc(sizeof(tc_result));
    if (!g->st || !g->res_dev) {
        free_graph(g);
        return TC_ENOMEM;
    }
    cudaMemsetAsync(g->st, 0, sizeof(DevState), s);

    // ---- canonical keys
    uint64_t m = 0;
    if (m_in > 0) {
        const uint32_t *dpairs = edges;
        void *tmp_pairs = nullptr;
        if (!edges_on_device) {
            tmp_pairs = g->alloc(m_in * 8);
            if (!tmp_pairs) { free_graph(g); return TC_ENOMEM; }
            cudaMemcpyAsync(tmp_pairs, edges, m_in * 8, cudaMemcpyHostToDevice, s);
            dpairs = (const uint32_t *)tmp_pairs;
        }
        uint64_t *keys = (uint64_t *)g->alloc(m_in * 8);
        if (!keys) { free_graph(g); return TC_ENOMEM; }
        canon_keys(dpairs, m_in, n, keys, g->st, s);
        cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); free_graph(g); return TC_ECUDA; }
        if (tmp_pairs) g->release(tmp_pairs);
        if (g->st_host->err & ERR_ENDPOINT) { free_graph(g); return TC_EINVAL; }
        if (g->st_host->unsorted == 0) {
            g->ekey = keys;  // already canonical: every pair u < v, strictly increasing
            m = m_in;
        } else {
            // sort by (u, v) on the used bits only, then drop repeats/self-loops
            uint64_t *keys2 = (uint64_t *)g->alloc(m_in * 8);
            const uint64_t nt = ceil_div(m_in, RX_TILE);
            uint32_t *hist = (uint32_t *)g->alloc((nt << RX_MAX_BITS) * 4);
            uint32_t *scan = (uint32_t *)g->alloc(scan_scratch_elems(nt << RX_MAX_BITS) * 4);
            uint32_t *tcnt = (uint32_t *)g->alloc((nt + 1) * 4);
            if (!keys2 || !hist || !scan || !tcnt) { free_graph(g); return TC_ENOMEM; }
            uint64_t *a = keys, *b = keys2;
            for (int half = 0; half < 2; ++half) {
                int shift = half ? 32 : 0;
                for (int w : pass_widths(g->nbits)) {
                    ItemSource src{ItemSource::PLAIN, a, m_in, nullptr, nullptr, 0, 0};
                    radix_pass(src, m_in, shift, w, hist, scan, nullptr, b, nullptr, nullptr, s);
                    std::swap(a, b);
                    shift += w;
                }
            }
            unique_keys(a, m_in, b, tcnt, scan, g->st, s);
            cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); free_graph(g); return TC_ECUDA; }
            m = g->st_host->m_canon;
            g->release(hist);
            g->release(scan);
            g->release(tcnt);
            g->release(a);
            g->ekey = b;
        }
    }
    g->m = m;

    // ---- scratch for counting, sized for p = 1
    const uint64_t nt = std::max<uint64_t>(ceil_div(m, RX_TILE), 1);
    const uint64_t hist_len = nt << RX_MAX_BITS;
    g->bufA = (uint64_t *)g->alloc(std::max<uint64_t>(m, 1) * 8);
    g->bufB = (uint64_t *)g->alloc(std::max<uint64_t>(m, 1) * 8);
    g->deg = (uint32_t *)g->alloc((uint64_t)n * 4);
    g->rowptr = (uint32_t *)g->alloc(((uint64_t)n + 1) * 4);
    g->heavy = (uint8_t *)g->alloc((uint64_t)n);
    g->inptr = (uint32_t *)g->alloc(((uint64_t)n + 2) * 4);
    g->colp = (uint32_t *)g->alloc(colp_capacity(n, m) * 4);
    g->ptrp = (uint32_t *)g->alloc(((uint64_t)n + 2) * 4);
    g->items_cap = items_capacity(n, m);
    g->items = (uint64_t *)g->alloc(g->items_cap * 8);
    g->hist = (uint32_t *)g->alloc(hist_len * 4);
    g->scan = (uint32_t *)g->alloc(scan_scratch_elems(std::max<uint64_t>(hist_len, (uint64_t)n + 1)) * 4);
    if (!g->bufA || !g->bufB || !g->deg || !g->rowptr || !g->heavy || !g->inptr || !g->colp || !g->ptrp ||
        !g->items || !g->hist || !g->scan) {
        free_graph(g);
        return TC_ENOMEM;
    }
    if (m == 0 && !g->ekey) {
        g->ekey = (uint64_t *)g->alloc(8);
        if (!g->ekey) { free_graph(g); return TC_ENOMEM; }
    }
    // hash set of the owners with d+ > 1024: every out-degree of the
    // degree-oriented graph is at most sqrt(2 m_p); a set of >= 4 d+ slots
    // up to 32768 slots (128 KiB) stays on chip, larger rows are searched in
    // place
    const uint64_t dmax = (uint64_t)std::sqrt(2.0 * (double)std::max<uint64_t>(m, 1)) + 2;
    uint64_t slots = 8192;
    while (slots < 4 * dmax && slots < 32768) slots <<= 1;
    g->smem_bytes = (int)(slots * 4);
    // dense heavy block: at most 2 m^(1/2) heavy vertices, padded to the
    // 128-row tile and capped at 32768 (2 x 2 GiB of bf16).  Graphs below
    // 2^20 edges, or without room for the block, have the intersection
    // kernels count the heavy class instead.
    if (m >= (1ull << 20)) {
        const uint64_t hbound = (uint64_t)(2.0 * std::sqrt((double)m)) + 2;
        const uint64_t hcap = std::min<uint64_t>((hbound + 127) / 128 * 128, 32768);
        g->hb.hlist_cap = (uint32_t)hbound;
        g->hb.hlist = (uint32_t *)g->alloc(hbound * 4);
        g->hb.hidx = (uint32_t *)g->alloc((uint64_t)n * 4);
        if (!g->hb.hlist || !g->hb.hidx) {
            free_graph(g);
            return TC_ENOMEM;
        }
        g->hb.U = (uint16_t *)g->alloc(hcap * hcap * 2);
        g->hb.UT = g->hb.U ? (uint16_t *)g->alloc(hcap * hcap * 2) : nullptr;
        g->hb.hcap = (uint32_t)hcap;
        if (!g->hb.U || !g->hb.UT || !heavy_make_maps(g->hb)) {
            if (g->hb.U) g->release(g->hb.U);
            if (g->hb.UT) g->release(g->hb.UT);
            g->hb.U = g->hb.UT = nullptr;
            g->hb.hcap = 0;
        }
    }
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        free_graph(g);
        return TC_ECUDA;
    }
    *out = g;
    return TC_OK;
}

void tc_graph_destroy(tc_graph *g) { free_graph(g); }

uint64_t tc_graph_num_edges(const tc_graph *g) { return g ? g->m : 0; }
uint32_t tc_graph_num_vertices(const tc_graph *g) { return g ? g->n : 0; }
uint64_t tc_graph_device_bytes(const tc_graph *g) { return g ? g->bytes : 0; }

tc_status tc_graph_set_timing(tc_graph *g, int on)
{
    if (!g) return TC_EINVAL;
    if (on && g->ring.empty()) {
        g->ring.resize((size_t)TC_TIMING_RING * NUM_EVENTS);
        for (auto &e : g->ring) {
            if (cudaEventCreate(&e) != cudaSuccess) {
                cudaGetLastError();
                e = nullptr;
                for (auto &f : g->ring)
                    if (f) cudaEventDestroy(f);
                g->ring.clear();
                return TC_ECUDA;
            }
        }
    }
    g->timing = on ? 1 : 0;
    return TC_OK;
}

int tc_graph_timing_drain(tc_graph *g, float *ms_out, uint32_t max_counts)
{
    if (!g || (!ms_out && max_counts)) return -1;
    if (g->ring.empty()) return 0;
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
        cudaGetLastError();
        return -1;
    }
    uint32_t k = 0;
    while (g->ring_tail < g->ring_head && k < max_counts) {
        ring_times(g, g->ring_tail, ms_out + (size_t)k * 8);
        ++g->ring_tail;
        ++k;
    }
    return (int)k;
}

tc_status tc_count(tc_graph *g, double p, uint64_t seed, tc_result *out)
{
    if (!g || !out || bad_p(p)) return TC_EINVAL;
    const bool timing = g->timing != 0 && !g->ring.empty();
    tc_status st = enqueue_count(g, p, seed, g->res_host, timing);
    if (st != TC_OK) return st;
    st = sync_graph(g);
    if (st != TC_OK) return st;
    *out = *g->res_host;
    if (timing) ring_times(g, g->ring_head - 1, out->ms);
    return TC_OK;
}

tc_status tc_count_async(tc_graph *g, double p, uint64_t seed, tc_result *out)
{
    if (!g || !out || bad_p(p)) return TC_EINVAL;
    return enqueue_count(g, p, seed, out, g->timing != 0 && !g->ring.empty());
}

tc_status tc_graph_sync(tc_graph *g)
{
    if (!g) return TC_EINVAL;
    return sync_graph(g);
}

tc_status tc_graph_export_sample(tc_graph *g, double p, uint64_t seed, uint32_t *kept_pairs_host,
                                 uint8_t *heavy_host, uint32_t *deg_host, uint64_t *m_sampled)
{
    if (!g || bad_p(p)) return TC_EINVAL;
    const uint64_t seed_mix = splitmix64(seed), thr = threshold_of(p);
    CountBuffers b = buffers_of(g);
    enqueue_sample(g, seed_mix, thr, b);
    if (kept_pairs_host && g->m > 0)
        compact_kept(b, seed_mix, thr, g->bufA, g->hist, g->scan, g->stream);
    cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream);
    tc_status st = sync_graph(g);
    if (st != TC_OK) return st;
    const uint64_t mp = g->st_host->m_sampled;
    if (m_sampled) *m_sampled = mp;
    if (heavy_host) cudaMemcpyAsync(heavy_host, g->heavy, g->n, cudaMemcpyDeviceToHost, g->stream);
    if (deg_host) cudaMemcpyAsync(deg_host, g->deg, (size_t)g->n * 4, cudaMemcpyDeviceToHost, g->stream);
    std::vector<uint64_t> keys;
    if (kept_pairs_host && mp > 0) {
        keys.resize(mp);
        cudaMemcpyAsync(keys.data(), g->bufA, mp * 8, cudaMemcpyDeviceToHost, g->stream);
    }
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { cudaGetLastError(); return TC_ECUDA; }
    for (uint64_t i = 0; i < keys.size(); ++i) {
        kept_pairs_host[2 * i] = (uint32_t)(keys[i] >> 32);
        kept_pairs_host[2 * i + 1] = (uint32_t)keys[i];
    }
    return TC_OK;
}

tc_status tc_graph_export_csr(tc_graph *g, double p, uint64_t seed, uint32_t *rowptr_host, uint32_t *col_host,
                              uint64_t *m_sampled)
{
    if (!g || bad_p(p)) return TC_EINVAL;
    const uint64_t seed_mix = splitmix64(seed), thr = threshold_of(p);
    CountBuffers b = buffers_of(g);
    enqueue_sample(g, seed_mix, thr, b);
    if (g->m > 0) {
        enqueue_csr(g, seed_mix, thr);
    } else {
        cudaMemsetAsync(g->rowptr, 0, ((size_t)g->n + 1) * 4, g->stream);
    }
    cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream);
    tc_status st = sync_graph(g);
    if (st != TC_OK) return st;
    const uint64_t mp = g->st_host->m_sampled;
    if (m_sampled) *m_sampled = mp;
    std::vector<uint32_t> rp(g->n + 1), pp(g->n + 1), cp;
    cudaMemcpyAsync(rp.data(), g->rowptr, ((size_t)g->n + 1) * 4, cudaMemcpyDeviceToHost, g->stream);
    if (g->m > 0) cudaMemcpyAsync(pp.data(), g->ptrp, ((size_t)g->n + 1) * 4, cudaMemcpyDeviceToHost, g->stream);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { cudaGetLastError(); return TC_ECUDA; }
    if (rowptr_host) std::copy(rp.begin(), rp.end(), rowptr_host);
    if (g->m == 0 || mp == 0) return TC_OK;
    // the columns are stored padded: check the layout and strip the padding
    const uint64_t total = pp[g->n];
    if (total > colp_capacity(g->n, g->m)) return TC_ECUDA;
    cp.resize(total);
    cudaMemcpyAsync(cp.data(), g->colp, total * 4, cudaMemcpyDeviceToHost, g->stream);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { cudaGetLastError(); return TC_ECUDA; }
    for (uint32_t x = 0; x < g->n; ++x) {
        const uint32_t d = rp[x + 1] - rp[x], beg = pp[x] & ~3u, pad = pp[x] & 3u;
        if (pad != ((4u - (d & 3u)) & 3u) || (pp[x + 1] & ~3u) != beg + d + pad) return TC_ECUDA;
        for (uint32_t i = 0; i < pad; ++i)
            if (cp[beg + d + i] != SENT) return TC_ECUDA;
        if (col_host) std::copy(cp.begin() + beg, cp.begin() + beg + d, col_host + rp[x]);
    }
    return TC_OK;
}

tc_status tc_graph_export_edges(tc_graph *g, uint32_t *pairs_host)
{
    if (!g || (!pairs_host && g->m > 0)) return TC_EINVAL;
    if (g->m == 0) return TC_OK;
    std::vector<uint64_t> keys(g->m);
    cudaMemcpyAsync(keys.data(), g->ekey, g->m * 8, cudaMemcpyDeviceToHost, g->stream);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { cudaGetLastError(); return TC_ECUDA; }
    for (uint64_t i = 0; i < g->m; ++i) {
        pairs_host[2 * i] = (uint32_t)(keys[i] >> 32);
        pairs_host[2 * i + 1] = (uint32_t)keys[i];
    }
    return TC_OK;
}

}  // extern "C"
