// C ABI of libtc (declared in include/tc.h): graph objects, the order of the
// device phases of one count, and the inspection entry points.
#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "kernels.h"

using namespace tcg;

namespace {

tc_alloc_fn g_alloc = nullptr;
tc_free_fn g_free = nullptr;
void *g_alloc_ctx = nullptr;

// Default device memory: a stream-ordered pool of the library's own per
// device.  Blocks are allocated and freed in order on the graph's stream, and
// freed blocks stay in the pool for the next graph (no release threshold)
// until tc_release_cached_memory.  Where a pool cannot be made, cudaMalloc.
std::mutex g_pool_mutex;
cudaMemPool_t g_pool[64] = {};
bool g_pool_failed[64] = {};

cudaMemPool_t pool_of_current_device()
{
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) {
        cudaGetLastError();
        return nullptr;
    }
    std::lock_guard<std::mutex> lock(g_pool_mutex);
    if (!g_pool[dev] && !g_pool_failed[dev]) {
        cudaMemPoolProps props = {};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = dev;
        cudaMemPool_t pool = nullptr;
        uint64_t keep = ~0ull;
        if (cudaMemPoolCreate(&pool, &props) == cudaSuccess &&
            cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &keep) == cudaSuccess) {
            g_pool[dev] = pool;
        } else {
            cudaGetLastError();
            g_pool_failed[dev] = true;
        }
    }
    return g_pool[dev];
}

void *dev_alloc(uint64_t bytes, cudaStream_t s)
{
    bytes = std::max<uint64_t>(bytes, 256);
    if (g_alloc) return g_alloc(bytes, s, g_alloc_ctx);
    void *p = nullptr;
    cudaMemPool_t pool = pool_of_current_device();
    const cudaError_t e = pool ? cudaMallocFromPoolAsync(&p, bytes, pool, s) : cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
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
    else if (pool_of_current_device())
        cudaFreeAsync(p, s);
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

// Host-side NVTX range (shows each phase's enqueue in a profiler timeline;
// a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange &) = delete;
    NvtxRange &operator=(const NvtxRange &) = delete;
};

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
    // device: the graph in rank order (csr.cu)
    uint64_t *rel = nullptr;    // [m] canonical keys in rank ids, sorted
    uint64_t *orig = nullptr;   // [m] original canonical key of each rel key
    uint32_t *perm = nullptr;   // [n] original id of each rank id
    uint32_t *rank = nullptr;   // [n] rank id of each original id
    // device: scratch of a count (rank ids)
    uint32_t *deg = nullptr;    // [n]
    uint32_t *rowptr = nullptr; // [n + 1]
    uint8_t *heavy = nullptr;   // [n]
    uint32_t *inptr = nullptr;  // [n + 2] in-list reservations (static: full in-degrees)
    uint32_t *frow = nullptr;   // [n + 1] row offsets of the full graph in rel (static)
    uint32_t *inend = nullptr;  // [n] in-list ends
    uint2 *inlist = nullptr;    // [m] in-list entries
    uint2 *olist = nullptr;     // [m] out-lists
    uint32_t *ocnt = nullptr;   // [n] out-list lengths
    uint32_t *colp = nullptr;   // [colp_capacity(n, m)] rows padded to 16 bytes
    uint32_t *ptrp = nullptr;   // [n + 2] padded row pointers
    uint32_t *keepw = nullptr;  // [ceil(m / 32)] keep bits
    uint32_t *tile_cnt = nullptr;  // [ceil(m / RX_TILE) + 1]
    uint32_t *spread = nullptr; // [hot_size(n)] per-vertex counters (kernels.h)
    uint64_t *items = nullptr;  // owner work items, all buckets [items_cap]
    uint64_t items_cap = 0;
    uint32_t *hist = nullptr;   // [RX_BINS * ntiles(m)]
    uint32_t *scan = nullptr;   // scan scratch
    HeavyBuffers hb;            // dense heavy block (hb.hcap == 0: not used)
    CoreBuffers core;           // dense core of the top ranks (core.hb.hcap == 0: not used)
    double core_w[CORE_LEVELS_MAX] = {};  // p = 1 probe entries inside the top CORE_MIN << k ranks
    // rates of the dense-core cost model: measured GB300 defaults until
    // tc_graph_autotune measures them on this graph
    double probe_rate = 0.0, tc_rate = 0.0;
    int64_t core_force = -1;    // dense core of every count: < 0 chosen per count, 0 none, else that many ranks
    DevState *st = nullptr;
    tc_result *res_dev = nullptr;
    // pinned host
    tc_result *res_host = nullptr;
    DevState *st_host = nullptr;
    // phase-timing ring: TC_TIMING_RING slots of NUM_EVENTS events
    std::vector<cudaEvent_t> ring;
    uint64_t ring_head = 0;  // next slot to record
    uint64_t ring_tail = 0;  // oldest undrained count
    int64_t sample_floor = -1;  // lower bound on m_p for the degree candidates (< 0: the default)
    cudaEvent_t join_in = nullptr, join_out = nullptr;  // order a count on a caller's stream with the graph's
    int partition = TC_PARTITION_SAMPLED;  // which graph the degree partition splits
    IsectConfig cfg;            // schedule of the intersection kernels
    uint32_t lookup_auto = LOOKUP_DEFAULT;  // its default lookup field on this graph
    TripleBuffers tri;          // triple sampling (built by the first tc_count_triples)
    bool tri_ready = false;
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
    if (g->join_in) cudaEventDestroy(g->join_in);
    if (g->join_out) cudaEventDestroy(g->join_out);
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

// Dense core of the top ranks for graphs of at least CORE_MIN_EDGES edges:
// K = CORE_MIN << k ranks, k < CORE_LEVELS.  Its cost is fixed (about
// K^3 / 3 executed tensor flops, the 128 x 256 tiles on and above the
// diagonal with the K chunks between, and the clearing of 2 K^2 bytes); the probe work it
// takes over is measured per graph at creation (core_work) and shrinks as
// p^2 with sampling (both lists of a pair thin out by p).  The graph keeps
// the size that gains most at p = 1; each count uses the size, up to that,
// that gains most at its p, or none.
constexpr uint32_t CORE_MIN = 8192;
constexpr int CORE_LEVELS = CORE_LEVELS_MAX;  // 8192 .. 65536 ranks
constexpr double CORE_MIN_EDGES = 33554432.0;
constexpr double CORE_PROBE_RATE = 5.0e11;    // streamed entries per second of the probe kernels
constexpr double CORE_TC_RATE = 3.5e15;       // executed fp8 flops per second of the contraction
constexpr double CORE_CLEAR_RATE = 5.0e12;    // bytes per second of clearing U and U^T

double core_cost_s(double K, double tc_rate) { return (K * K * K / 3.0) / tc_rate + 2.0 * K * K / CORE_CLEAR_RATE; }

// Seconds the core of CORE_MIN << k ranks saves at sampling rate p (w_cum:
// p = 1 probe entries inside each core size), at the given rates.
double core_gain(const double *w_cum, int k, double p, double probe_rate, double tc_rate)
{
    return p * p * w_cum[k] / probe_rate - core_cost_s((double)(CORE_MIN << k), tc_rate);
}

// The core size (ranks) a count of g at p uses by default: the one up to
// the allocated size that gains most, or 0.
uint32_t core_ranks_for(const tc_graph *g, double p)
{
    double best = 0.0;
    uint32_t ranks = 0;
    for (int k = 0; k < CORE_LEVELS && (CORE_MIN << k) <= g->core.hb.hcap; ++k) {
        const double gain = core_gain(g->core_w, k, p, g->probe_rate, g->tc_rate);
        if (gain > best) {
            best = gain;
            ranks = CORE_MIN << k;
        }
    }
    return ranks;
}

CountBuffers buffers_of(tc_graph *g)
{
    CountBuffers b;
    b.ekey = g->rel;
    b.m = g->m;
    b.n = g->n;
    b.deg = g->deg;
    b.heavy = g->heavy;
    b.rowptr = g->rowptr;
    b.col = g->colp;
    b.ptrp = g->ptrp;
    b.inptr = g->inptr;
    b.inend = g->inend;
    b.inlist = g->inlist;
    b.static_rows = true;
    b.spread = g->spread;
    b.olist = g->olist;
    b.ocnt = g->ocnt;
    b.items = g->items;
    b.items_cap = g->items_cap;
    b.st = g->st;
    b.cfg = g->cfg;
    if (g->partition == TC_PARTITION_ORIGINAL) {
        b.frow = g->frow;
        b.m_orig = g->m;
    }
    return b;
}

// m_lo: a lower bound on m_p below which the sample falls with probability
// under e^-60 (Chernoff, m_p ~ Binomial(m, p)); only vertices whose full
// degree^2 exceeds it can be heavy.  A sample below it is still counted
// exactly (k_in_fallback).
uint64_t sample_floor(uint64_t m, double p, uint64_t thr)
{
    if (thr >= (1ull << 53)) return m;
    const double mean = p * (double)m, lo = mean - std::sqrt(120.0 * mean) - 1.0;
    return lo > 0.0 ? (uint64_t)lo : 0ull;
}

RowsArgs rows_of(tc_graph *g, uint64_t seed_mix, uint64_t thr, uint64_t m_lo)
{
    RowsArgs a;
    a.rel = g->rel;
    a.orig = g->orig;
    a.m = g->m;
    a.n = g->n;
    a.seed_mix = seed_mix;
    a.thr = thr;
    a.scatter4 = thr >= (3ull << 51);  // p >= 0.75: nearly every compaction tile is full
    a.deg = g->deg;
    a.rowptr = g->rowptr;
    a.inptr = g->inptr;
    a.inend = g->inend;
    a.ptrp = g->ptrp;
    a.colp = g->colp;
    a.inlist = g->inlist;
    a.olist = g->olist;
    a.ocnt = g->ocnt;
    a.keepw = g->keepw;
    a.tile_cnt = g->tile_cnt;
    a.scan = g->scan;
    a.spread = g->spread;
    a.st = g->st;
    a.frow = g->frow;
    a.m_lo = m_lo;
    a.heavy = g->heavy;
    return a;
}

// Sampling, degrees and partition (Sections 3.1-3.2) into g->deg/heavy/st.
void enqueue_sample(tc_graph *g, const RowsArgs &ra)
{
    cudaMemsetAsync(g->st, 0, sizeof(DevState), g->stream);
    sample_rows(ra, g->stream);
    CountBuffers b = buffers_of(g);
    b.all_kept = ra.thr >= (1ull << 53);
    b.core_base = ra.core_base;
    partition(b, g->stream);
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
    RowsArgs ra = rows_of(g, seed_mix, thr,
                          g->sample_floor >= 0 ? (uint64_t)g->sample_floor : sample_floor(g->m, p, thr));
    // the core block pays off once the sample is large: its cost is fixed,
    // the intersections it replaces grow with the sample
    CoreBuffers core_p = g->core;
    const CoreBuffers *core = nullptr;
    if (g->core_force > 0 && g->core.hb.hcap >= (uint64_t)g->core_force) {
        core_p.base = g->n - (uint32_t)g->core_force;
        core = &core_p;
    } else if (g->core_force < 0 && g->core.hb.hcap) {
        const uint32_t ranks = core_ranks_for(g, p);
        if (ranks) {
            core_p.base = g->n - ranks;
            core = &core_p;
        }
    }
    if (core) ra.core_base = core->base;
    CountBuffers b = buffers_of(g);
    if (core) b.core_base = core->base;
    NvtxRange whole("tc_count");
    record(g, timing, 0);
    {
        NvtxRange r("tc_count: sample + partition");
        enqueue_sample(g, ra);
    }
    record(g, timing, 1);
    if (g->m > 0) {
        NvtxRange r("tc_count: oriented CSR");
        if (g->hb.hcap) heavy_decide(b, g->hb, core, g->stream);
        build_rows(ra, g->stream);
        if (g->hb.hcap) heavy_prepare(b, g->hb, core, g->stream);
        build_items(b, g->stream);
    }
    record(g, timing, 2);
    if (g->m > 0) {
        NvtxRange r("tc_count: light wedges (intersections)");
        intersect(b, g->smem_bytes, g->stream);
    }
    record(g, timing, 3);
    if (g->m > 0 && g->hb.hcap) {
        NvtxRange r("tc_count: heavy block (tensor cores)");
        heavy_contract(b, g->hb, core, g->stream);
    }
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

// The union count of tc_count_batch: k graphs (their keys at src[j] and
// src[k + j]) into out[0 .. k) (pinned host memory); blocks until done.
tc_status count_union_of(const std::vector<const uint64_t *> &src, const std::vector<uint64_t> &eoff,
                         const std::vector<uint32_t> &voff, const std::vector<uint64_t> &thr,
                         const std::vector<uint64_t> &mix, const std::vector<double> &p, uint32_t k, uint64_t m,
                         uint32_t n_total, tc_result *out)
{
    cudaStream_t s = nullptr;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    UnionScratch u;
    std::vector<void *> allocs;
    uint64_t bytes = 0;
    const uint64_t **d_src = nullptr;
    DevState st_host;
    tc_status st = TC_OK;
    if (!union_scratch_alloc(u, m, n_total, k, allocs, bytes) ||
        cudaMalloc((void **)&d_src, 2 * (size_t)k * sizeof(void *)) != cudaSuccess) {
        cudaGetLastError();
        st = TC_ENOMEM;
    }
    if (d_src) allocs.push_back((void *)d_src);
    if (st == TC_OK) {
        cudaMemcpyAsync(u.eoff, eoff.data(), (k + 1) * 8ull, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(u.voff, voff.data(), (k + 1) * 4ull, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(u.thr, thr.data(), k * 8ull, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(u.seed_mix, mix.data(), k * 8ull, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(u.p, p.data(), k * 8ull, cudaMemcpyHostToDevice, s);
        cudaMemcpyAsync(d_src, src.data(), 2 * (size_t)k * sizeof(void *), cudaMemcpyHostToDevice, s);
        gather_graphs(d_src, d_src + k, u.eoff, u.voff, k, m, u.rel, u.orig, s);
        union_count(u, m, n_total, k, IsectConfig{}, s);
        cudaMemcpyAsync(out, u.res_dev, k * sizeof(tc_result), cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&st_host, u.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) {
            cudaGetLastError();
            st = TC_ECUDA;
        } else {
            st = status_of_err(st_host.err);
        }
    }
    cudaStreamSynchronize(s);
    for (void *q : allocs) cudaFree(q);
    cudaStreamDestroy(s);
    cudaGetLastError();
    return st;
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

tc_status tc_check_bounded_wait(uint32_t limit_us)
{
    if (limit_us == 0 || limit_us > 1000000u) return TC_EINVAL;
    const int r = wait_check(limit_us);
    return r == 1 ? TC_ETIMEOUT : (r == 0 ? TC_OK : TC_ECUDA);
}

tc_status tc_release_cached_memory(void)
{
    cudaMemPool_t pool = pool_of_current_device();
    if (!pool) return TC_OK;
    if (cudaDeviceSynchronize() != cudaSuccess || cudaMemPoolTrimTo(pool, 0) != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    return TC_OK;
}

uint64_t tc_launch_count(void) { return g_launches.load(std::memory_order_relaxed); }

tc_status tc_graph_create(const uint32_t *edges, uint64_t m_in, uint32_t n, int edges_on_device,
                          void *cuda_stream, tc_graph **out)
{
    if (!out) return TC_EINVAL;
    *out = nullptr;
    if (n == 0 || n == 0xffffffffu || (m_in > 0 && !edges) || m_in > 0xfffffffeull) return TC_EINVAL;

    tc_graph *g = new (std::nothrow) tc_graph;
    if (!g) return TC_ENOMEM;
    g->probe_rate = CORE_PROBE_RATE;
    g->tc_rate = CORE_TC_RATE;
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
    g->deg = (uint32_t *)g->alloc((uint64_t)n * 4);
    if (!g->st || !g->res_dev || !g->deg) {
        free_graph(g);
        return TC_ENOMEM;
    }
    cudaMemsetAsync(g->st, 0, sizeof(DevState), s);
    cudaMemsetAsync(g->deg, 0, (size_t)n * 4, s);

    // ---- canonical keys
    uint64_t m = 0;
    bool deg_ready = m_in == 0;  // g->deg holds the full degrees
    uint64_t *canon = nullptr;  // canonical keys (original ids), sorted [m]
    if (m_in > 0) {
        const uint32_t *dpairs = edges;
        void *tmp_pairs = nullptr;
        // pinned host memory mapped into the device's address space is read
        // in place by the first kernel (over the host link); other host
        // memory is copied first
        cudaPointerAttributes pa;
        if (!edges_on_device && cudaPointerGetAttributes(&pa, edges) == cudaSuccess &&
            pa.type == cudaMemoryTypeHost && pa.devicePointer) {
            dpairs = (const uint32_t *)pa.devicePointer;
        } else if (!edges_on_device) {
            cudaGetLastError();
            tmp_pairs = g->alloc(m_in * 8);
            if (!tmp_pairs) { free_graph(g); return TC_ENOMEM; }
            cudaMemcpyAsync(tmp_pairs, edges, m_in * 8, cudaMemcpyHostToDevice, s);
            dpairs = (const uint32_t *)tmp_pairs;
        }
        uint64_t *keys = (uint64_t *)g->alloc(m_in * 8);
        if (!keys) { free_graph(g); return TC_ENOMEM; }
        // the degrees are counted on the way only when the list may be
        // canonical already (then they are the full degrees); a prefix out of
        // order shows it is not, and the degrees are taken after deduplication
        bool maybe_canonical = true;
        {
            const uint64_t cnt = std::min<uint64_t>(m_in, 1u << 16);
            std::vector<uint32_t> head;
            const uint32_t *hp = edges;
            if (edges_on_device) {
                head.resize(2 * cnt);
                if (cudaMemcpyAsync(head.data(), edges, cnt * 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
                    cudaStreamSynchronize(s) != cudaSuccess) {
                    cudaGetLastError();
                    free_graph(g);
                    return TC_ECUDA;
                }
                hp = head.data();
            }
            for (uint64_t i = 0; i < cnt && maybe_canonical; ++i) {
                const uint32_t a = hp[2 * i], b = hp[2 * i + 1];
                maybe_canonical = a < b && (i == 0 || hp[2 * i - 2] < a || (hp[2 * i - 2] == a && hp[2 * i - 1] < b));
            }
        }
        canon_keys(dpairs, m_in, n, keys, g->st, s, maybe_canonical ? g->deg : nullptr);
        cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); free_graph(g); return TC_ECUDA; }
        if (tmp_pairs) g->release(tmp_pairs);
        if (g->st_host->err & ERR_ENDPOINT) { free_graph(g); return TC_EINVAL; }
        if (g->st_host->unsorted == 0) {
            canon = keys;  // already canonical: every pair u < v, strictly increasing
            m = m_in;
            deg_ready = true;
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
                    radix_pass(a, m_in, shift, w, hist, scan, b, s);
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
            canon = b;
        }
    }
    g->m = m;

    // ---- rank relabeling (csr.cu), then the scratch of a count, sized for p = 1
    const uint64_t m1 = std::max<uint64_t>(m, 1);
    const uint64_t hist_len = std::max<uint64_t>(ceil_div(std::max<uint64_t>(m, n), RX_TILE), 1) << RX_MAX_BITS;
    g->rel = (uint64_t *)g->alloc(m1 * 8);
    g->orig = (uint64_t *)g->alloc(m1 * 8);
    g->perm = (uint32_t *)g->alloc((uint64_t)n * 4);
    g->rank = (uint32_t *)g->alloc((uint64_t)n * 4);
    g->inlist = (uint2 *)g->alloc(m1 * 8);
    g->hist = (uint32_t *)g->alloc(hist_len * 4);
    g->scan = (uint32_t *)g->alloc(scan_scratch_elems(std::max<uint64_t>(hist_len, (uint64_t)n + 2)) * 4);
    if (!g->rel || !g->orig || !g->perm || !g->rank || !g->inlist || !g->deg || !g->hist || !g->scan) {
        free_graph(g);
        return TC_ENOMEM;
    }
    {
        uint64_t *kB = (uint64_t *)g->alloc(m1 * 8);
        uint64_t *vA = (uint64_t *)g->alloc((uint64_t)n * 8), *vB = (uint64_t *)g->alloc((uint64_t)n * 8);
        if (!kB || !vA || !vB) {
            free_graph(g);
            return TC_ENOMEM;
        }
        const RelabelScratch sc{reinterpret_cast<uint64_t *>(g->inlist), kB, vA, vB, g->deg, g->hist, g->scan};
        relabel(canon, m, n, nullptr, 0, Relabeled{g->rel, g->orig, g->perm, g->rank}, sc, s, deg_ready);
        if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); free_graph(g); return TC_ECUDA; }
        g->release(kB);
        g->release(vA);
        g->release(vB);
        if (canon) g->release(canon);
    }
    g->rowptr = (uint32_t *)g->alloc(((uint64_t)n + 1) * 4);
    g->heavy = (uint8_t *)g->alloc((uint64_t)n);
    g->inptr = (uint32_t *)g->alloc(((uint64_t)n + 2) * 4);
    g->inend = (uint32_t *)g->alloc((uint64_t)n * 4);
    g->frow = (uint32_t *)g->alloc(((uint64_t)n + 1) * 4);
    g->olist = (uint2 *)g->alloc(m1 * 8);
    g->ocnt = (uint32_t *)g->alloc((uint64_t)n * 4);
    g->colp = (uint32_t *)g->alloc(colp_capacity(n, m) * 4);
    g->ptrp = (uint32_t *)g->alloc(((uint64_t)n + 2) * 4);
    g->keepw = (uint32_t *)g->alloc((m1 + 31) / 32 * 4);
    g->tile_cnt = (uint32_t *)g->alloc((ceil_div(m1, RX_TILE) + 1) * 4);
    g->spread = (uint32_t *)g->alloc(hot_size(n) * 4);
    g->items_cap = items_capacity(n, m);
    g->items = (uint64_t *)g->alloc(g->items_cap * 8);
    if (!g->rowptr || !g->heavy || !g->inptr || !g->inend || !g->frow || !g->olist || !g->ocnt || !g->colp || !g->ptrp ||
        !g->keepw || !g->tile_cnt || !g->spread || !g->items) {
        free_graph(g);
        return TC_ENOMEM;
    }
    // static rows (g->deg still holds the full degrees by original id)
    static_rows(g->rel, m, n, g->perm, g->deg, g->frow, g->inptr, g->scan, s);
    // table of the owners with d+ > 1024 (their hash set or rank-window
    // bitmap): every out-degree of the degree-oriented graph is at most
    // sqrt(2 m_p); a set of >= 4 d+ slots up to 32768 slots (128 KiB) stays
    // on chip, larger rows are searched in place
    const uint64_t dmax = (uint64_t)std::sqrt(2.0 * (double)std::max<uint64_t>(m, 1)) + 2;
    uint64_t slots = 8192;
    while (slots < 4 * dmax && slots < 32768) slots <<= 1;
    g->smem_bytes = (int)(slots * 4);
    // the rank-window bitmaps of the large owners by default when none can
    // exceed the table: an owner x of that kernel has d+(x) > 512 in any
    // sample, and every vertex ranked above it has a full degree >= that of
    // x, so its window holds at most #{v : deg(v) > 512} ranks
    {
        unsigned long long *cnt = (unsigned long long *)g->alloc(8), wide = ~0ull;
        if (cnt) {
            count_above(g->deg, n, 512, cnt, s);
            cudaMemcpyAsync(&wide, cnt, 8, cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); free_graph(g); return TC_ECUDA; }
            g->release(cnt);
        }
        if (wide <= slots * 32) g->lookup_auto |= LOOKUP_BITMAP_LARGE;
        g->cfg.lookup = g->lookup_auto;
    }
    // dense heavy block: at most 2 m^(1/2) heavy vertices, padded to the
    // 128-row tile and capped at 32768 (2 x 1 GiB of fp8).  Graphs below
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
        g->hb.U = (uint8_t *)g->alloc(hcap * hcap);
        g->hb.UT = g->hb.U ? (uint8_t *)g->alloc(hcap * hcap) : nullptr;
        g->hb.hcap = (uint32_t)hcap;
        if (!g->hb.U || !g->hb.UT || !heavy_make_maps(g->hb)) {
            if (g->hb.U) g->release(g->hb.U);
            if (g->hb.UT) g->release(g->hb.UT);
            g->hb.U = g->hb.UT = nullptr;
            g->hb.hcap = 0;
        }
    }
    // dense core, with the heavy block: the size that gains most at p = 1
    // (2 x K^2 bytes of fp8, 128 MiB for K = 8192, 8 GiB for 65536)
    int core_k = -1;
    if (g->hb.hcap && (double)m >= CORE_MIN_EDGES && n >= 2 * CORE_MIN) {
        int levels = 0;
        while (levels < CORE_LEVELS && (uint64_t)2 * (CORE_MIN << levels) <= n) ++levels;
        unsigned long long *w_dev = (unsigned long long *)g->alloc(CORE_LEVELS_MAX * 8);
        unsigned long long w[CORE_LEVELS_MAX] = {};
        if (w_dev) {
            core_work(g->rel, g->frow, g->inptr, n, m, CORE_MIN, levels, w_dev, s);
            cudaMemcpyAsync(w, w_dev, sizeof(w), cudaMemcpyDeviceToHost, s);
            cudaStreamSynchronize(s);
            g->release(w_dev);
        }
        double acc = 0.0, best = 0.0;
        for (int k = 0; k < levels; ++k) {
            acc += (double)w[k];
            g->core_w[k] = acc;
            const double gain = core_gain(g->core_w, k, 1.0, g->probe_rate, g->tc_rate);
            if (gain > best) {
                best = gain;
                core_k = k;
            }
        }
    }
    if (core_k >= 0) {
        CoreBuffers &c = g->core;
        const uint32_t K = CORE_MIN << core_k;
        const uint64_t bytes = (uint64_t)K * K;
        c.hb.U = (uint8_t *)g->alloc(bytes);
        c.hb.UT = c.hb.U ? (uint8_t *)g->alloc(bytes) : nullptr;
        c.hb.hcap = K;
        c.base = n - K;
        if (!c.hb.U || !c.hb.UT || !heavy_make_maps(c.hb)) {
            if (c.hb.U) g->release(c.hb.U);
            if (c.hb.UT) g->release(c.hb.UT);
            c.hb.U = c.hb.UT = nullptr;
            c.hb.hcap = 0;
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

tc_status tc_graph_set_sample_floor(tc_graph *g, int64_t m_lo)
{
    if (!g) return TC_EINVAL;
    g->sample_floor = m_lo < 0 ? -1 : m_lo;
    return TC_OK;
}

tc_status tc_graph_set_schedule(tc_graph *g, const tc_schedule *s)
{
    if (!g) return TC_EINVAL;
    if (!s) {
        g->cfg = IsectConfig{};
        g->cfg.lookup = g->lookup_auto;
        return TC_OK;
    }
    auto pow2_in = [](uint32_t v, uint32_t lo, uint32_t hi) { return v >= lo && v <= hi && (v & (v - 1)) == 0; };
    if (s->warp_max < 32 || s->warp_max > 256 || !pow2_in(s->seg_w, 64, 1024) || !pow2_in(s->seg_b, 256, 512) ||
        !pow2_in(s->seg_l, 256, 4096) || s->work_w < 4096 || s->work_b < 4096 || s->work_l < 4096 || s->run_b < 1 ||
        s->run_b > 8 || s->mid_max < 512 || s->mid_max > 1024 || s->lookup > 15)
        return TC_EINVAL;
    IsectConfig c;
    c.warp_max = s->warp_max;
    c.seg_w = s->seg_w;
    c.seg_b = s->seg_b;
    c.seg_l = s->seg_l;
    c.work_w = s->work_w;
    c.work_b = s->work_b;
    c.work_l = s->work_l;
    c.run_b = s->run_b;
    c.mid_max = s->mid_max;
    c.lookup = s->lookup;
    g->cfg = c;
    return TC_OK;
}

tc_status tc_graph_autotune(tc_graph *g, double p, uint64_t seed, char *desc, uint32_t desc_len)
{
    if (!g || bad_p(p)) return TC_EINVAL;
    if (sync_graph(g) == TC_ECUDA) return TC_ECUDA;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    // device time of a count under schedule c: one warm-up, then the best of two
    auto time_of = [&](const IsectConfig &c, float &ms) {
        g->cfg = c;
        ms = 1e30f;
        for (int rep = 0; rep < 3; ++rep) {
            cudaEventRecord(e0, g->stream);
            tc_status r = enqueue_count(g, p, seed, g->res_host, false);
            cudaEventRecord(e1, g->stream);
            if (r == TC_OK) r = sync_graph(g);
            if (r != TC_OK) return r;
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep) ms = std::min(ms, t);
        }
        return TC_OK;
    };
    struct Axis {
        uint32_t IsectConfig::*field;
        std::vector<uint32_t> values;
    };
    const Axis axes[] = {{&IsectConfig::warp_max, {64, 128, 256}},
                         {&IsectConfig::mid_max, {512, 1024}},
                         {&IsectConfig::seg_w, {256, 512}},
                         {&IsectConfig::seg_b, {256, 512}},
                         {&IsectConfig::seg_l, {1024, 2048, 4096}}};
    IsectConfig best = g->cfg;
    float best_ms = 1e30f;
    tc_status st = time_of(best, best_ms);
    auto consider = [&](const IsectConfig &c) {
        float ms = 0;
        st = time_of(c, ms);
        if (st == TC_OK && ms < best_ms) {
            best_ms = ms;
            best = c;
        }
    };
    for (const Axis &a : axes) {
        for (uint32_t v : a.values) {
            if (st != TC_OK || best.*(a.field) == v) continue;
            IsectConfig c = best;
            c.*(a.field) = v;
            consider(c);
        }
    }
    // the membership test of each block kernel: hash set, bitmap, binary search
    for (int k = 0; k < 2; ++k) {
        for (uint32_t v : {0u, 4u, 1u}) {
            IsectConfig c = best;
            c.lookup = lookup_with(best.lookup, k, v);
            if (st != TC_OK || c.lookup == best.lookup) continue;
            consider(c);
        }
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    cudaGetLastError();
    g->cfg = best;
    if (st != TC_OK) return st;
    // the dense-core cost model measured on this graph under that schedule:
    // the probe kernels' rate (streamed entries per second) from a count
    // without the core, the contraction's (flops per second) from the time
    // a count with the allocated core adds to the CSR and heavy phases
    if (g->core.hb.hcap) {
        const int timing0 = g->timing;
        const int64_t force0 = g->core_force;
        st = tc_graph_set_timing(g, 1);
        float ms_none[8] = {}, ms_core[8] = {};
        tc_result r_none{};
        auto timed = [&](int64_t force, float *ms, tc_result *r) {
            g->core_force = force;
            for (int rep = 0; rep < 2 && st == TC_OK; ++rep) {  // a warm-up, then the measured count
                st = enqueue_count(g, p, seed, g->res_host, true);
                if (st == TC_OK) st = sync_graph(g);
            }
            if (st == TC_OK) {
                ring_times(g, g->ring_head - 1, ms);
                if (r) *r = *g->res_host;
            }
        };
        const uint32_t K = (uint32_t)g->core.hb.hcap;
        if (st == TC_OK) timed(0, ms_none, &r_none);
        if (st == TC_OK) timed((int64_t)K, ms_core, nullptr);
        g->core_force = force0;
        g->timing = timing0;
        if (st != TC_OK) return st;
        if (ms_none[2] > 0.0f && r_none.nbr_elems > 0) {
            g->probe_rate = (double)r_none.nbr_elems / (ms_none[2] * 1e-3);
            const double Kd = (double)K;
            const double extra = (ms_core[1] - ms_none[1] + ms_core[3] - ms_none[3]) * 1e-3 - 2.0 * Kd * Kd / CORE_CLEAR_RATE;
            if (extra > 0.0) g->tc_rate = (Kd * Kd * Kd / 3.0) / extra;
        }
    }
    if (desc && desc_len)
        snprintf(desc, desc_len,
                 "warp_max=%u mid_max=%u seg_w=%u seg_b=%u seg_l=%u lookup=%u: warp per owner (d+<=%u, hash sets), "
                 "128-thread block per owner (d+<=%u, %s), 1024-thread block per owner (%s); count_ms=%.3f; "
                 "core model: probe %.3g entries/s, contraction %.3g flop/s, core at p=%g: %u ranks",
                 best.warp_max, best.mid_max, best.seg_w, best.seg_b, best.seg_l, best.lookup, best.warp_max,
                 best.mid_max, lookup_name(best.lookup, 0), lookup_name(best.lookup, 1), best_ms, g->probe_rate,
                 g->tc_rate, p, core_ranks_for(g, p));
    return TC_OK;
}

tc_status tc_graph_get_core_model(const tc_graph *g, double p, double *probe_entries_per_s,
                                  double *contraction_flops_per_s, uint32_t *core_ranks)
{
    if (!g || bad_p(p)) return TC_EINVAL;
    if (probe_entries_per_s) *probe_entries_per_s = g->probe_rate;
    if (contraction_flops_per_s) *contraction_flops_per_s = g->tc_rate;
    if (core_ranks) *core_ranks = core_ranks_for(g, p);
    return TC_OK;
}

tc_status tc_graph_get_schedule(const tc_graph *g, tc_schedule *out)
{
    if (!g || !out) return TC_EINVAL;
    const IsectConfig &c = g->cfg;
    *out = tc_schedule{c.warp_max, c.seg_w, c.seg_b, c.seg_l, c.work_w, c.work_b, c.work_l, c.run_b, c.mid_max,
                       c.lookup};
    return TC_OK;
}

tc_status tc_graph_set_partition(tc_graph *g, int mode)
{
    if (!g || (mode != TC_PARTITION_SAMPLED && mode != TC_PARTITION_ORIGINAL)) return TC_EINVAL;
    g->partition = mode;
    return TC_OK;
}

tc_status tc_graph_set_core_ranks(tc_graph *g, int64_t ranks)
{
    if (!g) return TC_EINVAL;
    if (ranks <= 0) {
        g->core_force = ranks < 0 ? -1 : 0;
        return TC_OK;
    }
    bool level = false;
    for (int k = 0; k < CORE_LEVELS; ++k) level |= ranks == (int64_t)(CORE_MIN << k);
    if (!level || 2 * (uint64_t)ranks > g->n || g->hb.hcap == 0 || (double)g->m < CORE_MIN_EDGES) return TC_EINVAL;
    if (g->core.hb.hcap < (uint64_t)ranks) {  // a larger core than creation kept
        if (sync_graph(g) != TC_OK) return TC_ECUDA;
        CoreBuffers &c = g->core;
        if (c.hb.U) g->release(c.hb.U);
        if (c.hb.UT) g->release(c.hb.UT);
        c.hb.U = c.hb.UT = nullptr;
        c.hb.hcap = 0;
        const uint64_t bytes = (uint64_t)ranks * (uint64_t)ranks;
        c.hb.U = (uint8_t *)g->alloc(bytes);
        c.hb.UT = c.hb.U ? (uint8_t *)g->alloc(bytes) : nullptr;
        c.hb.hcap = (uint32_t)ranks;
        c.base = g->n - (uint32_t)ranks;
        if (!c.hb.U || !c.hb.UT || !heavy_make_maps(c.hb)) {
            if (c.hb.U) g->release(c.hb.U);
            if (c.hb.UT) g->release(c.hb.UT);
            c.hb.U = c.hb.UT = nullptr;
            c.hb.hcap = 0;
            g->core_force = -1;
            return TC_ENOMEM;
        }
    }
    g->core_force = ranks;
    return TC_OK;
}

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

tc_status tc_count_async(tc_graph *g, double p, uint64_t seed, tc_result *out, void *cuda_stream)
{
    if (!g || !out || bad_p(p)) return TC_EINVAL;
    const bool timing = g->timing != 0 && !g->ring.empty();
    cudaStream_t s = (cudaStream_t)cuda_stream;
    if (!s || s == g->stream) return enqueue_count(g, p, seed, out, timing);
    // the count runs on the caller's stream, after the graph's pending work,
    // and the graph's stream waits for it (so tc_graph_sync covers it)
    if (!g->join_in) {
        if (cudaEventCreateWithFlags(&g->join_in, cudaEventDisableTiming) != cudaSuccess ||
            cudaEventCreateWithFlags(&g->join_out, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            if (g->join_in) cudaEventDestroy(g->join_in);
            g->join_in = g->join_out = nullptr;
            return TC_ECUDA;
        }
    }
    cudaStream_t own = g->stream;
    cudaEventRecord(g->join_in, own);
    cudaStreamWaitEvent(s, g->join_in, 0);
    g->stream = s;
    const tc_status st = enqueue_count(g, p, seed, out, timing);
    g->stream = own;
    cudaEventRecord(g->join_out, s);
    cudaStreamWaitEvent(own, g->join_out, 0);
    if (st != TC_OK) return st;
    return cudaGetLastError() == cudaSuccess ? TC_OK : TC_ECUDA;
}

tc_status tc_count_batch(tc_graph *const *graphs, const double *p, const uint64_t *seed, uint32_t k, tc_result *out)
{
    if (!graphs || !p || !seed || !out || k == 0 || k > 0xffffu) return TC_EINVAL;
    // graphs with a dense heavy block of their own count on their own path
    // (the block on the tensor cores); the others go into one union
    std::vector<uint32_t> own, uni;
    for (uint32_t i = 0; i < k; ++i) {
        if (!graphs[i] || bad_p(p[i])) return TC_EINVAL;
        (graphs[i]->hb.hcap ? own : uni).push_back(i);
    }
    const uint32_t ku = (uint32_t)uni.size();
    std::vector<uint64_t> eoff(ku + 1, 0), thr(ku), mix(ku);
    std::vector<uint32_t> voff(ku + 1, 0);
    std::vector<const uint64_t *> src(2 * (size_t)ku);
    std::vector<double> pu(ku);
    uint64_t n_total = 0;
    for (uint32_t j = 0; j < ku; ++j) {
        const uint32_t i = uni[j];
        const tc_graph *g = graphs[i];
        eoff[j + 1] = eoff[j] + g->m;
        n_total += g->n;
        if (n_total >= 0xffffffffull) return TC_EINVAL;
        voff[j + 1] = (uint32_t)n_total;
        thr[j] = threshold_of(p[i]);
        mix[j] = splitmix64(seed[i]);
        pu[j] = p[i];
        src[j] = g->rel;
        src[ku + j] = g->orig;
    }
    const uint64_t m = eoff[ku];
    if (m > 0xfffffffeull) return TC_EINVAL;
    NvtxRange whole("tc_count_batch");
    tc_result *stage = nullptr;  // pinned: the own-path results, then the union's
    if (cudaMallocHost((void **)&stage, (size_t)k * sizeof(tc_result)) != cudaSuccess) {
        cudaGetLastError();
        return TC_ENOMEM;
    }
    tc_status st = TC_OK;
    for (uint32_t j = 0; j < own.size() && st == TC_OK; ++j)
        st = enqueue_count(graphs[own[j]], p[own[j]], seed[own[j]], stage + j, false);
    if (st == TC_OK && ku) st = count_union_of(src, eoff, voff, thr, mix, pu, ku, m, (uint32_t)n_total, stage + own.size());
    for (uint32_t j = 0; j < own.size(); ++j) {
        const tc_status s2 = sync_graph(graphs[own[j]]);
        if (st == TC_OK) st = s2;
    }
    if (st == TC_OK) {
        for (uint32_t j = 0; j < own.size(); ++j) {
            out[own[j]] = stage[j];
            for (float &t : out[own[j]].ms) t = 0.0f;
        }
        for (uint32_t j = 0; j < ku; ++j) out[uni[j]] = stage[own.size() + j];
    }
    cudaFreeHost(stage);
    return st;
}

double tc_suggest_p(uint64_t m, uint32_t n, double t, double eps)
{
    if (!(eps > 0.0) || m == 0 || n < 2) return -1.0;
    if (!(t > 0.0)) return 1.0;
    // balance p m against m^(3/2) ln n / (p^(3/2) t eps^2)
    const double x = std::sqrt((double)m) * std::log((double)n) / (t * eps * eps);
    const double p = std::pow(x, 0.4);
    return p < 1.0 ? p : 1.0;
}

tc_status tc_count_sweep(tc_graph *g, const double *p, const uint64_t *seed, uint32_t k, tc_result *out)
{
    if (!g || !p || !seed || !out || k == 0) return TC_EINVAL;
    for (uint32_t i = 0; i < k; ++i)
        if (bad_p(p[i])) return TC_EINVAL;
    NvtxRange whole("tc_count_sweep");
    tc_result *stage = nullptr;
    if (cudaMallocHost((void **)&stage, (size_t)k * sizeof(tc_result)) != cudaSuccess) {
        cudaGetLastError();
        return TC_ENOMEM;
    }
    tc_status st = TC_OK;
    for (uint32_t i = 0; i < k && st == TC_OK; ++i) st = enqueue_count(g, p[i], seed[i], stage + i, false);
    const tc_status sy = sync_graph(g);
    if (st == TC_OK) st = sy;
    if (st == TC_OK) std::copy(stage, stage + k, out);
    cudaFreeHost(stage);
    return st;
}

tc_status tc_count_adaptive(tc_graph *g, double p0, double growth, double tol, uint64_t seed, uint32_t max_counts,
                            tc_result *out, double *p_used, uint32_t *counts_used)
{
    if (!g || !out || bad_p(p0) || !(growth > 1.0) || !(tol >= 0.0) || max_counts == 0 || max_counts > 64)
        return TC_EINVAL;
    std::vector<double> ps;
    for (double q = p0; ps.size() < max_counts; q *= growth) {
        ps.push_back(q < 1.0 ? q : 1.0);
        if (q >= 1.0) break;
    }
    std::vector<uint64_t> seeds(ps.size(), seed);
    std::vector<tc_result> res(ps.size());
    const tc_status st = tc_count_sweep(g, ps.data(), seeds.data(), (uint32_t)ps.size(), res.data());
    if (st != TC_OK) return st;
    size_t pick = ps.size() - 1;
    for (size_t i = 1; i < ps.size(); ++i) {
        if (std::fabs(res[i].estimate - res[i - 1].estimate) <= tol * std::fabs(res[i].estimate)) {
            pick = i;
            break;
        }
    }
    *out = res[pick];
    if (p_used) *p_used = ps[pick];
    if (counts_used) *counts_used = (uint32_t)ps.size();
    return TC_OK;
}

tc_status tc_count_auto(tc_graph *g, double eps, double pilot_p, uint64_t seed, tc_result *out, double *p_used)
{
    if (!g || !out || bad_p(pilot_p) || !(eps > 0.0)) return TC_EINVAL;
    tc_result pilot;
    tc_status st = tc_count(g, pilot_p, seed, &pilot);
    if (st != TC_OK) return st;
    const double p = tc_suggest_p(g->m, g->n, pilot.estimate, eps);
    if (p <= 0.0) {  // no edges or a single vertex: the pilot is the count
        *out = pilot;
        if (p_used) *p_used = pilot_p;
        return TC_OK;
    }
    st = tc_count(g, p, seed, out);
    if (st == TC_OK && p_used) *p_used = p;
    return st;
}

tc_status tc_count_triples(tc_graph *g, double p, uint64_t seed, uint64_t samples, int mode, tc_triple_result *out)
{
    if (!g || !out || bad_p(p) || (mode != TC_TRIPLES_SIMPLE && mode != TC_TRIPLES_HYBRID)) return TC_EINVAL;
    if (2 * g->m > 0xffffffffull) return TC_EINVAL;
    NvtxRange whole("tc_count_triples");
    if (sync_graph(g) == TC_ECUDA) return TC_ECUDA;
    const uint32_t n = g->n;
    const uint64_t m = g->m, len = std::max<uint64_t>(2 * m, 1);
    TripleBuffers &tb = g->tri;
    if (!g->tri_ready) {
        NvtxRange r("tc_count_triples: symmetric adjacency");
        tb.n = n;
        tb.m = m;
        tb.hcap = (uint32_t)(2.0 * std::sqrt((double)m)) + 2;
        tb.soff = (uint32_t *)g->alloc(((uint64_t)n + 1) * 4);
        tb.snbr = (uint32_t *)g->alloc(len * 4);
        tb.off_p = (uint32_t *)g->alloc(((uint64_t)n + 1) * 4);
        tb.nbr_p = (uint32_t *)g->alloc(len * 4);
        tb.qpre = (uint32_t *)g->alloc(len * 4);
        tb.cnt = (unsigned long long *)g->alloc(((uint64_t)n + 1) * 8);
        tb.scan64 = (unsigned long long *)g->alloc((ceil_div((uint64_t)n + 1, SC_CHUNK) + 1) * 8);
        tb.scan32 = (uint32_t *)g->alloc(scan_scratch_elems((uint64_t)n + 1) * 4);
        tb.hlist = (uint32_t *)g->alloc((uint64_t)tb.hcap * 4);
        tb.dev = (TripleDev *)g->alloc(sizeof(TripleDev));
        tb.res = (tc_triple_result *)g->alloc(sizeof(tc_triple_result));
        const uint64_t hist_len = std::max<uint64_t>(ceil_div(len, RX_TILE), 1) << RX_MAX_BITS;
        uint64_t *ka = (uint64_t *)g->alloc(len * 8), *kb = (uint64_t *)g->alloc(len * 8);
        uint32_t *hist = (uint32_t *)g->alloc(hist_len * 4);
        uint32_t *hscan = (uint32_t *)g->alloc(scan_scratch_elems(hist_len) * 4);
        auto drop_all = [&]() {
            for (void *q : {(void *)ka, (void *)kb, (void *)hist, (void *)hscan, (void *)tb.soff, (void *)tb.snbr,
                            (void *)tb.off_p, (void *)tb.nbr_p, (void *)tb.qpre, (void *)tb.cnt, (void *)tb.scan64,
                            (void *)tb.scan32, (void *)tb.hlist, (void *)tb.dev, (void *)tb.res})
                if (q) g->release(q);
            tb = TripleBuffers{};
        };
        if (!tb.soff || !tb.snbr || !tb.off_p || !tb.nbr_p || !tb.qpre || !tb.cnt || !tb.scan64 || !tb.scan32 ||
            !tb.hlist || !tb.dev || !tb.res || !ka || !kb || !hist || !hscan) {
            drop_all();
            return TC_ENOMEM;
        }
        triples_build(g->orig, m, n, g->nbits, tb, ka, kb, hist, hscan, g->stream);
        if (cudaStreamSynchronize(g->stream) != cudaSuccess) {
            cudaGetLastError();
            drop_all();
            return TC_ECUDA;
        }
        g->release(ka);
        g->release(kb);
        g->release(hist);
        g->release(hscan);
        g->tri_ready = true;
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (timed) cudaEventRecord(e0, g->stream);
    triples_count(tb, splitmix64(seed), threshold_of(p), seed, samples, mode == TC_TRIPLES_HYBRID, p, tb.res,
                  g->stream);
    if (timed) cudaEventRecord(e1, g->stream);
    tc_triple_result host;
    cudaMemcpyAsync(&host, tb.res, sizeof(host), cudaMemcpyDeviceToHost, g->stream);
    const cudaError_t e = cudaStreamSynchronize(g->stream);
    float ms = 0.0f;
    if (timed && e == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (e != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    host.ms = ms;
    *out = host;
    return TC_OK;
}

tc_status tc_stream_count(const uint64_t *offsets, const uint32_t *adj, uint32_t n, uint64_t seed, uint64_t samples,
                          double heavy_factor, uint64_t chunk_entries, void *cuda_stream, tc_stream_result *out)
{
    if (!offsets || !out || n == 0 || n == 0xffffffffu || !(heavy_factor > 0.0)) return TC_EINVAL;
    if (offsets[0] != 0) return TC_EINVAL;
    for (uint32_t u = 0; u < n; ++u)
        if (offsets[u + 1] < offsets[u]) return TC_EINVAL;
    const uint64_t len = offsets[n];
    if ((len & 1) || len >= (1ull << 33) || (len > 0 && !adj)) return TC_EINVAL;
    NvtxRange whole("tc_stream_count");
    cudaStream_t s = (cudaStream_t)cuda_stream;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    const bool timed = cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess;
    if (timed) cudaEventRecord(e0, s);
    tc_stream_result r;
    const tc_status st = stream_count(offsets, adj, n, seed, samples, heavy_factor, chunk_entries, s, &r);
    float ms = 0.0f;
    if (timed) {
        cudaEventRecord(e1, s);
        if (cudaEventSynchronize(e1) == cudaSuccess) cudaEventElapsedTime(&ms, e0, e1);
    }
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaGetLastError();
    if (st != TC_OK) return st;
    r.ms = ms;
    *out = r;
    return TC_OK;
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
    enqueue_sample(g, rows_of(g, seed_mix, thr, 0));  // every vertex with an edge: exact degrees
    cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream);
    tc_status st = sync_graph(g);
    if (st != TC_OK) return st;
    const uint64_t mp = g->st_host->m_sampled;
    if (m_sampled) *m_sampled = mp;
    // the device holds the graph in rank order: map back to original ids
    const uint32_t n = g->n;
    std::vector<uint32_t> rank(n), deg(n), keepw;
    std::vector<uint8_t> heavy(n);
    std::vector<uint64_t> orig;
    cudaMemcpyAsync(rank.data(), g->rank, (size_t)n * 4, cudaMemcpyDeviceToHost, g->stream);
    cudaMemcpyAsync(deg.data(), g->deg, (size_t)n * 4, cudaMemcpyDeviceToHost, g->stream);
    cudaMemcpyAsync(heavy.data(), g->heavy, n, cudaMemcpyDeviceToHost, g->stream);
    if (kept_pairs_host && g->m > 0) {
        keepw.resize((g->m + 31) / 32);
        orig.resize(g->m);
        cudaMemcpyAsync(keepw.data(), g->keepw, keepw.size() * 4, cudaMemcpyDeviceToHost, g->stream);
        cudaMemcpyAsync(orig.data(), g->orig, g->m * 8, cudaMemcpyDeviceToHost, g->stream);
    }
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { cudaGetLastError(); return TC_ECUDA; }
    for (uint32_t v = 0; v < n; ++v) {
        if (deg_host) deg_host[v] = deg[rank[v]];
        if (heavy_host) heavy_host[v] = heavy[rank[v]];
    }
    if (kept_pairs_host && g->m > 0) {
        std::vector<uint64_t> kept;
        kept.reserve(mp);
        for (uint64_t i = 0; i < g->m; ++i)
            if ((keepw[i >> 5] >> (i & 31)) & 1u) kept.push_back(orig[i]);
        if (kept.size() != mp) return TC_ECUDA;
        std::sort(kept.begin(), kept.end());  // canonical order of the original ids
        for (uint64_t i = 0; i < kept.size(); ++i) {
            kept_pairs_host[2 * i] = (uint32_t)(kept[i] >> 32);
            kept_pairs_host[2 * i + 1] = (uint32_t)kept[i];
        }
    }
    return TC_OK;
}

tc_status tc_graph_export_csr(tc_graph *g, double p, uint64_t seed, uint32_t *rowptr_host, uint32_t *col_host,
                              uint64_t *m_sampled)
{
    if (!g || bad_p(p)) return TC_EINVAL;
    const uint64_t seed_mix = splitmix64(seed), thr = threshold_of(p);
    const RowsArgs ra = rows_of(g, seed_mix, thr, sample_floor(g->m, p, thr));
    enqueue_sample(g, ra);
    if (g->m > 0) build_rows(ra, g->stream);
    cudaMemcpyAsync(g->st_host, g->st, sizeof(DevState), cudaMemcpyDeviceToHost, g->stream);
    tc_status st = sync_graph(g);
    if (st != TC_OK) return st;
    const uint64_t mp = g->st_host->m_sampled;
    if (m_sampled) *m_sampled = mp;
    const uint32_t n = g->n;
    std::vector<uint32_t> rp(n + 1, 0), pp(n + 1, 0), perm(n), rank(n), cp;
    cudaMemcpyAsync(perm.data(), g->perm, (size_t)n * 4, cudaMemcpyDeviceToHost, g->stream);
    cudaMemcpyAsync(rank.data(), g->rank, (size_t)n * 4, cudaMemcpyDeviceToHost, g->stream);
    if (g->m > 0) {
        cudaMemcpyAsync(rp.data(), g->rowptr, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost, g->stream);
        cudaMemcpyAsync(pp.data(), g->ptrp, ((size_t)n + 1) * 4, cudaMemcpyDeviceToHost, g->stream);
    }
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { cudaGetLastError(); return TC_ECUDA; }
    // rows of the original ids: vertex v's row is rank row rank[v]
    if (rowptr_host) {
        rowptr_host[0] = 0;
        for (uint32_t v = 0; v < n; ++v) rowptr_host[v + 1] = rowptr_host[v] + (rp[rank[v] + 1] - rp[rank[v]]);
    }
    if (g->m == 0 || mp == 0) return TC_OK;
    // the columns are stored padded: check the layout and strip the padding
    const uint64_t total = pp[n];
    if (total > colp_capacity(n, g->m)) return TC_ECUDA;
    cp.resize(total);
    cudaMemcpyAsync(cp.data(), g->colp, total * 4, cudaMemcpyDeviceToHost, g->stream);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { cudaGetLastError(); return TC_ECUDA; }
    uint64_t out_pos = 0;
    for (uint32_t v = 0; v < n; ++v) {
        const uint32_t x = rank[v];
        const uint32_t d = rp[x + 1] - rp[x], beg = pp[x] & ~3u, pad = pp[x] & 3u;
        if (pad != ((4u - (d & 3u)) & 3u) || (pp[x + 1] & ~3u) != beg + d + pad) return TC_ECUDA;
        for (uint32_t i = 0; i < pad; ++i)
            if (cp[beg + d + i] != SENT) return TC_ECUDA;
        if (col_host)
            for (uint32_t i = 0; i < d; ++i) col_host[out_pos + i] = perm[cp[beg + i]];
        out_pos += d;
    }
    return TC_OK;
}

tc_status tc_graph_export_edges(tc_graph *g, uint32_t *pairs_host)
{
    if (!g || (!pairs_host && g->m > 0)) return TC_EINVAL;
    if (g->m == 0) return TC_OK;
    std::vector<uint64_t> keys(g->m);
    cudaMemcpyAsync(keys.data(), g->orig, g->m * 8, cudaMemcpyDeviceToHost, g->stream);
    if (cudaStreamSynchronize(g->stream) != cudaSuccess) { cudaGetLastError(); return TC_ECUDA; }
    std::sort(keys.begin(), keys.end());
    for (uint64_t i = 0; i < g->m; ++i) {
        pairs_host[2 * i] = (uint32_t)(keys[i] >> 32);
        pairs_host[2 * i + 1] = (uint32_t)keys[i];
    }
    return TC_OK;
}

}  // extern "C"
