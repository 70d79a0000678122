// Batched counting: many independent graphs counted by one launch.
//
// The graphs are stored as one disjoint union (graph g owns vertices
// [voff[g], voff[g+1]) and edges [eoff[g], eoff[g+1]) of the union's sorted
// key array, every graph in its own rank order, csr.cu), so every kernel of
// the count runs once over all of them.  Each edge is sampled with its own graph's (p, seed) on its
// graph-local key, each vertex is split against its own graph's m_p, and the
// class counts go to per-graph counters: every graph gets exactly the
// result a separate tc_count would give.  For tc_batch the whole sequence
// (parameter upload, ~33 kernels, result download) is captured once into a
// CUDA graph and replayed by each tc_batch_count.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <map>
#include <mutex>
#include <new>
#include <vector>

#include "kernels.h"

using namespace tcg;

namespace {

int batch_bits(uint32_t n)
{
    int b = 1;
    while (b < 32 && (1ull << b) < n) ++b;
    return b;
}

// Union keys of the input pairs: graph g's local pair (a, b) becomes
// (min + voff[g]) << 32 | (max + voff[g]); self-loops become ~0; endpoints
// outside their graph raise ERR_ENDPOINT.
__global__ void k_batch_keys(const uint32_t *__restrict__ pairs, uint64_t m_in, const uint64_t *__restrict__ in_off,
                             const uint32_t *__restrict__ voff, uint32_t k, uint64_t *__restrict__ keys, DevState *st)
{
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned bad = 0;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < m_in; base += stride) {
        const uint64_t i = base + lane, ii = i < m_in ? i : m_in - 1;
        const uint32_t g = find_part_warp(in_off, k, ii);
        if (i >= m_in) continue;
        const uint32_t a = pairs[2 * i], b = pairs[2 * i + 1];
        const uint32_t vo = voff[g], ng = voff[g + 1] - vo;
        uint64_t key = ~0ull;
        if (a >= ng || b >= ng) {
            bad = 1;
        } else if (a != b) {
            key = ((uint64_t)(min(a, b) + vo) << 32) | (uint64_t)(max(a, b) + vo);
        }
        keys[i] = key;
    }
    if (bad) atomicOr(&st->err, ERR_ENDPOINT);
}

// eoff[g] = first union key of graph g (keys sorted by source vertex).
__global__ void k_batch_eoff(const uint64_t *__restrict__ keys, uint64_t m, const uint32_t *__restrict__ voff,
                             uint32_t k, uint64_t *__restrict__ eoff)
{
    const uint32_t g = blockIdx.x * blockDim.x + threadIdx.x;
    if (g > k) return;
    if (g == k) {
        eoff[k] = m;
        return;
    }
    const uint64_t target = (uint64_t)voff[g] << 32;
    uint64_t lo = 0, hi = m;
    while (lo < hi) {
        const uint64_t mid = (lo + hi) >> 1;
        if (keys[mid] < target) lo = mid + 1; else hi = mid;
    }
    eoff[g] = lo;
}

void *dev_alloc_track(std::vector<void *> &allocs, uint64_t &total, uint64_t bytes)
{
    void *p = nullptr;
    bytes = std::max<uint64_t>(bytes, 256);
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    allocs.push_back(p);
    total += bytes;
    return p;
}

BatchView view_of(const UnionScratch &u, uint32_t k)
{
    BatchView bv;
    bv.k = k;
    bv.eoff = u.eoff;
    bv.voff = u.voff;
    bv.thr = u.thr;
    bv.seed_mix = u.seed_mix;
    bv.m_p = u.counters;
    bv.t_light = u.counters + u.k_cap;
    bv.t_heavy = u.counters + 2 * (uint64_t)u.k_cap;
    bv.n_heavy = reinterpret_cast<unsigned int *>(u.counters + 3 * (uint64_t)u.k_cap);
    return bv;
}

}  // namespace

namespace tcg {

bool union_scratch_alloc(UnionScratch &u, uint64_t m_cap, uint32_t n_cap, uint32_t k_cap, std::vector<void *> &allocs,
                         uint64_t &bytes)
{
    u.m_cap = m_cap;
    u.n_cap = n_cap;
    u.k_cap = k_cap;
    const uint64_t m1 = std::max<uint64_t>(m_cap, 1);
    const uint64_t hist_len = std::max<uint64_t>(ceil_div(std::max<uint64_t>(m1, n_cap), RX_TILE), 1) << RX_MAX_BITS;
    u.rel = (uint64_t *)dev_alloc_track(allocs, bytes, m1 * 8);
    u.orig = (uint64_t *)dev_alloc_track(allocs, bytes, m1 * 8);
    u.inlist = (uint2 *)dev_alloc_track(allocs, bytes, m1 * 8);
    u.olist = (uint2 *)dev_alloc_track(allocs, bytes, m1 * 8);
    u.ocnt = (uint32_t *)dev_alloc_track(allocs, bytes, (uint64_t)n_cap * 4);
    u.keepw = (uint32_t *)dev_alloc_track(allocs, bytes, (m1 + 31) / 32 * 4);
    u.tile_cnt = (uint32_t *)dev_alloc_track(allocs, bytes, (ceil_div(m1, RX_TILE) + 1) * 4);
    u.spread = (uint32_t *)dev_alloc_track(allocs, bytes, hot_size(n_cap) * 4);
    u.inend = (uint32_t *)dev_alloc_track(allocs, bytes, (uint64_t)n_cap * 4);
    u.deg = (uint32_t *)dev_alloc_track(allocs, bytes, (uint64_t)n_cap * 4);
    u.rowptr = (uint32_t *)dev_alloc_track(allocs, bytes, ((uint64_t)n_cap + 1) * 4);
    u.inptr = (uint32_t *)dev_alloc_track(allocs, bytes, ((uint64_t)n_cap + 2) * 4);
    u.colp = (uint32_t *)dev_alloc_track(allocs, bytes, colp_capacity(n_cap, m1) * 4);
    u.ptrp = (uint32_t *)dev_alloc_track(allocs, bytes, ((uint64_t)n_cap + 2) * 4);
    u.heavy = (uint8_t *)dev_alloc_track(allocs, bytes, n_cap);
    u.items_cap = items_capacity(n_cap, m1);
    u.items = (uint64_t *)dev_alloc_track(allocs, bytes, u.items_cap * 8);
    u.hist = (uint32_t *)dev_alloc_track(allocs, bytes, hist_len * 4);
    u.scan = (uint32_t *)dev_alloc_track(allocs, bytes,
                                         scan_scratch_elems(std::max<uint64_t>(hist_len, (uint64_t)n_cap + 2)) * 4);
    u.st = (DevState *)dev_alloc_track(allocs, bytes, sizeof(DevState));
    u.eoff = (uint64_t *)dev_alloc_track(allocs, bytes, ((uint64_t)k_cap + 1) * 8);
    u.voff = (uint32_t *)dev_alloc_track(allocs, bytes, ((uint64_t)k_cap + 1) * 4);
    u.thr = (uint64_t *)dev_alloc_track(allocs, bytes, (uint64_t)k_cap * 8);
    u.seed_mix = (uint64_t *)dev_alloc_track(allocs, bytes, (uint64_t)k_cap * 8);
    u.p = (double *)dev_alloc_track(allocs, bytes, (uint64_t)k_cap * 8);
    u.counters = (unsigned long long *)dev_alloc_track(allocs, bytes, (uint64_t)k_cap * 28 + 8);
    u.res_dev = (tc_result *)dev_alloc_track(allocs, bytes, (uint64_t)k_cap * sizeof(tc_result));
    // every out-degree of any graph of the union is below sqrt(2 m_cap)
    const uint64_t dmax = (uint64_t)std::sqrt(2.0 * (double)m1) + 2;
    uint64_t slots = 8192;
    while (slots < 4 * dmax && slots < 32768) slots <<= 1;
    u.smem_bytes = (int)(slots * 4);
    intersect_prepare(u.smem_bytes);
    return u.rel && u.orig && u.inlist && u.olist && u.ocnt && u.keepw && u.tile_cnt && u.spread && u.inend && u.deg && u.rowptr && u.inptr && u.colp &&
           u.ptrp && u.heavy && u.items && u.hist && u.scan &&
           u.st && u.eoff && u.voff && u.thr && u.seed_mix && u.p && u.counters && u.res_dev;
}

void union_count(UnionScratch &u, uint64_t m, uint32_t n, uint32_t k, const IsectConfig &cfg, cudaStream_t s)
{
    cudaMemsetAsync(u.st, 0, sizeof(DevState), s);
    cudaMemsetAsync(u.counters, 0, (uint64_t)u.k_cap * 28, s);
    CountBuffers cb;
    cb.ekey = u.rel;
    cb.m = m;
    cb.n = n;
    cb.deg = u.deg;
    cb.heavy = u.heavy;
    cb.rowptr = u.rowptr;
    cb.col = u.colp;
    cb.ptrp = u.ptrp;
    cb.inptr = u.inptr;
    cb.inend = u.inend;
    cb.inlist = u.inlist;
    cb.olist = u.olist;
    cb.ocnt = u.ocnt;
    cb.items = u.items;
    cb.items_cap = items_capacity(n, std::max<uint64_t>(m, 1));
    cb.st = u.st;
    cb.bv = view_of(u, k);
    cb.cfg = cfg;
    RowsArgs ra;
    ra.rel = u.rel;
    ra.orig = u.orig;
    ra.m = m;
    ra.n = n;
    ra.seed_mix = 0;
    ra.thr = 0;
    ra.bv = cb.bv;
    ra.deg = u.deg;
    ra.rowptr = u.rowptr;
    ra.inptr = u.inptr;
    ra.inend = u.inend;
    ra.ptrp = u.ptrp;
    ra.colp = u.colp;
    ra.inlist = u.inlist;
    ra.olist = u.olist;
    ra.ocnt = u.ocnt;
    ra.heavy = u.heavy;
    ra.keepw = u.keepw;
    ra.tile_cnt = u.tile_cnt;
    ra.scan = u.scan;
    ra.spread = u.spread;
    ra.st = u.st;
    sample_rows(ra, s);
    partition(cb, s);
    if (m > 0) {
        build_rows(ra, s);
        build_items(cb, s);
        intersect(cb, u.smem_bytes, s);
    }
    finalize_batch(cb, u.p, u.res_dev, s);
}

// Key i of a union of resident graphs: graph g's rank-order key and its
// original key (rel_src[g], orig_src[g], m_g keys each), both endpoints
// shifted by voff[g]; keys stay sorted because the vertex ranges increase.
__global__ void k_gather_graphs(const uint64_t *const *__restrict__ rel_src, const uint64_t *const *__restrict__ orig_src,
                                const uint64_t *__restrict__ eoff, const uint32_t *__restrict__ voff, uint32_t k,
                                uint64_t m, uint64_t *__restrict__ rel, uint64_t *__restrict__ orig)
{
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < m; base += stride) {
        const uint64_t i = base + lane, ii = i < m ? i : m - 1;
        const uint32_t g = find_part_warp(eoff, k, ii);
        if (i >= m) continue;
        const uint64_t vo = __ldg(voff + g), j = i - __ldg(eoff + g), shift = (vo << 32) | vo;
        rel[i] = __ldg(rel_src[g] + j) + shift;
        orig[i] = __ldg(orig_src[g] + j) + shift;
    }
}

void gather_graphs(const uint64_t *const *rel_src, const uint64_t *const *orig_src, const uint64_t *eoff,
                   const uint32_t *voff, uint32_t k, uint64_t m, uint64_t *rel, uint64_t *orig, cudaStream_t s)
{
    if (m == 0) return;
    k_gather_graphs<<<grid_for(m, 256, 152 * 8), 256, 0, s>>>(rel_src, orig_src, eoff, voff, k, m, rel, orig);
    note_launch();
}

}  // namespace tcg

struct tc_batch {
    uint32_t k = 0, n = 0;
    uint64_t m = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    uint64_t bytes = 0;
    std::vector<void *> allocs;
    UnionScratch u;
    // pinned staging
    uint64_t *h_thr = nullptr, *h_seed_mix = nullptr;
    double *h_p = nullptr;
    tc_result *h_res = nullptr;
    DevState *h_st = nullptr;
    // captured launch and its intersection schedule
    cudaGraphExec_t exec = nullptr;
    unsigned long long launches_per_run = 0;
    IsectConfig cfg;
};

namespace {

void free_batch(tc_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    for (void *p : b->allocs) cudaFree(p);
    cudaFreeHost(b->h_thr);
    cudaFreeHost(b->h_seed_mix);
    cudaFreeHost(b->h_p);
    cudaFreeHost(b->h_res);
    cudaFreeHost(b->h_st);
    if (b->own_stream && b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

// The whole batched count, stream-ordered (captured into a CUDA graph).
void enqueue_batch(tc_batch *b)
{
    cudaStream_t s = b->stream;
    const uint64_t k = b->k;
    cudaMemcpyAsync(b->u.thr, b->h_thr, k * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->u.seed_mix, b->h_seed_mix, k * 8, cudaMemcpyHostToDevice, s);
    cudaMemcpyAsync(b->u.p, b->h_p, k * 8, cudaMemcpyHostToDevice, s);
    union_count(b->u, b->m, b->n, b->k, b->cfg, s);
    cudaMemcpyAsync(b->h_res, b->u.res_dev, k * sizeof(tc_result), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(b->h_st, b->u.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
}

// ---- schedule autotuning
// Shape signature of a batch: floor(log2) of total edges, vertices, graphs
// and average degree.  Tuned schedules are remembered per signature for the
// rest of the process.
uint64_t shape_signature(const tc_batch *b)
{
    auto lg = [](uint64_t x) {
        uint64_t r = 0;
        while (x > 1) {
            x >>= 1;
            ++r;
        }
        return r;
    };
    const uint64_t avg = b->n ? (2 * b->m) / b->n : 0;
    return (lg(b->m) << 24) | (lg(b->n) << 16) | (lg(b->k) << 8) | lg(avg);
}

std::mutex g_tune_mutex;
std::map<uint64_t, IsectConfig> g_tuned;

void drop_exec(tc_batch *b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    b->exec = nullptr;
}

tc_status status_of(unsigned err)
{
    if (err & ERR_ENDPOINT) return TC_EINVAL;
    if (err & ERR_TIMEOUT) return TC_ETIMEOUT;
    if (err) return TC_ECUDA;
    return TC_OK;
}

tc_status stage_params(tc_batch *b, const double *p, const uint64_t *seed)
{
    for (uint32_t g = 0; g < b->k; ++g)
        if (!(p[g] > 0.0 && p[g] <= 1.0)) return TC_EINVAL;
    for (uint32_t g = 0; g < b->k; ++g) {
        b->h_p[g] = p[g];
        b->h_thr[g] = (uint64_t)(p[g] * 9007199254740992.0);
        b->h_seed_mix[g] = splitmix64(seed[g]);
    }
    return TC_OK;
}

// Capture (if needed) and run the batched count once; blocks.
tc_status run_once(tc_batch *b)
{
    if (!b->exec) {
        const uint64_t l0 = tc_launch_count();
        cudaGraph_t graph = nullptr;
        if (cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
            cudaGetLastError();
            return TC_ECUDA;
        }
        enqueue_batch(b);
        if (cudaStreamEndCapture(b->stream, &graph) != cudaSuccess || !graph) {
            cudaGetLastError();
            return TC_ECUDA;
        }
        const cudaError_t ie = cudaGraphInstantiate(&b->exec, graph, 0);
        cudaGraphDestroy(graph);
        if (ie != cudaSuccess) {
            cudaGetLastError();
            b->exec = nullptr;
            return TC_ECUDA;
        }
        b->launches_per_run = tc_launch_count() - l0;
    } else {
        add_launches(b->launches_per_run);
    }
    if (cudaGraphLaunch(b->exec, b->stream) != cudaSuccess || cudaStreamSynchronize(b->stream) != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    return status_of(b->h_st->err);
}

}  // namespace

extern "C" {

tc_status tc_batch_create(const uint32_t *edges, const uint64_t *m_per_graph, const uint32_t *n_per_graph, uint32_t k,
                          int edges_on_device, void *cuda_stream, tc_batch **out)
{
    if (!out) return TC_EINVAL;
    *out = nullptr;
    if (k == 0 || k > 0xffffu || !m_per_graph || !n_per_graph) return TC_EINVAL;
    std::vector<uint64_t> in_off(k + 1, 0);
    std::vector<uint32_t> voff(k + 1, 0);
    uint64_t n_total = 0;
    for (uint32_t g = 0; g < k; ++g) {
        if (n_per_graph[g] == 0) return TC_EINVAL;
        in_off[g + 1] = in_off[g] + m_per_graph[g];
        n_total += n_per_graph[g];
        if (n_total >= 0xffffffffull) return TC_EINVAL;
        voff[g + 1] = (uint32_t)n_total;
    }
    const uint64_t m_in = in_off[k];
    if (m_in > 0xfffffffeull || (m_in > 0 && !edges)) return TC_EINVAL;

    tc_batch *b = new (std::nothrow) tc_batch;
    if (!b) return TC_ENOMEM;
    b->k = k;
    b->n = (uint32_t)n_total;
    if (cuda_stream) {
        b->stream = (cudaStream_t)cuda_stream;
    } else {
        if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess) {
            cudaGetLastError();
            delete b;
            return TC_ECUDA;
        }
        b->own_stream = true;
    }
    cudaStream_t s = b->stream;
    if (cudaMallocHost((void **)&b->h_thr, k * 8) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_seed_mix, k * 8) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_p, k * 8) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_res, k * sizeof(tc_result)) != cudaSuccess ||
        cudaMallocHost((void **)&b->h_st, sizeof(DevState)) != cudaSuccess) {
        cudaGetLastError();
        free_batch(b);
        return TC_ENOMEM;
    }
    // scratch of the count, sized for p = 1 (m_in bounds the canonical m)
    if (!union_scratch_alloc(b->u, m_in, b->n, k, b->allocs, b->bytes)) {
        free_batch(b);
        return TC_ENOMEM;
    }
    cudaMemsetAsync(b->u.st, 0, sizeof(DevState), s);
    cudaMemcpyAsync(b->u.voff, voff.data(), (k + 1) * 4ull, cudaMemcpyHostToDevice, s);

    // ---- union keys: offset, canonicalise, sort, deduplicate, then the rank
    // relabeling of every graph (into u.rel / u.orig, csr.cu)
    uint64_t m = 0;
    {
        std::vector<void *> tmp;
        uint64_t tmp_bytes = 0;
        auto drop_tmp = [&]() {
            cudaStreamSynchronize(s);
            for (void *p : tmp) cudaFree(p);
            tmp.clear();
        };
        const uint64_t m1 = std::max<uint64_t>(m_in, 1);
        uint64_t *ka = (uint64_t *)dev_alloc_track(tmp, tmp_bytes, m1 * 8);
        uint64_t *kb = (uint64_t *)dev_alloc_track(tmp, tmp_bytes, m1 * 8);
        uint64_t *va = (uint64_t *)dev_alloc_track(tmp, tmp_bytes, (uint64_t)b->n * 8);
        uint64_t *vb = (uint64_t *)dev_alloc_track(tmp, tmp_bytes, (uint64_t)b->n * 8);
        uint32_t *perm = (uint32_t *)dev_alloc_track(tmp, tmp_bytes, (uint64_t)b->n * 4);
        uint32_t *rank = (uint32_t *)dev_alloc_track(tmp, tmp_bytes, (uint64_t)b->n * 4);
        if (!ka || !kb || !va || !vb || !perm || !rank) { drop_tmp(); free_batch(b); return TC_ENOMEM; }
        uint64_t *canon = ka;
        if (m_in > 0) {
            const uint32_t *dpairs = edges;
            if (!edges_on_device) {
                void *p = dev_alloc_track(tmp, tmp_bytes, m_in * 8);
                if (!p) { drop_tmp(); free_batch(b); return TC_ENOMEM; }
                cudaMemcpyAsync(p, edges, m_in * 8, cudaMemcpyHostToDevice, s);
                dpairs = (const uint32_t *)p;
            }
            uint64_t *d_in_off = (uint64_t *)dev_alloc_track(tmp, tmp_bytes, (k + 1) * 8ull);
            if (!d_in_off) { drop_tmp(); free_batch(b); return TC_ENOMEM; }
            cudaMemcpyAsync(d_in_off, in_off.data(), (k + 1) * 8ull, cudaMemcpyHostToDevice, s);
            k_batch_keys<<<grid_for(m_in, 256, 152 * 16), 256, 0, s>>>(dpairs, m_in, d_in_off, b->u.voff, k, ka,
                                                                       b->u.st);
            note_launch();
            uint64_t *a = ka, *c = kb;
            const int nbits = batch_bits(b->n);
            for (int half = 0; half < 2; ++half) {
                int shift = half ? 32 : 0;
                const int P = (nbits + RX_MAX_BITS - 1) / RX_MAX_BITS;
                for (int i = 0; i < P; ++i) {
                    const int w = nbits / P + (i < nbits % P ? 1 : 0);
                    radix_pass(a, m_in, shift, w, b->u.hist, b->u.scan, c, s);
                    std::swap(a, c);
                    shift += w;
                }
            }
            unique_keys(a, m_in, c, b->u.hist, b->u.scan, b->u.st, s);
            canon = c;
            cudaMemcpyAsync(b->h_st, b->u.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
            if (cudaStreamSynchronize(s) != cudaSuccess) { cudaGetLastError(); drop_tmp(); free_batch(b); return TC_ECUDA; }
            if (b->h_st->err & ERR_ENDPOINT) { drop_tmp(); free_batch(b); return TC_EINVAL; }
            m = b->h_st->m_canon;
        }
        uint64_t *spare = canon == ka ? kb : ka;
        const RelabelScratch sc{reinterpret_cast<uint64_t *>(b->u.inlist), spare, va, vb, b->u.deg, b->u.hist,
                                b->u.scan};
        relabel(canon, m, b->n, b->u.voff, k, Relabeled{b->u.rel, b->u.orig, perm, rank}, sc, s);
        drop_tmp();
    }
    b->m = m;
    k_batch_eoff<<<(k + 1 + 127) / 128, 128, 0, s>>>(b->u.rel, m, b->u.voff, k, b->u.eoff);
    note_launch();
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        auto it = g_tuned.find(shape_signature(b));
        if (it != g_tuned.end()) b->cfg = it->second;
    }
    if (cudaStreamSynchronize(s) != cudaSuccess || cudaGetLastError() != cudaSuccess) {
        free_batch(b);
        return TC_ECUDA;
    }
    *out = b;
    return TC_OK;
}

void tc_batch_destroy(tc_batch *b) { free_batch(b); }

uint32_t tc_batch_size(const tc_batch *b) { return b ? b->k : 0; }
uint64_t tc_batch_num_edges(const tc_batch *b) { return b ? b->m : 0; }
uint64_t tc_batch_device_bytes(const tc_batch *b) { return b ? b->bytes : 0; }

tc_status tc_batch_count(tc_batch *b, const double *p, const uint64_t *seed, tc_result *out)
{
    if (!b || !p || !seed || !out) return TC_EINVAL;
    tc_status st = stage_params(b, p, seed);
    if (st != TC_OK) return st;
    st = run_once(b);
    if (st != TC_OK) return st;
    std::copy(b->h_res, b->h_res + b->k, out);
    return TC_OK;
}

tc_status tc_batch_autotune(tc_batch *b, const double *p, const uint64_t *seed, char *desc, uint32_t desc_len)
{
    if (!b || !p || !seed) return TC_EINVAL;
    tc_status st = stage_params(b, p, seed);
    if (st != TC_OK) return st;
    cudaEvent_t e0, e1;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    // time of one batched count under schedule c (capture + warm-up, then the
    // best of two replays)
    auto time_of = [&](const IsectConfig &c, float &ms) {
        b->cfg = c;
        drop_exec(b);
        tc_status r = run_once(b);
        ms = 1e30f;
        for (int rep = 0; rep < 2 && r == TC_OK; ++rep) {
            cudaEventRecord(e0, b->stream);
            add_launches(b->launches_per_run);
            cudaGraphLaunch(b->exec, b->stream);
            cudaEventRecord(e1, b->stream);
            if (cudaEventSynchronize(e1) != cudaSuccess) {
                cudaGetLastError();
                r = TC_ECUDA;
                break;
            }
            float t = 0;
            cudaEventElapsedTime(&t, e0, e1);
            ms = std::min(ms, t);
        }
        return r;
    };
    // coordinate search, one axis at a time from the current schedule: the
    // warp / block split of the owners, the mid / large split, the items'
    // sizes and the membership test of each block kernel
    struct Axis {
        uint32_t IsectConfig::*field;
        std::vector<uint32_t> values;
    };
    const Axis axes[] = {{&IsectConfig::warp_max, {64, 128, 256}}, {&IsectConfig::mid_max, {512, 1024}},
                         {&IsectConfig::seg_w, {256, 512}},       {&IsectConfig::seg_b, {256, 512}}};
    IsectConfig best = b->cfg;
    float best_ms = 1e30f;
    st = time_of(best, best_ms);
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
    for (int k = 0; k < 2; ++k) {  // the membership test of each block kernel
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
    b->cfg = best;
    drop_exec(b);
    if (st != TC_OK) return st;
    {
        std::lock_guard<std::mutex> lock(g_tune_mutex);
        g_tuned[shape_signature(b)] = best;
    }
    if (desc && desc_len)
        snprintf(desc, desc_len,
                 "warp_max=%u seg_w=%u seg_b=%u mid_max=%u lookup=%u: warp per owner (d+<=%u, hash sets), "
                 "128-thread block per owner (d+<=%u, %s), 1024-thread block per owner (%s); best_ms=%.3f",
                 best.warp_max, best.seg_w, best.seg_b, best.mid_max, best.lookup, best.warp_max, best.mid_max,
                 lookup_name(best.lookup, 0), lookup_name(best.lookup, 1), best_ms);
    return TC_OK;
}

}  // extern "C"
