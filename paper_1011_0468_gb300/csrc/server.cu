// Continuous-batching request server (tc_server_*).
//
// A request is (graph, p, seed): one instance of the problem of Section 1
// with the sample of Section 3.1.  Registered graphs stay resident in device
// memory in rank order (csr.cu: the sorted canonical keys in rank ids, then
// the original key of each), with a pinned host copy from which an evicted
// graph is uploaded again.  A worker thread owns the count slots; each slot holds the
// scratch of one batched count (union_count, batch.cu) and its own stream.
// When a slot is free the worker admits the longest first-come prefix of the
// queue that fits the slot and the HBM budget, gathers the requests' edge
// lists into the slot's union (one copy kernel), and enqueues the batched
// count followed by a host callback that wakes the worker again.  Because
// the union gives every request its own vertex range, counters and (p,
// seed), each result equals the one tc_count returns for that graph alone.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <list>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <unordered_map>
#include <vector>

#include "kernels.h"

using namespace tcg;

namespace {

constexpr uint32_t MAX_SLOTS = 8;

// Key i of the union: request g's rank-order keys and their original keys
// (src[g] holds m_g of each, one after the other), both endpoints shifted by
// voff[g] (keys stay sorted because the vertex ranges increase).
__global__ void k_gather(const uint64_t *const *__restrict__ src, const uint64_t *__restrict__ eoff,
                         const uint32_t *__restrict__ voff, uint32_t k, uint64_t m, uint64_t *__restrict__ rel,
                         uint64_t *__restrict__ orig)
{
    const unsigned lane = lane_id();
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < m; base += stride) {
        const uint64_t i = base + lane, ii = i < m ? i : m - 1;
        const uint32_t g = find_part_warp(eoff, k, ii);
        if (i >= m) continue;
        const uint64_t vo = __ldg(voff + g), e0 = __ldg(eoff + g), mg = __ldg(eoff + g + 1) - e0;
        const uint64_t *sg = src[g];
        rel[i] = __ldg(sg + (i - e0)) + ((vo << 32) | vo);
        orig[i] = __ldg(sg + mg + (i - e0)) + ((vo << 32) | vo);
    }
}

int key_bits(uint32_t n)
{
    int b = 1;
    while (b < 32 && (1ull << b) < n) ++b;
    return b;
}

double now_us(std::chrono::steady_clock::time_point t0)
{
    return std::chrono::duration<double, std::micro>(std::chrono::steady_clock::now() - t0).count();
}

struct GraphEntry {
    uint64_t m = 0;
    uint32_t n = 0;
    uint64_t *host = nullptr;   // pinned keys [2 m]: rank-order keys, then their original keys
    uint64_t *dev = nullptr;    // resident copy (NULL when evicted or m == 0)
    uint64_t dev_bytes = 0;     // bytes charged to the budget while resident
    bool resident = false;      // charged (upload may still be in flight)
    uint32_t pins = 0;          // admitted requests not yet finished
    std::list<uint32_t>::iterator lru;
    cudaEvent_t ready = nullptr;  // recorded after each re-upload
    int upload_slot = -1;
    uint64_t upload_wave = 0;
    // a wave of one request on this graph, captured once per slot while the
    // resident copy stays in place (kernels baked for its m, n and address)
    cudaGraphExec_t exec[MAX_SLOTS] = {};
    unsigned long long exec_launches[MAX_SLOTS] = {};
};

struct Req {
    uint64_t ticket;
    uint32_t gid;
    double p;
    uint64_t seed;
    double t_submit;
};

struct Record {
    tc_request_info info;
    bool done = false;
};

struct Slot {
    UnionScratch u;
    cudaStream_t s = nullptr;
    // one wave's parameters, packed for a single copy (wave_params), pinned
    // staging and its device twin, and the pinned results
    unsigned char *h_params = nullptr, *d_params = nullptr;
    tc_result *h_res = nullptr;
    DevState *h_st = nullptr;
    cudaEvent_t done_ev = nullptr;  // recorded when the wave's results are on the host
    // wave in flight
    std::vector<Req> wave;
    std::vector<GraphEntry *> wave_graphs;
    bool busy = false;  // a wave is in flight (its end: done_ev)
    tc_status launch_status = TC_OK;
    double t_admit = 0;
    uint64_t serial = 0;
};

// Byte offsets of a wave's parameters in one block (k requests): eoff[k + 1],
// src[k], p[k], thr[k], seed mixes[k] (8 bytes each), then voff[k + 1].
struct WaveLayout {
    uint64_t eoff, src, p, thr, mix, voff, bytes;
};
WaveLayout wave_layout(uint32_t k)
{
    WaveLayout L;
    L.eoff = 0;
    L.src = L.eoff + (k + 1ull) * 8;
    L.p = L.src + k * 8ull;
    L.thr = L.p + k * 8ull;
    L.mix = L.thr + k * 8ull;
    L.voff = L.mix + k * 8ull;
    L.bytes = L.voff + (k + 1ull) * 4;
    return L;
}

struct CallbackCtx {
    tc_server *srv;
    uint32_t slot;
};

tc_status status_of(unsigned err)
{
    if (err & ERR_ENDPOINT) return TC_EINVAL;
    if (err & ERR_TIMEOUT) return TC_ETIMEOUT;
    if (err) return TC_ECUDA;
    return TC_OK;
}

}  // namespace

struct tc_server {
    int device = 0;
    uint64_t budget = 0, slot_bytes = 0, resident_bytes = 0;
    uint64_t slot_edges = 0;
    uint32_t slot_vertices = 0, slot_requests = 0, nslots = 0;
    std::vector<void *> allocs;  // slot scratch (cudaMalloc)
    Slot slots[MAX_SLOTS];
    CallbackCtx cb[MAX_SLOTS];

    std::mutex mu;
    std::condition_variable work_cv, done_cv;
    std::vector<std::unique_ptr<GraphEntry>> graphs;
    std::list<uint32_t> lru;  // resident graphs, least recently used first
    std::deque<Req> queue;
    std::unordered_map<uint64_t, Record> records;
    uint64_t next_ticket = 1, wave_serial = 0;
    bool stop = false;
    tc_server_stats stats{};

    std::atomic<uint64_t> arrivals{0};  // submissions so far (read by the polling worker)

    std::mutex ingest_mu;
    cudaStream_t ingest = nullptr;
    std::thread worker;
    std::chrono::steady_clock::time_point t0;
};

namespace {

void CUDART_CB on_slot_done(void *arg)
{
    // runs on a CUDA callback thread: no CUDA calls here
    CallbackCtx *c = static_cast<CallbackCtx *>(arg);
    {
        // a wake-up only: the worker tells a finished wave by its done_ev
        std::lock_guard<std::mutex> lock(c->srv->mu);
    }
    c->srv->work_cv.notify_all();
}

// Under the lock: finish the slot's wave (results to the records, graphs
// unpinned).
void complete_wave(tc_server *srv, uint32_t si)
{
    Slot &sl = srv->slots[si];
    tc_status st = sl.launch_status;
    if (st == TC_OK) st = status_of(sl.h_st->err);
    const double t_done = now_us(srv->t0);
    for (size_t j = 0; j < sl.wave.size(); ++j) {
        auto it = srv->records.find(sl.wave[j].ticket);
        if (it != srv->records.end()) {
            tc_request_info &info = it->second.info;
            if (st == TC_OK) {
                info.res = sl.h_res[j];
                std::memset(info.res.ms, 0, sizeof(info.res.ms));
            }
            info.status = st;
            info.wave_size = (uint32_t)sl.wave.size();
            info.t_admit_us = sl.t_admit;
            info.t_done_us = t_done;
            it->second.done = true;
        }
    }
    for (GraphEntry *g : sl.wave_graphs) --g->pins;
    srv->stats.completed += sl.wave.size();
    sl.wave.clear();
    sl.wave_graphs.clear();
    sl.busy = false;
    srv->done_cv.notify_all();
}

// Under the lock: admit the longest queue prefix that fits slot si and the
// budget.  Graphs to (re)upload go to `uploads`, device copies to free to
// `frees`.  Returns false if nothing could be admitted.
bool form_wave(tc_server *srv, uint32_t si, std::vector<GraphEntry *> &uploads, std::vector<uint64_t *> &frees,
               std::vector<cudaGraphExec_t> &dead)
{
    Slot &sl = srv->slots[si];
    const uint64_t room = srv->budget - srv->slot_bytes;
    uint64_t m_sum = 0, n_sum = 0;
    while (!srv->queue.empty() && sl.wave.size() < srv->slot_requests) {
        const Req &r = srv->queue.front();
        GraphEntry *g = srv->graphs[r.gid].get();
        if (m_sum + g->m > srv->slot_edges || n_sum + g->n > srv->slot_vertices) break;
        if (g->m > 0 && !g->resident) {
            if (srv->resident_bytes + g->dev_bytes > room) {
                uint64_t reclaim = 0;  // evict only if that makes enough room
                for (uint32_t id : srv->lru)
                    if (!srv->graphs[id]->pins) reclaim += srv->graphs[id]->dev_bytes;
                if (srv->resident_bytes - reclaim + g->dev_bytes > room) break;  // wait for running slots
            }
            // evict least recently used graphs no slot is using
            auto it = srv->lru.begin();
            while (srv->resident_bytes + g->dev_bytes > room && it != srv->lru.end()) {
                GraphEntry *v = srv->graphs[*it].get();
                if (v->pins) {
                    ++it;
                    continue;
                }
                if (v->dev) frees.push_back(v->dev);
                v->dev = nullptr;
                for (cudaGraphExec_t &e : v->exec)  // its captured waves name the old copy
                    if (e) {
                        dead.push_back(e);
                        e = nullptr;
                    }
                v->resident = false;
                srv->resident_bytes -= v->dev_bytes;
                --srv->stats.resident_graphs;
                ++srv->stats.evictions;
                it = srv->lru.erase(it);
            }
            if (srv->resident_bytes + g->dev_bytes > room) break;  // wait for running slots
            g->resident = true;
            srv->resident_bytes += g->dev_bytes;
            ++srv->stats.resident_graphs;
            ++srv->stats.uploads;
            g->lru = srv->lru.insert(srv->lru.end(), r.gid);
            uploads.push_back(g);
        } else if (g->m > 0) {
            srv->lru.splice(srv->lru.end(), srv->lru, g->lru);  // most recently used
        }
        ++g->pins;
        sl.wave.push_back(r);
        sl.wave_graphs.push_back(g);
        m_sum += g->m;
        n_sum += g->n;
        srv->queue.pop_front();
    }
    return !sl.wave.empty();
}

// Outside the lock (worker thread only): enqueue the wave of slot si.
tc_status enqueue_wave(tc_server *srv, uint32_t si, const std::vector<GraphEntry *> &uploads,
                       const std::vector<uint64_t *> &frees, const std::vector<cudaGraphExec_t> &dead)
{
    Slot &sl = srv->slots[si];
    cudaStream_t s = sl.s;
    for (cudaGraphExec_t e : dead) cudaGraphExecDestroy(e);  // their graphs ran no wave in flight
    for (uint64_t *ptr : frees) cudaFreeAsync(ptr, s);
    for (GraphEntry *g : uploads) {
        if (cudaMallocAsync((void **)&g->dev, g->m * 16, s) != cudaSuccess) {
            cudaGetLastError();
            g->dev = nullptr;
            return TC_ENOMEM;
        }
        cudaMemcpyAsync(g->dev, g->host, g->m * 16, cudaMemcpyHostToDevice, s);
        cudaEventRecord(g->ready, s);
        g->upload_slot = (int)si;
        g->upload_wave = sl.serial;
    }
    const uint32_t k = (uint32_t)sl.wave.size();
    uint64_t m = 0, n = 0;
    for (uint32_t j = 0; j < k; ++j) {
        GraphEntry *g = sl.wave_graphs[j];
        // a copy uploaded by another slot's wave that may still be running
        if (g->upload_slot >= 0 && g->upload_slot != (int)si) {
            const Slot &o = srv->slots[g->upload_slot];
            if (o.busy && o.serial == g->upload_wave) cudaStreamWaitEvent(s, g->ready, 0);
        }
    }
    // the wave's parameters in one pinned block, copied once
    const WaveLayout L = wave_layout(k);
    UnionScratch u = sl.u;
    uint64_t *h_eoff = reinterpret_cast<uint64_t *>(sl.h_params + L.eoff);
    uint32_t *h_voff = reinterpret_cast<uint32_t *>(sl.h_params + L.voff);
    const uint64_t **h_src = reinterpret_cast<const uint64_t **>(sl.h_params + L.src);
    double *h_p = reinterpret_cast<double *>(sl.h_params + L.p);
    uint64_t *h_thr = reinterpret_cast<uint64_t *>(sl.h_params + L.thr);
    uint64_t *h_mix = reinterpret_cast<uint64_t *>(sl.h_params + L.mix);
    for (uint32_t j = 0; j < k; ++j) {
        GraphEntry *g = sl.wave_graphs[j];
        const Req &r = sl.wave[j];
        h_eoff[j] = m;
        h_voff[j] = (uint32_t)n;
        h_src[j] = g->dev;
        h_p[j] = r.p;
        h_thr[j] = (uint64_t)(r.p * 9007199254740992.0);
        h_mix[j] = splitmix64(r.seed);
        m += g->m;
        n += g->n;
    }
    h_eoff[k] = m;
    h_voff[k] = (uint32_t)n;
    u.eoff = reinterpret_cast<uint64_t *>(sl.d_params + L.eoff);
    u.voff = reinterpret_cast<uint32_t *>(sl.d_params + L.voff);
    u.p = reinterpret_cast<double *>(sl.d_params + L.p);
    u.thr = reinterpret_cast<uint64_t *>(sl.d_params + L.thr);
    u.seed_mix = reinterpret_cast<uint64_t *>(sl.d_params + L.mix);
    if (k == 1 && m > 0) {
        // a wave of one request counts the resident copy in place (its keys
        // are already the union's: one graph at vertex offset 0), as one
        // CUDA graph captured the first time this graph comes alone to this
        // slot: parameters in, the count, results out
        GraphEntry *g = sl.wave_graphs[0];
        u.rel = g->dev;
        u.orig = g->dev + m;
        if (!g->exec[si]) {
            const unsigned long long l0 = tc_launch_count();
            cudaGraph_t graph = nullptr;
            if (cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal) == cudaSuccess) {
                cudaMemcpyAsync(sl.d_params, sl.h_params, L.bytes, cudaMemcpyHostToDevice, s);
                union_count(u, m, (uint32_t)n, 1, IsectConfig{}, s);
                cudaMemcpyAsync(sl.h_res, u.res_dev, sizeof(tc_result), cudaMemcpyDeviceToHost, s);
                cudaMemcpyAsync(sl.h_st, u.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
                if (cudaStreamEndCapture(s, &graph) == cudaSuccess && graph) {
                    if (cudaGraphInstantiate(&g->exec[si], graph, 0) != cudaSuccess) g->exec[si] = nullptr;
                    cudaGraphDestroy(graph);
                }
            }
            cudaGetLastError();
            g->exec_launches[si] = tc_launch_count() - l0;  // counted once, at capture
        } else {
            add_launches(g->exec_launches[si]);
        }
        if (g->exec[si]) {
            if (cudaGraphLaunch(g->exec[si], s) != cudaSuccess) {
                cudaGetLastError();
                return TC_ECUDA;
            }
            cudaEventRecord(sl.done_ev, s);
            if (cudaLaunchHostFunc(s, on_slot_done, &srv->cb[si]) != cudaSuccess) {
                cudaGetLastError();
                return TC_ECUDA;
            }
            return TC_OK;
        }
    }
    cudaMemcpyAsync(sl.d_params, sl.h_params, L.bytes, cudaMemcpyHostToDevice, s);
    if (k == 1 && m > 0) {
        u.rel = sl.wave_graphs[0]->dev;
        u.orig = sl.wave_graphs[0]->dev + m;
    } else if (m > 0) {
        k_gather<<<grid_for(m, 256, 152 * 8), 256, 0, s>>>(
            reinterpret_cast<const uint64_t *const *>(sl.d_params + L.src), u.eoff, u.voff, k, m, u.rel, u.orig);
        note_launch();
    }
    union_count(u, m, (uint32_t)n, k, IsectConfig{}, s);
    cudaMemcpyAsync(sl.h_res, sl.u.res_dev, k * sizeof(tc_result), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(sl.h_st, sl.u.st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
    cudaEventRecord(sl.done_ev, s);
    if (cudaGetLastError() != cudaSuccess) return TC_ECUDA;
    if (cudaLaunchHostFunc(s, on_slot_done, &srv->cb[si]) != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    return TC_OK;
}

void worker_main(tc_server *srv)
{
    cudaSetDevice(srv->device);
    std::unique_lock<std::mutex> lock(srv->mu);
    for (;;) {
        for (uint32_t i = 0; i < srv->nslots; ++i)
            if (srv->slots[i].busy && cudaEventQuery(srv->slots[i].done_ev) == cudaSuccess) complete_wave(srv, i);
        cudaGetLastError();  // cudaErrorNotReady of the waves still running
        bool any_busy = false;
        for (uint32_t i = 0; i < srv->nslots; ++i) any_busy |= srv->slots[i].busy;
        if (srv->stop && !any_busy) break;
        bool launched = false;
        if (!srv->stop) {
            // slots are tried from the one the head request's graph maps to, so
            // that its single-request waves keep using the same captured launch
            const uint32_t first = srv->queue.empty() ? 0u : srv->queue.front().gid % srv->nslots;
            for (uint32_t j = 0; j < srv->nslots && !srv->queue.empty(); ++j) {
                const uint32_t i = (first + j) % srv->nslots;
                Slot &sl = srv->slots[i];
                if (sl.busy) continue;
                std::vector<GraphEntry *> uploads;
                std::vector<uint64_t *> frees;
                std::vector<cudaGraphExec_t> dead;
                if (!form_wave(srv, i, uploads, frees, dead)) break;  // the head waits for memory
                sl.busy = true;
                sl.serial = ++srv->wave_serial;
                sl.t_admit = now_us(srv->t0);
                srv->stats.waves += 1;
                srv->stats.max_wave = std::max<uint64_t>(srv->stats.max_wave, sl.wave.size());
                srv->stats.queued = srv->queue.size();
                lock.unlock();
                const tc_status st = enqueue_wave(srv, i, uploads, frees, dead);
                if (st != TC_OK) cudaStreamSynchronize(sl.s);  // no callback will come
                lock.lock();
                if (st != TC_OK) {
                    sl.launch_status = st;
                    for (GraphEntry *g : uploads)
                        if (!g->dev && g->resident) {  // upload failed: uncharge
                            g->resident = false;
                            srv->resident_bytes -= g->dev_bytes;
                            --srv->stats.resident_graphs;
                            srv->lru.erase(g->lru);
                        }
                    complete_wave(srv, i);
                    sl.launch_status = TC_OK;
                }
                launched = true;
            }
        }
        if (launched) continue;
        // waves in flight: poll their completion events for up to 2 ms before
        // sleeping (the host callback of each wave still wakes a sleeping
        // worker), so that a finished wave and a new request are seen at once
        bool in_flight = false;
        for (uint32_t i = 0; i < srv->nslots; ++i) in_flight |= srv->slots[i].busy;
        if (in_flight && !srv->stop) {
            const uint64_t seen = srv->arrivals.load(std::memory_order_acquire);
            const auto until = std::chrono::steady_clock::now() + std::chrono::milliseconds(2);
            bool progressed = false;
            lock.unlock();  // busy is written by this thread only
            while (!progressed && std::chrono::steady_clock::now() < until) {
                for (uint32_t i = 0; i < srv->nslots && !progressed; ++i)
                    progressed = srv->slots[i].busy && cudaEventQuery(srv->slots[i].done_ev) == cudaSuccess;
                progressed |= srv->arrivals.load(std::memory_order_acquire) != seen;
                if (!progressed) std::this_thread::yield();
            }
            cudaGetLastError();
            lock.lock();
            if (progressed) continue;
        }
        srv->work_cv.wait(lock);
    }
}

void free_server(tc_server *srv)
{
    if (!srv) return;
    if (srv->worker.joinable()) {
        {
            std::lock_guard<std::mutex> lock(srv->mu);
            srv->stop = true;
        }
        srv->work_cv.notify_all();
        srv->worker.join();
    }
    cudaSetDevice(srv->device);
    for (uint32_t i = 0; i < srv->nslots; ++i) {
        Slot &sl = srv->slots[i];
        if (sl.s) cudaStreamSynchronize(sl.s);
    }
    for (auto &g : srv->graphs) {
        if (g->dev) cudaFreeAsync(g->dev, srv->ingest);
        for (cudaGraphExec_t e : g->exec)
            if (e) cudaGraphExecDestroy(e);
        if (g->host) cudaFreeHost(g->host);
        if (g->ready) cudaEventDestroy(g->ready);
    }
    if (srv->ingest) {
        cudaStreamSynchronize(srv->ingest);
        cudaStreamDestroy(srv->ingest);
    }
    for (uint32_t i = 0; i < srv->nslots; ++i) {
        Slot &sl = srv->slots[i];
        cudaFreeHost(sl.h_params);
        cudaFreeHost(sl.h_res);
        cudaFreeHost(sl.h_st);
        if (sl.done_ev) cudaEventDestroy(sl.done_ev);
        if (sl.s) cudaStreamDestroy(sl.s);
    }
    for (void *p : srv->allocs) cudaFree(p);
    cudaGetLastError();
    delete srv;
}

template <typename T>
bool pinned(T **p, uint64_t count)
{
    if (cudaMallocHost((void **)p, std::max<uint64_t>(count, 1) * sizeof(T)) != cudaSuccess) {
        cudaGetLastError();
        *p = nullptr;
        return false;
    }
    return true;
}

}  // namespace

extern "C" {

tc_status tc_server_create(uint64_t budget_bytes, uint32_t slots, uint64_t slot_edges, uint32_t slot_vertices,
                           uint32_t slot_requests, tc_server **out)
{
    if (!out) return TC_EINVAL;
    *out = nullptr;
    if (slots == 0 || slots > MAX_SLOTS || slot_edges == 0 || slot_edges > 0xfffffffeull || slot_vertices == 0 ||
        slot_vertices > 0xfffffffeu || slot_requests == 0 || slot_requests > 0xffffu)
        return TC_EINVAL;
    tc_server *srv = new (std::nothrow) tc_server;
    if (!srv) return TC_ENOMEM;
    cudaGetDevice(&srv->device);
    srv->budget = budget_bytes;
    srv->slot_edges = slot_edges;
    srv->slot_vertices = slot_vertices;
    srv->slot_requests = slot_requests;
    srv->t0 = std::chrono::steady_clock::now();
    if (cudaStreamCreateWithFlags(&srv->ingest, cudaStreamNonBlocking) != cudaSuccess) {
        cudaGetLastError();
        free_server(srv);
        return TC_ECUDA;
    }
    for (uint32_t i = 0; i < slots; ++i) {
        Slot &sl = srv->slots[i];
        srv->nslots = i + 1;
        srv->cb[i] = CallbackCtx{srv, i};
        if (cudaStreamCreateWithFlags(&sl.s, cudaStreamNonBlocking) != cudaSuccess ||
            cudaEventCreateWithFlags(&sl.done_ev, cudaEventDisableTiming) != cudaSuccess) {
            cudaGetLastError();
            free_server(srv);
            return TC_ECUDA;
        }
        const uint64_t k = slot_requests, pbytes = wave_layout((uint32_t)k).bytes;
        if (!pinned(&sl.h_params, pbytes) || !pinned(&sl.h_res, k) || !pinned(&sl.h_st, 1)) {
            free_server(srv);
            return TC_ENOMEM;
        }
        void *dparams = nullptr;
        if (cudaMalloc(&dparams, pbytes) != cudaSuccess) {
            cudaGetLastError();
            free_server(srv);
            return TC_ENOMEM;
        }
        srv->allocs.push_back(dparams);
        srv->slot_bytes += pbytes;
        sl.d_params = (unsigned char *)dparams;
        if (!union_scratch_alloc(sl.u, slot_edges, slot_vertices, slot_requests, srv->allocs, srv->slot_bytes)) {
            free_server(srv);
            return TC_ENOMEM;
        }
    }
    if (srv->slot_bytes > budget_bytes) {
        free_server(srv);
        return TC_ENOMEM;
    }
    srv->stats.budget_bytes = budget_bytes;
    srv->stats.slot_bytes = srv->slot_bytes;
    if (cudaDeviceSynchronize() != cudaSuccess) {
        cudaGetLastError();
        free_server(srv);
        return TC_ECUDA;
    }
    try {
        srv->worker = std::thread(worker_main, srv);
    } catch (...) {
        free_server(srv);
        return TC_ENOMEM;
    }
    *out = srv;
    return TC_OK;
}

void tc_server_destroy(tc_server *srv) { free_server(srv); }

tc_status tc_server_add_graph(tc_server *srv, const uint32_t *edges, uint64_t m_in, uint32_t n, int edges_on_device,
                              uint32_t *gid)
{
    if (!srv || !gid || n == 0 || n == 0xffffffffu || m_in > 0xfffffffeull || (m_in > 0 && !edges))
        return TC_EINVAL;
    std::lock_guard<std::mutex> ingest_lock(srv->ingest_mu);
    cudaSetDevice(srv->device);
    cudaStream_t s = srv->ingest;
    auto g = std::make_unique<GraphEntry>();
    g->n = n;
    if (cudaEventCreateWithFlags(&g->ready, cudaEventDisableTiming) != cudaSuccess) {
        cudaGetLastError();
        return TC_ECUDA;
    }
    // ---- canonical keys (as tc_graph_create): map, sort by (u, v), unique
    std::vector<void *> tmp;
    auto talloc = [&](uint64_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMallocAsync(&p, std::max<uint64_t>(bytes, 16), s) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        tmp.push_back(p);
        return p;
    };
    auto drop = [&](tc_status st) {
        for (void *p : tmp) cudaFreeAsync(p, s);
        cudaStreamSynchronize(s);
        cudaGetLastError();
        if (g->ready) cudaEventDestroy(g->ready);
        if (g->host) cudaFreeHost(g->host);
        return st;
    };
    uint64_t m = 0;
    uint64_t *canon = nullptr;
    if (m_in > 0) {
        const uint32_t *dpairs = edges;
        if (!edges_on_device) {
            void *p = talloc(m_in * 8);
            if (!p) return drop(TC_ENOMEM);
            cudaMemcpyAsync(p, edges, m_in * 8, cudaMemcpyHostToDevice, s);
            dpairs = (const uint32_t *)p;
        }
        const uint64_t nt = ceil_div(m_in, RX_TILE);
        uint64_t *a = (uint64_t *)talloc(m_in * 8), *b = (uint64_t *)talloc(m_in * 8);
        uint32_t *hist = (uint32_t *)talloc((nt << RX_MAX_BITS) * 4);
        uint32_t *scan = (uint32_t *)talloc(scan_scratch_elems(nt << RX_MAX_BITS) * 4);
        DevState *st = (DevState *)talloc(sizeof(DevState));
        DevState *h_st = nullptr;
        if (!a || !b || !hist || !scan || !st) return drop(TC_ENOMEM);
        if (!pinned(&h_st, 1)) return drop(TC_ENOMEM);
        cudaMemsetAsync(st, 0, sizeof(DevState), s);
        canon_keys(dpairs, m_in, n, a, st, s);
        const int nbits = key_bits(n);
        for (int half = 0; half < 2; ++half) {
            int shift = half ? 32 : 0;
            const int P = (nbits + RX_MAX_BITS - 1) / RX_MAX_BITS;
            for (int i = 0; i < P; ++i) {
                const int w = nbits / P + (i < nbits % P ? 1 : 0);
                radix_pass(a, m_in, shift, w, hist, scan, b, s);
                std::swap(a, b);
                shift += w;
            }
        }
        unique_keys(a, m_in, b, hist, scan, st, s);
        cudaMemcpyAsync(h_st, st, sizeof(DevState), cudaMemcpyDeviceToHost, s);
        const bool ok = cudaStreamSynchronize(s) == cudaSuccess;
        const DevState hs = *h_st;
        cudaFreeHost(h_st);
        if (!ok) return drop(TC_ECUDA);
        if (hs.err & ERR_ENDPOINT) return drop(TC_EINVAL);
        m = hs.m_canon;
        if (m > 0) {
            // rank relabeling (csr.cu) into one block: rel keys, then original keys
            const uint64_t hl = std::max<uint64_t>(ceil_div(std::max<uint64_t>(m, n), RX_TILE), 1) << RX_MAX_BITS;
            uint64_t *blk = (uint64_t *)talloc(m * 16), *kb = (uint64_t *)talloc(m * 8);
            uint64_t *va = (uint64_t *)talloc((uint64_t)n * 8), *vb = (uint64_t *)talloc((uint64_t)n * 8);
            uint32_t *perm = (uint32_t *)talloc((uint64_t)n * 4), *rank = (uint32_t *)talloc((uint64_t)n * 4);
            uint32_t *deg = (uint32_t *)talloc((uint64_t)n * 4), *hist2 = (uint32_t *)talloc(hl * 4);
            uint32_t *scan2 = (uint32_t *)talloc(scan_scratch_elems(std::max<uint64_t>(hl, (uint64_t)n + 2)) * 4);
            if (!blk || !kb || !va || !vb || !perm || !rank || !deg || !hist2 || !scan2) return drop(TC_ENOMEM);
            const RelabelScratch sc{a, kb, va, vb, deg, hist2, scan2};
            relabel(b, m, n, nullptr, 0, Relabeled{blk, blk + m, perm, rank}, sc, s);
            canon = blk;
        }
    }
    g->m = m;
    g->dev_bytes = m * 16;
    if (m > srv->slot_edges || n > srv->slot_vertices) return drop(TC_EINVAL);
    if (g->dev_bytes > srv->budget - srv->slot_bytes) return drop(TC_ENOMEM);
    if (m > 0) {
        if (!pinned(&g->host, 2 * m)) return drop(TC_ENOMEM);
        cudaMemcpyAsync(g->host, canon, m * 16, cudaMemcpyDeviceToHost, s);
    }
    // resident right away if that needs no eviction
    bool keep = false;
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        keep = m > 0 && srv->resident_bytes + g->dev_bytes <= srv->budget - srv->slot_bytes;
        if (keep) srv->resident_bytes += g->dev_bytes;  // reserve
    }
    if (keep) {
        if (cudaMallocAsync((void **)&g->dev, m * 16, s) == cudaSuccess) {
            cudaMemcpyAsync(g->dev, canon, m * 16, cudaMemcpyDeviceToDevice, s);
        } else {
            cudaGetLastError();
            g->dev = nullptr;
        }
    }
    for (void *p : tmp) cudaFreeAsync(p, s);
    tmp.clear();
    if (cudaStreamSynchronize(s) != cudaSuccess) {
        cudaGetLastError();
        if (keep) {
            std::lock_guard<std::mutex> lock(srv->mu);
            srv->resident_bytes -= g->dev_bytes;
        }
        if (g->dev) cudaFreeAsync(g->dev, s);
        g->dev = nullptr;
        return drop(TC_ECUDA);
    }
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        if (keep && !g->dev) srv->resident_bytes -= g->dev_bytes;  // allocation failed: upload on demand
        g->resident = g->dev != nullptr;
        const uint32_t id = (uint32_t)srv->graphs.size();
        if (g->resident) {
            g->lru = srv->lru.insert(srv->lru.end(), id);
            ++srv->stats.resident_graphs;
        }
        srv->graphs.push_back(std::move(g));
        srv->stats.graphs = srv->graphs.size();
        *gid = id;
    }
    srv->work_cv.notify_all();  // a released reservation may let the queue head in
    return TC_OK;
}

tc_status tc_server_submit(tc_server *srv, uint32_t gid, double p, uint64_t seed, uint64_t *ticket)
{
    if (!srv || !ticket || !(p > 0.0 && p <= 1.0)) return TC_EINVAL;
    const double t = now_us(srv->t0);
    {
        std::lock_guard<std::mutex> lock(srv->mu);
        if (gid >= srv->graphs.size() || srv->stop) return TC_EINVAL;
        const uint64_t id = srv->next_ticket++;
        Record rec;
        std::memset(&rec.info, 0, sizeof(rec.info));
        rec.info.t_submit_us = t;
        srv->records.emplace(id, rec);
        srv->queue.push_back(Req{id, gid, p, seed, t});
        srv->arrivals.fetch_add(1, std::memory_order_release);
        ++srv->stats.submitted;
        srv->stats.queued = srv->queue.size();
        *ticket = id;
    }
    srv->work_cv.notify_all();
    return TC_OK;
}

tc_status tc_server_poll(tc_server *srv, uint64_t ticket, tc_request_info *info)
{
    if (!srv || !info) return TC_EINVAL;
    std::lock_guard<std::mutex> lock(srv->mu);
    auto it = srv->records.find(ticket);
    if (it == srv->records.end()) return TC_EINVAL;
    if (!it->second.done) return TC_EBUSY;
    *info = it->second.info;
    srv->records.erase(it);
    return TC_OK;
}

tc_status tc_server_wait(tc_server *srv, uint64_t ticket, uint32_t timeout_ms, tc_request_info *info)
{
    if (!srv || !info) return TC_EINVAL;
    std::unique_lock<std::mutex> lock(srv->mu);
    const auto deadline = std::chrono::steady_clock::now() + std::chrono::milliseconds(timeout_ms);
    for (;;) {
        auto it = srv->records.find(ticket);
        if (it == srv->records.end()) return TC_EINVAL;
        if (it->second.done) {
            *info = it->second.info;
            srv->records.erase(it);
            return TC_OK;
        }
        if (srv->done_cv.wait_until(lock, deadline) == std::cv_status::timeout) {
            auto again = srv->records.find(ticket);
            if (again != srv->records.end() && again->second.done) continue;
            return TC_EBUSY;
        }
    }
}

tc_status tc_server_get_stats(tc_server *srv, tc_server_stats *out)
{
    if (!srv || !out) return TC_EINVAL;
    std::lock_guard<std::mutex> lock(srv->mu);
    srv->stats.resident_bytes = srv->resident_bytes;
    srv->stats.queued = srv->queue.size();
    *out = srv->stats;
    return TC_OK;
}

}  // extern "C"
