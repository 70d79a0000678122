// Semi-streaming triangle counting (Section 5.2): three passes over an
// adjacency-list stream that stays in host memory, for graphs whose edges
// do not fit in device memory.
//
// The stream is the symmetric adjacency of a simple graph, off[n + 1] and
// adj[2 m] with every list sorted by id (each edge appears in both of its
// endpoints' lists).  Only O(n) vertex arrays, the samples and the query
// table live on the device; the edges pass through it in chunks (mapped
// pinned memory is read in place over the host link, other host memory is
// copied chunk by chunk into two device buffers).
//   Pass 1: degrees are the offsets; stream entry j is sampled iff
//     (splitmix64(j ^ splitmix64(seed + 1)) >> 11) < floor(q 2^53),
//     q = min(1, c m^(1/2) ln n / (2 m)), and both endpoints of a sampled
//     entry are heavy candidates; H = the candidates with deg^2 > m.  The
//     pass also counts every vertex's entries above itself and checks the
//     lists (sorted, no self-loops, endpoints < n).
//   U: the wedges of the vertices outside H (C(d, 2) each, vertex order,
//     wedge b (b - 1) / 2 + a), then the pairs (edge e, H[i]), index
//     |U_L| + e |H| + i, the edges being the entries u < v in stream order.
//     Every triangle is in U three times (once per corner).
//   Draws: sample i is U's triple floor(h_i |U| / 2^64), h_i =
//     splitmix64(i ^ splitmix64(~seed)); the stream positions of the list
//     entries it needs are sorted so that each chunk fills its own.
//   Pass 2: the chunks hand the samples their entries; the third edges of
//     the samples go into a device hash table of queries.
//   Pass 3: every edge of the stream is looked up in the table, marking the
//     queries that exist.
// estimate = |U| (c_w + c_p) / (3 s).
#include <algorithm>
#include <cmath>
#include <vector>

#include "kernels.h"

namespace tcg {
namespace {

constexpr unsigned SP_THREADS = 256;
constexpr uint64_t SP_EMPTY = ~0ull;
constexpr int SLOT_BITS = 31;  // request = stream position << 31 | sample slot
constexpr uint64_t SLOT_MASK = (1ull << SLOT_BITS) - 1;

struct StreamDev {
    unsigned long long sampled, candidates, cw, cp, r0, r1;
    unsigned int n_heavy, err;
};

__device__ __forceinline__ uint64_t edge_key(uint32_t a, uint32_t b)
{
    return a < b ? ((uint64_t)a << 32) | b : ((uint64_t)b << 32) | a;
}

__device__ __forceinline__ uint64_t table_slot(uint64_t key, int bits)
{
    return (key * 0x9e3779b97f4a7c15ull) >> (64 - bits);
}

__device__ void table_insert(unsigned long long *keys, int bits, uint64_t key)
{
    const uint64_t mask = (1ull << bits) - 1;
    uint64_t s = table_slot(key, bits);
    for (uint64_t it = 0; it <= mask; ++it, s = (s + 1) & mask) {
        const unsigned long long prev = atomicCAS(keys + s, SP_EMPTY, (unsigned long long)key);
        if (prev == SP_EMPTY || prev == key) return;
    }
}

__device__ __forceinline__ int64_t table_find(const unsigned long long *keys, int bits, uint64_t key)
{
    const uint64_t mask = (1ull << bits) - 1;
    uint64_t s = table_slot(key, bits);
    for (uint64_t it = 0; it <= mask; ++it, s = (s + 1) & mask) {
        const unsigned long long k = keys[s];
        if (k == key) return (int64_t)s;
        if (k == SP_EMPTY) return -1;
    }
    return -1;
}

// Pass 1 over entries [j0, j1) (chunk[j - j0]): list checks, entries above
// their row, sampled entries' endpoints as heavy candidates.  prev: the
// entry before j0 (its row's order continues across the chunk border).
__global__ void k_sp_pass1(const uint32_t *__restrict__ chunk, uint64_t j0, uint64_t j1,
                           const uint64_t *__restrict__ off, uint32_t n, uint32_t prev, uint64_t hmix, uint64_t thr,
                           uint8_t *__restrict__ cand, unsigned long long *__restrict__ up, StreamDev *sd)
{
    const unsigned lane = lane_id();
    const uint64_t len = j1 - j0, stride = (uint64_t)gridDim.x * blockDim.x;
    unsigned long long sampled = 0;
    unsigned bad = 0;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < len; base += stride) {
        const uint64_t t = base + lane, j = j0 + (t < len ? t : len - 1);
        const uint32_t u = find_part_warp(off, n, (uint64_t)j);
        const bool live = t < len;
        const uint32_t v = live ? chunk[t] : 0u;
        bool above = false;
        if (live) {
            if (v >= n || v == u) bad = 1;
            if (j > off[u]) {
                const uint32_t pv = t > 0 ? chunk[t - 1] : prev;
                if (pv >= v) bad = 1;
            }
            above = v > u;
            if ((splitmix64(j ^ hmix) >> 11) < thr) {
                ++sampled;
                if (v < n) {
                    cand[u] = 1;
                    cand[v] = 1;
                }
            }
        }
        const unsigned act = __ballot_sync(FULL, above);
        if (above) {
            const unsigned grp = __match_any_sync(act, u);
            if ((int)lane == __ffs(grp) - 1) atomicAdd(up + u, (unsigned long long)__popc(grp));
        }
    }
    sampled = warp_sum(sampled);
    if (lane == 0 && sampled) atomicAdd(&sd->sampled, sampled);
    if (bad) atomicOr(&sd->err, ERR_ENDPOINT);
}

// Classes: H = candidates with deg^2 > m; wedge counts of the rest; H's
// members numbered in id order through hpos (an exclusive scan follows).
__global__ void k_sp_classes(const uint64_t *__restrict__ off, uint32_t n, unsigned long long m,
                             const uint8_t *__restrict__ cand, unsigned long long *__restrict__ wcnt,
                             uint32_t *__restrict__ hflag, StreamDev *sd)
{
    uint32_t h = 0, c = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u <= n; u += stride) {
        if (u == n) {
            wcnt[n] = 0;
            hflag[n] = 0;
            continue;
        }
        const unsigned long long d = off[u + 1] - off[u];
        const bool heavy = cand[u] && d * d > m;
        c += cand[u];
        h += heavy;
        hflag[u] = heavy;
        wcnt[u] = heavy ? 0ull : d * (d - (d > 0 ? 1ull : 0ull)) / 2;
    }
    h = warp_sum(h);
    c = warp_sum(c);
    if (lane_id() == 0) {
        if (h) atomicAdd(&sd->n_heavy, h);
        if (c) atomicAdd(&sd->candidates, (unsigned long long)c);
    }
}

// H[hpos[u]] = u for the heavy vertices (hpos: exclusive scan of the flags).
__global__ void k_sp_hlist(const uint32_t *__restrict__ hpos, uint32_t n, uint32_t *__restrict__ H)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t u = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride)
        if (hpos[u + 1] != hpos[u]) H[hpos[u]] = (uint32_t)u;
}

// Largest u in [0, n) with pre[u] <= r.
__device__ __forceinline__ uint32_t prefix_owner(const unsigned long long *__restrict__ pre, uint32_t n, uint64_t r)
{
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        const uint32_t mid = lo + ((hi - lo) >> 1);
        if (__ldg(pre + mid) <= r) lo = mid; else hi = mid;
    }
    return lo;
}

// The draws: each sample's kind, vertices and the stream positions of the
// entries it needs (requests; unused slots ~0).
__global__ void k_sp_draw(const uint64_t *__restrict__ off, uint32_t n, const unsigned long long *__restrict__ wpre,
                          const unsigned long long *__restrict__ uppre, const uint32_t *__restrict__ H, uint32_t h,
                          unsigned long long U, unsigned long long UL, uint64_t s, uint64_t tmix,
                          uint8_t *__restrict__ kind, uint32_t *__restrict__ ru, uint32_t *__restrict__ rx,
                          unsigned long long *__restrict__ req)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += stride) {
        const unsigned long long r = __umul64hi(splitmix64(i ^ tmix), U);
        if (r < UL) {
            const uint32_t u = prefix_owner(wpre, n, r);
            const unsigned long long k = r - __ldg(wpre + u);
            unsigned long long b = (unsigned long long)((1.0 + __dsqrt_rn(1.0 + 8.0 * (double)k)) * 0.5);
            if (b < 1) b = 1;
            while (b > 1 && b * (b - 1) / 2 > k) --b;
            while ((b + 1) * b / 2 <= k) ++b;
            const unsigned long long a = k - b * (b - 1) / 2;
            kind[i] = 0;
            ru[i] = u;
            req[2 * i] = ((off[u] + a) << SLOT_BITS) | (2 * i);
            req[2 * i + 1] = ((off[u] + b) << SLOT_BITS) | (2 * i + 1);
        } else {
            const unsigned long long k = r - UL, e = k / h;
            const uint32_t x = prefix_owner(uppre, n, e);
            const unsigned long long d = off[x + 1] - off[x], upx = __ldg(uppre + x + 1) - __ldg(uppre + x);
            kind[i] = 1;
            ru[i] = __ldg(H + (uint32_t)(k % h));
            rx[i] = x;
            req[2 * i] = ((off[x] + (d - upx) + (e - __ldg(uppre + x))) << SLOT_BITS) | (2 * i);
            req[2 * i + 1] = SP_EMPTY;
        }
    }
}

// The sorted requests whose positions lie in [j0, j1): [r0, r1).
__global__ void k_sp_range(const unsigned long long *__restrict__ req, uint64_t nreq, uint64_t j0, uint64_t j1,
                           StreamDev *sd)
{
    auto lower = [&](uint64_t pos) {
        uint64_t lo = 0, hi = nreq;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if ((req[mid] >> SLOT_BITS) < pos) lo = mid + 1; else hi = mid;
        }
        return lo;
    };
    sd->r0 = lower(j0);
    sd->r1 = lower(j1);
}

// Pass 2: the chunk's entries into the requesting samples' slots.
__global__ void k_sp_fill(const uint32_t *__restrict__ chunk, uint64_t j0, const unsigned long long *__restrict__ req,
                          const StreamDev *sd, uint32_t *__restrict__ val)
{
    const uint64_t r0 = sd->r0, r1 = sd->r1, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t t = r0 + (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < r1; t += stride) {
        const unsigned long long q = req[t];
        val[q & SLOT_MASK] = chunk[(q >> SLOT_BITS) - j0];
    }
}

// The samples' third edges into the query table.
__global__ void k_sp_queries(const uint8_t *__restrict__ kind, const uint32_t *__restrict__ ru,
                             const uint32_t *__restrict__ rx, const uint32_t *__restrict__ val, uint64_t s,
                             unsigned long long *__restrict__ keys, int bits)
{
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += stride) {
        if (kind[i] == 0) {
            table_insert(keys, bits, edge_key(val[2 * i], val[2 * i + 1]));
        } else {
            const uint32_t hv = ru[i], x = rx[i], y = val[2 * i];
            if (hv != x && hv != y) {
                table_insert(keys, bits, edge_key(hv, x));
                table_insert(keys, bits, edge_key(hv, y));
            }
        }
    }
}

// Pass 3: every edge (entries u < v) of the chunk marks its query.
__global__ void k_sp_pass3(const uint32_t *__restrict__ chunk, uint64_t j0, uint64_t j1,
                           const uint64_t *__restrict__ off, uint32_t n, const unsigned long long *__restrict__ keys,
                           int bits, uint8_t *__restrict__ found)
{
    const unsigned lane = lane_id();
    const uint64_t len = j1 - j0, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t base = (uint64_t)blockIdx.x * blockDim.x + (threadIdx.x & ~31u); base < len; base += stride) {
        const uint64_t t = base + lane, j = j0 + (t < len ? t : len - 1);
        const uint32_t u = find_part_warp(off, n, (uint64_t)j);
        if (t >= len) continue;
        const uint32_t v = chunk[t];
        if (v <= u) continue;
        const int64_t slot = table_find(keys, bits, ((uint64_t)u << 32) | v);
        if (slot >= 0) found[slot] = 1;
    }
}

__global__ void k_sp_count(const uint8_t *__restrict__ kind, const uint32_t *__restrict__ ru,
                           const uint32_t *__restrict__ rx, const uint32_t *__restrict__ val, uint64_t s,
                           const unsigned long long *__restrict__ keys, int bits, const uint8_t *__restrict__ found,
                           StreamDev *sd)
{
    unsigned long long cw = 0, cp = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < s; i += stride) {
        if (kind[i] == 0) {
            const int64_t q = table_find(keys, bits, edge_key(val[2 * i], val[2 * i + 1]));
            cw += q >= 0 && found[q];
        } else {
            const uint32_t hv = ru[i], x = rx[i], y = val[2 * i];
            if (hv == x || hv == y) continue;
            const int64_t q1 = table_find(keys, bits, edge_key(hv, x)), q2 = table_find(keys, bits, edge_key(hv, y));
            cp += q1 >= 0 && q2 >= 0 && found[q1] && found[q2];
        }
    }
    cw = warp_sum(cw);
    cp = warp_sum(cp);
    if (lane_id() == 0) {
        if (cw) atomicAdd(&sd->cw, cw);
        if (cp) atomicAdd(&sd->cp, cp);
    }
}

}  // namespace

// ---------------------------------------------------------------- host

tc_status stream_count(const uint64_t *off_host, const uint32_t *adj_host, uint32_t n, uint64_t seed,
                       uint64_t samples, double c, uint64_t chunk_entries, cudaStream_t s, tc_stream_result *res)
{
    const uint64_t len = off_host[n], m = len / 2;
    *res = tc_stream_result{};
    res->m = m;
    res->n = n;
    std::vector<void *> allocs;
    auto alloc = [&](uint64_t bytes) -> void * {
        void *p = nullptr;
        if (cudaMalloc(&p, std::max<uint64_t>(bytes, 256)) != cudaSuccess) {
            cudaGetLastError();
            return nullptr;
        }
        allocs.push_back(p);
        return p;
    };
    auto finish = [&](tc_status st) {
        cudaStreamSynchronize(s);
        for (void *p : allocs) cudaFree(p);
        cudaGetLastError();
        return st;
    };

    // the stream: read in place when it is mapped pinned memory, else staged
    const uint32_t *adj_dev = nullptr;
    cudaPointerAttributes pa;
    if (len > 0 && cudaPointerGetAttributes(&pa, adj_host) == cudaSuccess && pa.type == cudaMemoryTypeHost &&
        pa.devicePointer)
        adj_dev = (const uint32_t *)pa.devicePointer;
    cudaGetLastError();
    if (chunk_entries == 0) chunk_entries = 1ull << 26;
    chunk_entries = std::min<uint64_t>(chunk_entries, std::max<uint64_t>(len, 1));
    const uint64_t nchunks = len ? (len + chunk_entries - 1) / chunk_entries : 0;

    uint64_t *d_off = (uint64_t *)alloc(((uint64_t)n + 1) * 8);
    uint8_t *cand = (uint8_t *)alloc((uint64_t)n + 1);
    unsigned long long *up = (unsigned long long *)alloc(((uint64_t)n + 1) * 8);
    unsigned long long *wcnt = (unsigned long long *)alloc(((uint64_t)n + 1) * 8);
    uint32_t *hflag = (uint32_t *)alloc(((uint64_t)n + 1) * 4);
    unsigned long long *scan64 = (unsigned long long *)alloc((ceil_div((uint64_t)n + 1, SC_CHUNK) + 1) * 8);
    uint32_t *scan32 = (uint32_t *)alloc(scan_scratch_elems((uint64_t)n + 1) * 4);
    StreamDev *sd = (StreamDev *)alloc(sizeof(StreamDev));
    uint32_t *buf[2] = {nullptr, nullptr};
    if (!adj_dev && len > 0) {
        buf[0] = (uint32_t *)alloc(chunk_entries * 4);
        buf[1] = (uint32_t *)alloc(chunk_entries * 4);
    }
    if (!d_off || !cand || !up || !wcnt || !hflag || !scan64 || !scan32 || !sd || (!adj_dev && len > 0 && !buf[1]))
        return finish(TC_ENOMEM);
    cudaMemcpyAsync(d_off, off_host, ((uint64_t)n + 1) * 8, cudaMemcpyHostToDevice, s);
    cudaMemsetAsync(cand, 0, (uint64_t)n + 1, s);
    cudaMemsetAsync(up, 0, ((uint64_t)n + 1) * 8, s);
    cudaMemsetAsync(sd, 0, sizeof(StreamDev), s);

    // one pass over the stream: kernel(chunk pointer, j0, j1, entry before j0)
    auto pass = [&](auto &&kernel) {
        for (uint64_t ci = 0; ci < nchunks; ++ci) {
            const uint64_t j0 = ci * chunk_entries, j1 = std::min(len, j0 + chunk_entries);
            const uint32_t *chunk = adj_dev ? adj_dev + j0 : buf[ci & 1];
            if (!adj_dev)
                cudaMemcpyAsync(buf[ci & 1], adj_host + j0, (j1 - j0) * 4, cudaMemcpyHostToDevice, s);
            kernel(chunk, j0, j1, j0 > 0 ? adj_host[j0 - 1] : 0u);
            res->bytes_streamed += (j1 - j0) * 4;
        }
        res->passes++;
    };
    const unsigned egrid = grid_for(std::min<uint64_t>(chunk_entries, std::max<uint64_t>(len, 1)), SP_THREADS, 152 * 16);

    // ---- pass 1
    double q = 0.0;
    if (m > 0 && n > 1) {
        q = c * std::sqrt((double)m) * std::log((double)n) / (2.0 * (double)m);
        if (q > 1.0) q = 1.0;
    }
    const uint64_t thr = (uint64_t)(q * 9007199254740992.0), hmix = splitmix64(seed + 1);
    pass([&](const uint32_t *chunk, uint64_t j0, uint64_t j1, uint32_t prev) {
        k_sp_pass1<<<egrid, SP_THREADS, 0, s>>>(chunk, j0, j1, d_off, n, prev, hmix, thr, cand, up, sd);
        note_launch();
    });
    k_sp_classes<<<grid_for((uint64_t)n + 1, SP_THREADS, 152 * 8), SP_THREADS, 0, s>>>(d_off, n, m, cand, wcnt, hflag,
                                                                                     sd);
    note_launch();
    scan_excl_u64(wcnt, (uint64_t)n + 1, nullptr, scan64, s);
    scan_excl_u64(up, (uint64_t)n + 1, nullptr, scan64, s);
    scan_excl_u32(hflag, (uint64_t)n + 1, nullptr, scan32, s);
    StreamDev hs;
    unsigned long long tails[2];
    cudaMemcpyAsync(&hs, sd, sizeof(hs), cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&tails[0], wcnt + n, 8, cudaMemcpyDeviceToHost, s);
    cudaMemcpyAsync(&tails[1], up + n, 8, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return finish(TC_ECUDA);
    if (hs.err || tails[1] != m) return finish(TC_EINVAL);  // not a sorted symmetric simple adjacency
    const uint32_t h = hs.n_heavy;
    res->n_heavy = h;
    res->candidates = hs.candidates;
    res->sampled_entries = hs.sampled;
    const unsigned long long UL = tails[0];
    if (h && m > (~0ull - UL) / h) return finish(TC_EINVAL);  // |U| beyond 64 bits
    const unsigned long long U = UL + (unsigned long long)m * h;
    res->universe = U;
    const uint64_t ns = samples ? samples : m;
    res->samples = ns;
    if (ns > (1ull << 30)) return finish(TC_EINVAL);
    if (U == 0 || ns == 0) return finish(TC_OK);

    uint32_t *H = (uint32_t *)alloc((uint64_t)std::max<uint32_t>(h, 1) * 4);
    uint8_t *kind = (uint8_t *)alloc(ns);
    uint32_t *ru = (uint32_t *)alloc(ns * 4), *rx = (uint32_t *)alloc(ns * 4), *val = (uint32_t *)alloc(ns * 8);
    unsigned long long *req = (unsigned long long *)alloc(ns * 16), *req2 = (unsigned long long *)alloc(ns * 16);
    int bits = 4;
    while ((1ull << bits) < 4 * ns) ++bits;  // at most 2 s queries: load <= 1/2
    unsigned long long *keys = (unsigned long long *)alloc((1ull << bits) * 8);
    uint8_t *found = (uint8_t *)alloc(1ull << bits);
    const uint64_t nreq = 2 * ns;
    const uint64_t hist_len = std::max<uint64_t>(ceil_div(nreq, RX_TILE), 1) << RX_MAX_BITS;
    uint32_t *hist = (uint32_t *)alloc(hist_len * 4), *hscan = (uint32_t *)alloc(scan_scratch_elems(hist_len) * 4);
    if (!H || !kind || !ru || !rx || !val || !req || !req2 || !keys || !found || !hist || !hscan)
        return finish(TC_ENOMEM);
    k_sp_hlist<<<grid_for(n, SP_THREADS, 152 * 8), SP_THREADS, 0, s>>>(hflag, n, H);
    note_launch();

    // ---- the draws, and their requests sorted by stream position
    const unsigned sgrid = grid_for(ns, SP_THREADS, 152 * 16);
    k_sp_draw<<<sgrid, SP_THREADS, 0, s>>>(d_off, n, wcnt, up, H, h, U, UL, ns, splitmix64(~seed), kind, ru, rx, req);
    note_launch();
    int pbits = 1;
    while (pbits < 64 - SLOT_BITS && (1ull << pbits) < len + 1) ++pbits;
    unsigned long long *a = req, *b = req2;
    for (int shift = SLOT_BITS, left = pbits; left > 0;) {
        const int w = std::min(left, RX_MAX_BITS);
        radix_pass((const uint64_t *)a, nreq, shift, w, hist, hscan, (uint64_t *)b, s);
        std::swap(a, b);
        shift += w;
        left -= w;
    }

    // ---- pass 2: entries into the samples, then the query table
    pass([&](const uint32_t *chunk, uint64_t j0, uint64_t j1, uint32_t) {
        k_sp_range<<<1, 1, 0, s>>>(a, nreq, j0, j1, sd);
        k_sp_fill<<<sgrid, SP_THREADS, 0, s>>>(chunk, j0, a, sd, val);
        note_launch();
        note_launch();
    });
    cudaMemsetAsync(keys, 0xff, (1ull << bits) * 8, s);
    cudaMemsetAsync(found, 0, 1ull << bits, s);
    k_sp_queries<<<sgrid, SP_THREADS, 0, s>>>(kind, ru, rx, val, ns, keys, bits);
    note_launch();

    // ---- pass 3: the stream's edges mark the queries that exist
    pass([&](const uint32_t *chunk, uint64_t j0, uint64_t j1, uint32_t) {
        k_sp_pass3<<<egrid, SP_THREADS, 0, s>>>(chunk, j0, j1, d_off, n, keys, bits, found);
        note_launch();
    });
    k_sp_count<<<sgrid, SP_THREADS, 0, s>>>(kind, ru, rx, val, ns, keys, bits, found, sd);
    note_launch();
    cudaMemcpyAsync(&hs, sd, sizeof(hs), cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return finish(TC_ECUDA);
    res->closed_wedge = hs.cw;
    res->closed_pair = hs.cp;
    res->estimate = ((double)U * (double)(hs.cw + hs.cp)) / (3.0 * (double)ns);
    return finish(TC_OK);
}

}  // namespace tcg
