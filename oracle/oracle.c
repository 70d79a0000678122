/*
 * CPU oracle for the edge-sampled, degree-partitioned triangle counter.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * statement of what the method computes.  Only the tests, the smoke check
 * and the CPU-baseline leg of the benchmark use it; the CUDA library never
 * links, calls or includes it, and it shares no code with that library.
 *
 * What it follows (Kolountzakis, Miller, Peng, Tsourakakis, "Efficient
 * Triangle Counting in Large Graphs via Degree-based Vertex Partitioning"):
 *   - Section 4.1: graphs are simple; multi-edges and self-loops are removed.
 *   - Section 3.1 (edge sparsification): keep every edge independently with
 *     probability p; a triangle survives with probability p^3, so the number
 *     of surviving triangles divided by p^3 estimates t.
 *   - Section 3.2 (degree partition): a vertex is of low degree when
 *     deg <= m^(1/2) and of high degree when deg > m^(1/2).  Triangles with
 *     at least one low-degree vertex form the light class, triangles whose
 *     three vertices all have high degree form the heavy class.
 *
 * Readings where the paper leaves a choice open:
 *   - The random draw of Section 3.1 is a counter-based hash: edge (u, v),
 *     u < v, with key (u << 32 | v) is kept iff
 *       (splitmix64(key ^ splitmix64(seed)) >> 11) < floor(p * 2^53).
 *     splitmix64 is Steele, Lea and Flood's generator as published by Vigna:
 *     mix(z + 0x9e3779b97f4a7c15) with the two multiply-xorshift rounds below.
 *   - The degree partition of Section 3.2 is taken on the sampled graph
 *     (its degrees and its edge count m_p) and evaluated exactly in integers
 *     as heavy <=> deg^2 > m_p.
 *   - Each class is rescaled by 1/p^3: est = T_L/p^3 + T_H/p^3 (Section 3.1).
 *
 * The counting is the plain definition: for every sampled edge (u, v) with
 * u < v, every common neighbour w > v closes the triangle {u, v, w}; each
 * triangle is therefore seen exactly once, at its two smallest ids, and is
 * put into the heavy class iff all three vertices are heavy.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------ splitmix64 */

uint64_t oracle_splitmix64(uint64_t x)
{
    uint64_t z = x + 0x9e3779b97f4a7c15ULL;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

/* floor(p * 2^53); p * 2^53 is exact in double, the cast truncates. */
uint64_t oracle_threshold(double p)
{
    return (uint64_t)(p * 9007199254740992.0);
}

/* Section 3.1: the keep decision for the canonical edge (u, v), u < v. */
int oracle_keep(uint32_t u, uint32_t v, uint64_t seed, uint64_t threshold)
{
    uint64_t key = ((uint64_t)u << 32) | (uint64_t)v;
    uint64_t h = oracle_splitmix64(key ^ oracle_splitmix64(seed));
    return (h >> 11) < threshold;
}

/* ------------------------------------------------------- canonical input */

static int cmp_u64(const void *a, const void *b)
{
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * Section 4.1: a simple undirected graph.  Maps every pair to (min, max),
 * drops self-loops, sorts and removes repeats.  out_pairs holds up to m_in
 * pairs.  Returns the number of distinct edges, or -1 if an endpoint is >= n,
 * or -2 if memory runs out.
 */
int64_t oracle_canonicalize(const uint32_t *pairs, uint64_t m_in, uint32_t n, uint32_t *out_pairs)
{
    uint64_t *keys = (uint64_t *)malloc((m_in ? m_in : 1) * sizeof(uint64_t));
    if (!keys) return -2;
    uint64_t k = 0;
    for (uint64_t i = 0; i < m_in; ++i) {
        uint32_t a = pairs[2 * i], b = pairs[2 * i + 1];
        if (a >= n || b >= n) { free(keys); return -1; }
        if (a == b) continue;
        uint32_t u = a < b ? a : b, v = a < b ? b : a;
        keys[k++] = ((uint64_t)u << 32) | v;
    }
    qsort(keys, k, sizeof(uint64_t), cmp_u64);
    uint64_t m = 0;
    for (uint64_t i = 0; i < k; ++i) {
        if (i > 0 && keys[i] == keys[i - 1]) continue;
        out_pairs[2 * m] = (uint32_t)(keys[i] >> 32);
        out_pairs[2 * m + 1] = (uint32_t)(keys[i] & 0xffffffffULL);
        ++m;
    }
    free(keys);
    return (int64_t)m;
}

/* ------------------------------------------------------- sparsification */

/*
 * Section 3.1: keep each canonical edge independently with probability p.
 * Kept edges are written in input order.  Returns m_p.
 */
uint64_t oracle_sample(const uint32_t *pairs, uint64_t m, double p, uint64_t seed, uint32_t *kept)
{
    uint64_t thr = oracle_threshold(p);
    uint64_t mp = 0;
    for (uint64_t i = 0; i < m; ++i) {
        if (oracle_keep(pairs[2 * i], pairs[2 * i + 1], seed, thr)) {
            kept[2 * mp] = pairs[2 * i];
            kept[2 * mp + 1] = pairs[2 * i + 1];
            ++mp;
        }
    }
    return mp;
}

/* ------------------------------------------------------- degree partition */

void oracle_degrees(const uint32_t *pairs, uint64_t m, uint32_t n, uint32_t *deg)
{
    memset(deg, 0, (size_t)n * sizeof(uint32_t));
    for (uint64_t i = 0; i < m; ++i) {
        deg[pairs[2 * i]]++;
        deg[pairs[2 * i + 1]]++;
    }
}

/* Section 3.2: heavy iff deg > m^(1/2), i.e. deg^2 > m.  Returns the number
   of heavy vertices. */
uint32_t oracle_partition(const uint32_t *deg, uint32_t n, uint64_t m, uint8_t *heavy)
{
    uint32_t h = 0;
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t d = deg[u];
        heavy[u] = d * d > m;
        h += heavy[u];
    }
    return h;
}

/* ------------------------------------------------------- triangle classes */

static int cmp_u32(const void *a, const void *b)
{
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/*
 * The full symmetric adjacency N(u) of a simple graph as sorted lists:
 * N(u) = adj[start[u] .. start[u+1]).  start holds n+1 entries, adj 2*m.
 * Built by a counting sort on the first endpoint, each list then sorted.
 * Returns 0, or -2 if memory runs out.
 */
int oracle_adjacency(const uint32_t *pairs, uint64_t m, uint32_t n, uint64_t *start, uint32_t *adj)
{
    memset(start, 0, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < m; ++i) {
        start[pairs[2 * i] + 1]++;
        start[pairs[2 * i + 1] + 1]++;
    }
    for (uint32_t u = 0; u < n; ++u) start[u + 1] += start[u];
    uint64_t *fill = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!fill) return -2;
    memcpy(fill, start, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t a = pairs[2 * i], b = pairs[2 * i + 1];
        adj[fill[a]++] = b;
        adj[fill[b]++] = a;
    }
    free(fill);
    for (uint32_t u = 0; u < n; ++u)
        qsort(adj + start[u], start[u + 1] - start[u], sizeof(uint32_t), cmp_u32);
    return 0;
}

/*
 * Triangle enumeration over the sorted lists, for the triangles whose
 * smallest vertex u lies in [u_lo, u_hi).  For each edge (u, v), u < v, the
 * common neighbours w > v are found by merging N(u) and N(v).  A triangle
 * goes to *t_heavy iff heavy[u], heavy[v] and heavy[w] are all set,
 * otherwise to *t_light (Section 3.2).  Every triangle is seen once, at its
 * smallest vertex, so the counts of disjoint ranges add up.
 */
void oracle_count_range(const uint64_t *start, const uint32_t *adj, const uint8_t *heavy,
                        uint32_t u_lo, uint32_t u_hi, uint64_t *t_light, uint64_t *t_heavy)
{
    uint64_t tl = 0, th = 0;
    for (uint32_t u = u_lo; u < u_hi; ++u) {
        for (uint64_t a = start[u]; a < start[u + 1]; ++a) {
            uint32_t v = adj[a];
            if (v <= u) continue;
            /* merge the parts of N(u) and N(v) above v */
            uint64_t i = a + 1, iend = start[u + 1];
            uint64_t j = start[v], jend = start[v + 1];
            while (j < jend && adj[j] <= v) ++j;
            while (i < iend && j < jend) {
                if (adj[i] < adj[j]) {
                    ++i;
                } else if (adj[i] > adj[j]) {
                    ++j;
                } else {
                    uint32_t w = adj[i];
                    if (heavy[u] && heavy[v] && heavy[w]) ++th; else ++tl;
                    ++i;
                    ++j;
                }
            }
        }
    }
    *t_light = tl;
    *t_heavy = th;
}

/*
 * Both classes of the whole graph: the adjacency, then the enumeration over
 * every vertex.  Returns 0, or -2 if memory runs out.
 */
int oracle_count_classes(const uint32_t *pairs, uint64_t m, uint32_t n, const uint8_t *heavy,
                         uint64_t *t_light, uint64_t *t_heavy)
{
    uint64_t *start = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t *adj = (uint32_t *)malloc((m ? 2 * m : 1) * sizeof(uint32_t));
    if (!start || !adj) { free(start); free(adj); return -2; }
    int rc = oracle_adjacency(pairs, m, n, start, adj);
    if (rc == 0) oracle_count_range(start, adj, heavy, 0, n, t_light, t_heavy);
    free(start);
    free(adj);
    return rc;
}

/* ------------------------------------------------------- whole method */

typedef struct {
    uint64_t m;         /* canonical edges */
    uint64_t m_sampled; /* kept edges, m_p */
    uint32_t n;
    uint32_t n_heavy;   /* vertices with deg_p^2 > m_p */
    uint64_t t_light;   /* sampled triangles with >= 1 light vertex */
    uint64_t t_heavy;   /* sampled triangles with 3 heavy vertices */
    double estimate;    /* T_L / p^3 + T_H / p^3 */
} oracle_result;

/* Section 3.1: the rescaled estimate of the triangle count. */
double oracle_estimate(uint64_t t_light, uint64_t t_heavy, double p)
{
    double p3 = p * p * p;
    return (double)t_light / p3 + (double)t_heavy / p3;
}

/*
 * Sections 3.1 and 3.2 end to end on a canonical edge list: sample, take
 * degrees and the partition on the sampled graph, count both classes and
 * rescale.  kept (2*m uint32) and heavy (n bytes) receive the sampled edges
 * and the heavy flags when non-NULL.  Returns 0, -1 on a bad p, -2 when
 * memory runs out.
 */
int oracle_run_partition(const uint32_t *pairs, uint64_t m, uint32_t n, double p, uint64_t seed,
                         int partition_original, uint32_t *kept_out, uint8_t *heavy_out, oracle_result *res);

int oracle_run(const uint32_t *pairs, uint64_t m, uint32_t n, double p, uint64_t seed,
               uint32_t *kept_out, uint8_t *heavy_out, oracle_result *res)
{
    return oracle_run_partition(pairs, m, n, p, seed, 0, kept_out, heavy_out, res);
}

/*
 * The same with the choice of graph for the degree partition of Section 3.2:
 * partition_original = 0 splits the sampled graph (deg_p^2 > m_p, the
 * default reading), 1 splits the original graph (deg^2 > m over the whole
 * canonical edge list) and classifies the sampled triangles by those flags.
 */
int oracle_run_partition(const uint32_t *pairs, uint64_t m, uint32_t n, double p, uint64_t seed,
                         int partition_original, uint32_t *kept_out, uint8_t *heavy_out, oracle_result *res)
{
    if (!(p > 0.0 && p <= 1.0)) return -1;
    uint32_t *kept = kept_out ? kept_out : (uint32_t *)malloc((m ? 2 * m : 1) * sizeof(uint32_t));
    uint32_t *deg = (uint32_t *)malloc(((size_t)n ? n : 1) * sizeof(uint32_t));
    uint8_t *heavy = heavy_out ? heavy_out : (uint8_t *)malloc((size_t)n ? n : 1);
    int rc = 0;
    if (!kept || !deg || !heavy) { rc = -2; goto done; }
    res->m = m;
    res->n = n;
    res->m_sampled = oracle_sample(pairs, m, p, seed, kept);
    if (partition_original) {
        oracle_degrees(pairs, m, n, deg);
        res->n_heavy = oracle_partition(deg, n, m, heavy);
    } else {
        oracle_degrees(kept, res->m_sampled, n, deg);
        res->n_heavy = oracle_partition(deg, n, res->m_sampled, heavy);
    }
    rc = oracle_count_classes(kept, res->m_sampled, n, heavy, &res->t_light, &res->t_heavy);
    res->estimate = oracle_estimate(res->t_light, res->t_heavy, p);
done:
    if (!kept_out) free(kept);
    if (!heavy_out) free(heavy);
    free(deg);
    return rc;
}

/* ------------------------------------------------------- choice of p */

/*
 * Section 3.3: the sparsification rate that balances the O(mp) pass over
 * the kept edges against the O((mp)^(3/2) log n / (eps^2 t p^3)) triple
 * samples, p = (m^(1/2) ln n / (t eps^2))^(2/5), clamped to at most 1.
 * t is a pilot estimate of the triangle count.  Returns 1 when t <= 0 (no
 * triangle seen: do not sparsify), -1 for eps <= 0, m == 0 or n < 2.
 */
double oracle_suggest_p(uint64_t m, uint32_t n, double t, double eps)
{
    if (!(eps > 0.0) || m == 0 || n < 2) return -1.0;
    if (!(t > 0.0)) return 1.0;
    double x = sqrt((double)m) * log((double)n) / (t * eps * eps);
    double p = pow(x, 0.4);
    return p < 1.0 ? p : 1.0;
}

/* ------------------------------------------------------- triple sampling */

/* floor(a * b / 2^64): a 64-bit hash a mapped to a uniform index in [0, b). */
static uint64_t mulhi64(uint64_t a, uint64_t b)
{
    return (uint64_t)(((unsigned __int128)a * (unsigned __int128)b) >> 64);
}

/* Is w in the sorted list a[0 .. len)? */
static int sorted_contains(const uint32_t *a, uint64_t len, uint32_t w)
{
    uint64_t lo = 0, hi = len;
    while (lo < hi) {
        uint64_t mid = (lo + hi) / 2;
        if (a[mid] < w) lo = mid + 1; else hi = mid;
    }
    return lo < len && a[lo] == w;
}

/*
 * The class of every vertex (path[u] = 1: heavy in the hybrid mode, its
 * triples are 2-paths) and the prefix counts of U: pre[u] = triples of the
 * vertices before u (n + 1 entries), qpre (aligned with adj) for heavy
 * rows.  Returns the number of heavy vertices.
 */
static uint32_t triple_universe(const uint64_t *start, const uint32_t *adj, uint32_t n, uint64_t mp, int hybrid,
                                uint64_t *pre, uint64_t *qpre, uint8_t *path)
{
    uint32_t h = 0;
    pre[0] = 0;
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t d = start[u + 1] - start[u], cnt;
        path[u] = hybrid && d * d > mp;
        h += path[u];
        if (path[u]) {
            cnt = 0;
            for (uint64_t j = start[u]; j < start[u + 1]; ++j) {
                uint32_t v = adj[j];
                qpre[j] = cnt;  /* 2-paths through the earlier neighbours of u */
                cnt += start[v + 1] - start[v];
            }
        } else {
            cnt = d * (d - (d > 0)) / 2;
        }
        pre[u + 1] = pre[u] + cnt;
    }
    return h;
}

/*
 * Triple r of U (0 <= r < |U|, see oracle_triples): its vertex u, its pair
 * (v, w) (a wedge v-u-w, or the 2-path u - v - w at a heavy u), and whether
 * it is a triangle.  pre[u] = triples of the vertices before u; qpre[j] for
 * a heavy u's list position j = 2-paths through the earlier neighbours.
 */
static int triple_at(const uint64_t *start, const uint32_t *adj, const uint64_t *pre, const uint64_t *qpre,
                     const uint8_t *path, uint32_t n, uint64_t r, uint32_t *pu, uint32_t *pv, uint32_t *pw)
{
    /* the vertex u with pre[u] <= r < pre[u + 1] */
    uint32_t lo = 0, hi = n;
    while (hi - lo > 1) {
        uint32_t mid = lo + (hi - lo) / 2;
        if (pre[mid] <= r) lo = mid; else hi = mid;
    }
    uint32_t u = lo;
    uint64_t k = r - pre[u];
    const uint32_t *nu = adj + start[u];
    uint64_t du = start[u + 1] - start[u];
    *pu = u;
    if (!path[u]) {
        /* wedge k: b = the largest b >= 1 with b (b - 1) / 2 <= k */
        uint64_t b = 1, bhi = du;
        while (bhi - b > 1) {
            uint64_t mid = b + (bhi - b) / 2;
            if (mid * (mid - 1) / 2 <= k) b = mid; else bhi = mid;
        }
        uint64_t a = k - b * (b - 1) / 2;
        *pv = nu[a];
        *pw = nu[b];
        return sorted_contains(adj + start[*pv], start[*pv + 1] - start[*pv], *pw);
    }
    /* 2-path k: j = the last neighbour position with qpre <= k */
    uint64_t j = 0, jhi = du;
    while (jhi - j > 1) {
        uint64_t mid = j + (jhi - j) / 2;
        if (qpre[start[u] + mid] <= k) j = mid; else jhi = mid;
    }
    uint32_t v = nu[j];
    uint32_t w = adj[start[v] + (k - qpre[start[u] + j])];
    *pv = v;
    *pw = w;
    return w != u && sorted_contains(nu, du, w);
}

typedef struct {
    uint64_t m, m_sampled;
    uint32_t n, n_heavy;   /* n_heavy: vertices whose triples are 2-paths (0 in the simple mode) */
    uint64_t universe;     /* |U| */
    uint64_t samples;      /* s */
    uint64_t closed_wedge; /* sampled wedges that are triangles */
    uint64_t closed_path;  /* sampled 2-paths that are triangles */
    double estimate;
} oracle_triple_result;

/*
 * Triple sampling (Section 3.2), after the edge sparsification of Section
 * 3.1 when p < 1 (the hybrid of Section 3.3).
 *
 * U is a set of vertex triples that holds every triangle of the (sampled)
 * graph, built vertex by vertex:
 *   - a light vertex u (every vertex in the simple mode) contributes its
 *     wedges: the C(d, 2) unordered pairs {N(u)[a], N(u)[b]}, a < b, of its
 *     neighbours (at most deg(u)^2 of them);
 *   - in the hybrid mode a heavy vertex u (deg^2 > m, Section 3.2 on the
 *     sampled graph) contributes the triples of u with the edges at its
 *     neighbours, sum over v in N(u) of deg(v) of them: the 2-paths
 *     u - v - w, w in N(v) (w = u included; it never closes).
 * Vertices are taken in id order and neighbour lists are sorted by id; a
 * vertex's wedges are numbered in the order b = 1, 2, ..., a = 0 .. b - 1
 * (index b (b - 1) / 2 + a), its 2-paths by v's position in N(u) and then
 * w's position in N(v).  A wedge {v, w} at u is a triangle iff vw is an
 * edge, a 2-path u - v - w iff w != u and uw is an edge.  Every triangle
 * is in U once per light corner (one wedge) and twice per heavy corner (two
 * 2-paths), so with weight 1 per closed wedge and 1/2 per closed 2-path the
 * weights of U sum to 3 t.
 *
 * Sample i (0 <= i < s) is the triple of index floor(h_i |U| / 2^64),
 * h_i = splitmix64(i ^ splitmix64(~seed)): s independent uniform draws
 * from U.  The estimate is |U| (2 c_w + c_p) / (6 s), which has expected
 * value t (c_w, c_p: closed wedges and 2-paths among the samples),
 * divided by p^3 for the sparsified graph.  s = 0 draws m_p samples (the
 * paper sizes the number of queries like the graph).
 *
 * pairs: the canonical edge list (m pairs); the sample of Section 3.1 with
 * (p, seed) is drawn from it first, and the same seed drives the triples.
 * hybrid: 0 for the simple mode, 1 for the hybrid mode.  Returns 0, -1 on a
 * bad p, -2 when memory runs out.
 */
int oracle_triples(const uint32_t *pairs, uint64_t m, uint32_t n, double p, uint64_t seed, uint64_t samples,
                   int hybrid, oracle_triple_result *res)
{
    if (!(p > 0.0 && p <= 1.0)) return -1;
    uint32_t *kept = (uint32_t *)malloc((m ? 2 * m : 1) * sizeof(uint32_t));
    uint64_t *start = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t *adj = (uint32_t *)malloc((m ? 2 * m : 1) * sizeof(uint32_t));
    uint64_t *pre = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint64_t *qpre = (uint64_t *)malloc((m ? 2 * m : 1) * sizeof(uint64_t));
    uint8_t *path = (uint8_t *)malloc((size_t)n ? n : 1);
    int rc = 0;
    if (!kept || !start || !adj || !pre || !qpre || !path) { rc = -2; goto done; }
    memset(res, 0, sizeof(*res));
    res->m = m;
    res->n = n;
    res->m_sampled = oracle_sample(pairs, m, p, seed, kept);
    uint64_t mp = res->m_sampled;
    if (oracle_adjacency(kept, mp, n, start, adj)) { rc = -2; goto done; }

    res->n_heavy = triple_universe(start, adj, n, mp, hybrid, pre, qpre, path);
    res->universe = pre[n];
    res->samples = samples ? samples : mp;
    uint64_t s = res->samples;
    if (res->universe == 0 || s == 0) goto rescale;

    uint64_t tmix = oracle_splitmix64(~seed);
    for (uint64_t i = 0; i < s; ++i) {
        uint64_t r = mulhi64(oracle_splitmix64(i ^ tmix), res->universe);
        uint32_t u, v, w;
        int closed = triple_at(start, adj, pre, qpre, path, n, r, &u, &v, &w);
        if (closed && path[u]) res->closed_path++;
        else if (closed) res->closed_wedge++;
    }
rescale:
    if (res->universe && s) {
        double raw = ((double)res->universe * (double)(2 * res->closed_wedge + res->closed_path)) / (6.0 * (double)s);
        double p3 = p * p * p;
        res->estimate = raw / p3;
    }
done:
    free(kept);
    free(start);
    free(adj);
    free(pre);
    free(qpre);
    free(path);
    return rc;
}

/*
 * Every triple of U in index order, for tests on small graphs (no edge
 * sampling: pairs is the whole canonical graph).  out_u / out_v / out_w /
 * out_closed hold |U| entries (ask with cap = 0 first: returns |U|).
 * Returns |U|, or -2 when memory runs out, -3 when cap < |U|.
 */
int64_t oracle_triple_enumerate(const uint32_t *pairs, uint64_t m, uint32_t n, int hybrid, uint64_t cap,
                                uint32_t *out_u, uint32_t *out_v, uint32_t *out_w, uint8_t *out_closed)
{
    uint64_t *start = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t *adj = (uint32_t *)malloc((m ? 2 * m : 1) * sizeof(uint32_t));
    uint64_t *pre = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint64_t *qpre = (uint64_t *)malloc((m ? 2 * m : 1) * sizeof(uint64_t));
    uint8_t *path = (uint8_t *)malloc((size_t)n ? n : 1);
    int64_t rc = 0;
    if (!start || !adj || !pre || !qpre || !path || oracle_adjacency(pairs, m, n, start, adj)) { rc = -2; goto done; }
    triple_universe(start, adj, n, m, hybrid, pre, qpre, path);
    rc = (int64_t)pre[n];
    if (cap == 0) goto done;
    if (cap < pre[n]) { rc = -3; goto done; }
    for (uint64_t r = 0; r < pre[n]; ++r)
        out_closed[r] = (uint8_t)triple_at(start, adj, pre, qpre, path, n, r, out_u + r, out_v + r, out_w + r);
done:
    free(start);
    free(adj);
    free(pre);
    free(qpre);
    free(path);
    return rc;
}

/* ------------------------------------------------------- semi-streaming */

typedef struct {
    uint64_t m;
    uint32_t n;
    uint32_t n_heavy;      /* candidates with deg^2 > m */
    uint64_t candidates;   /* distinct endpoints of the sampled entries */
    uint64_t sampled_entries;
    uint64_t universe;     /* |U| */
    uint64_t samples;      /* s */
    uint64_t closed_wedge; /* sampled wedges that are triangles */
    uint64_t closed_pair;  /* sampled (edge, heavy vertex) pairs that are triangles */
    double estimate;
} oracle_stream_result;

static int cmp_u64_key(const void *a, const void *b) { return cmp_u64(a, b); }

/*
 * Section 5.2: triangle counting over an adjacency-list stream in three
 * passes (the edges of each vertex given together, in order).  The stream
 * is the symmetric adjacency of a simple graph: off[n + 1], adj[2 m], every
 * list sorted by id.
 *   Pass 1 (heavy vertices): stream entry j (0 <= j < 2 m) is sampled iff
 *     (splitmix64(j ^ splitmix64(seed + 1)) >> 11) < floor(q 2^53),
 *     q = min(1, c m^(1/2) ln n / (2 m)), about c m^(1/2) ln n entries; both
 *     endpoints of a sampled entry are candidates, and the candidates with
 *     deg^2 > m form H (a vertex of degree > m^(1/2) has 2 deg of the 2 m
 *     entries, so it is missed with probability about n^-c).
 *   U: the wedges of the vertices outside H (C(d, 2) each, in vertex order,
 *     wedge b (b - 1) / 2 + a of N(u)), then the pairs (edge e, H[i]) of
 *     every edge (the entries u < v in stream order) and every vertex of H,
 *     index |U_L| + e |H| + i.  A wedge closes iff its third edge exists, a
 *     pair iff H[i] is neither endpoint and joins both.  Every triangle is
 *     in U once per corner: three times.
 *   Pass 2 (queries): sample i (0 <= i < s) is U's triple of index
 *     floor(h_i |U| / 2^64), h_i = splitmix64(i ^ splitmix64(~seed)); its
 *     list entries are read from the stream and its third edges become
 *     queries.
 *   Pass 3 (checks): the queries are sorted and merged against the stream's
 *     edges in one pass (the offline check of Section 4.2).
 * estimate = |U| (c_w + c_p) / (3 s), c_w and c_p the closed wedges and
 * pairs among the samples.  s = 0 draws m samples.  Returns 0, -2 when
 * memory runs out.
 */
int oracle_stream_triples(const uint64_t *off, const uint32_t *adj, uint32_t n, uint64_t seed, uint64_t samples,
                          double c, oracle_stream_result *res)
{
    memset(res, 0, sizeof(*res));
    const uint64_t len = off[n], m = len / 2;
    res->m = m;
    res->n = n;
    uint8_t *cand = (uint8_t *)calloc((size_t)n ? n : 1, 1);
    uint32_t *hlist = (uint32_t *)malloc(((size_t)n ? n : 1) * sizeof(uint32_t));
    uint64_t *wpre = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint64_t *uppre = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    int rc = 0;
    uint64_t *qs = NULL;
    uint8_t *found = NULL;
    uint32_t *sv = NULL, *sw = NULL, *sh = NULL;
    uint8_t *stype = NULL;
    if (!cand || !hlist || !wpre || !uppre) { rc = -2; goto done; }

    /* pass 1: candidates from the sampled entries, H = those of degree^2 > m */
    double q = 0.0;
    if (m > 0 && n > 1) {
        q = c * sqrt((double)m) * log((double)n) / (2.0 * (double)m);
        if (q > 1.0) q = 1.0;
    }
    uint64_t thr = (uint64_t)(q * 9007199254740992.0);
    uint64_t hmix = oracle_splitmix64(seed + 1);
    for (uint32_t u = 0; u < n; ++u) {
        for (uint64_t j = off[u]; j < off[u + 1]; ++j) {
            if ((oracle_splitmix64(j ^ hmix) >> 11) < thr) {
                res->sampled_entries++;
                cand[u] = 1;
                cand[adj[j]] = 1;
            }
        }
    }
    uint32_t h = 0;
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t d = off[u + 1] - off[u];
        res->candidates += cand[u];
        if (cand[u] && d * d > m) hlist[h++] = u;
    }
    res->n_heavy = h;

    /* U: wedge counts of the vertices outside H, edges (u < v entries) */
    uint32_t hi = 0;
    wpre[0] = uppre[0] = 0;
    for (uint32_t u = 0; u < n; ++u) {
        uint64_t d = off[u + 1] - off[u], up = 0;
        int heavy = hi < h && hlist[hi] == u;
        hi += heavy;
        for (uint64_t j = off[u]; j < off[u + 1]; ++j) up += adj[j] > u;
        wpre[u + 1] = wpre[u] + (heavy ? 0 : d * (d - (d > 0)) / 2);
        uppre[u + 1] = uppre[u] + up;
    }
    uint64_t UL = wpre[n];
    res->universe = UL + uppre[n] * h;
    res->samples = samples ? samples : m;
    uint64_t s = res->samples;
    if (res->universe == 0 || s == 0) goto rescale;

    /* pass 2: the samples' list entries, and their third edges as queries */
    stype = (uint8_t *)malloc(s);
    sv = (uint32_t *)malloc(s * sizeof(uint32_t));
    sw = (uint32_t *)malloc(s * sizeof(uint32_t));
    sh = (uint32_t *)malloc(s * sizeof(uint32_t));
    qs = (uint64_t *)malloc(2 * s * sizeof(uint64_t));
    if (!stype || !sv || !sw || !sh || !qs) { rc = -2; goto done; }
    uint64_t tmix = oracle_splitmix64(~seed), nq = 0;
    for (uint64_t i = 0; i < s; ++i) {
        uint64_t r = mulhi64(oracle_splitmix64(i ^ tmix), res->universe);
        if (r < UL) {
            uint32_t lo = 0, hi2 = n;  /* wpre[u] <= r < wpre[u + 1] */
            while (hi2 - lo > 1) {
                uint32_t mid = lo + (hi2 - lo) / 2;
                if (wpre[mid] <= r) lo = mid; else hi2 = mid;
            }
            uint32_t u = lo;
            uint64_t k = r - wpre[u], d = off[u + 1] - off[u];
            uint64_t b = 1, bhi = d;
            while (bhi - b > 1) {
                uint64_t mid = b + (bhi - b) / 2;
                if (mid * (mid - 1) / 2 <= k) b = mid; else bhi = mid;
            }
            uint64_t a = k - b * (b - 1) / 2;
            uint32_t v = adj[off[u] + a], w = adj[off[u] + b];
            stype[i] = 0;
            sv[i] = v;
            sw[i] = w;
            qs[nq++] = ((uint64_t)(v < w ? v : w) << 32) | (v < w ? w : v);
        } else {
            uint64_t k = r - UL, e = k / h;
            uint32_t hv = hlist[k % h];
            uint32_t lo = 0, hi2 = n;  /* uppre[x] <= e < uppre[x + 1] */
            while (hi2 - lo > 1) {
                uint32_t mid = lo + (hi2 - lo) / 2;
                if (uppre[mid] <= e) lo = mid; else hi2 = mid;
            }
            uint32_t x = lo;
            uint64_t kk = e - uppre[x];
            uint64_t d = off[x + 1] - off[x], up = uppre[x + 1] - uppre[x];
            uint32_t y = adj[off[x] + (d - up) + kk];  /* the entries above x are the list's tail */
            stype[i] = 1;
            sv[i] = x;
            sw[i] = y;
            sh[i] = hv;
            if (hv != x && hv != y) {
                qs[nq++] = ((uint64_t)(hv < x ? hv : x) << 32) | (hv < x ? x : hv);
                qs[nq++] = ((uint64_t)(hv < y ? hv : y) << 32) | (hv < y ? y : hv);
            }
        }
    }

    /* pass 3: sort the distinct queries, one merge pass over the edges */
    qsort(qs, nq, sizeof(uint64_t), cmp_u64_key);
    uint64_t nd = 0;
    for (uint64_t i = 0; i < nq; ++i)
        if (i == 0 || qs[i] != qs[i - 1]) qs[nd++] = qs[i];
    found = (uint8_t *)calloc(nd ? nd : 1, 1);
    if (!found) { rc = -2; goto done; }
    uint64_t qi = 0;
    for (uint32_t u = 0; u < n && qi < nd; ++u) {
        for (uint64_t j = off[u]; j < off[u + 1] && qi < nd; ++j) {
            if (adj[j] <= u) continue;
            uint64_t key = ((uint64_t)u << 32) | adj[j];
            while (qi < nd && qs[qi] < key) ++qi;
            if (qi < nd && qs[qi] == key) found[qi] = 1;
        }
    }
    for (uint64_t i = 0; i < s; ++i) {
        if (stype[i] == 0) {
            uint32_t v = sv[i], w = sw[i];
            uint64_t key = ((uint64_t)(v < w ? v : w) << 32) | (v < w ? w : v);
            uint64_t *p = (uint64_t *)bsearch(&key, qs, nd, sizeof(uint64_t), cmp_u64_key);
            res->closed_wedge += found[p - qs];
        } else {
            uint32_t x = sv[i], y = sw[i], hv = sh[i];
            if (hv == x || hv == y) continue;
            uint64_t k1 = ((uint64_t)(hv < x ? hv : x) << 32) | (hv < x ? x : hv);
            uint64_t k2 = ((uint64_t)(hv < y ? hv : y) << 32) | (hv < y ? y : hv);
            uint64_t *p1 = (uint64_t *)bsearch(&k1, qs, nd, sizeof(uint64_t), cmp_u64_key);
            uint64_t *p2 = (uint64_t *)bsearch(&k2, qs, nd, sizeof(uint64_t), cmp_u64_key);
            res->closed_pair += found[p1 - qs] && found[p2 - qs];
        }
    }
rescale:
    if (res->universe && s)
        res->estimate = ((double)res->universe * (double)(res->closed_wedge + res->closed_pair)) / (3.0 * (double)s);
done:
    free(cand);
    free(hlist);
    free(wpre);
    free(uppre);
    free(qs);
    free(found);
    free(sv);
    free(sw);
    free(sh);
    free(stype);
    return rc;
}
