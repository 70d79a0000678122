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
 * Plain triangle enumeration over sorted adjacency lists.  For each edge
 * (u, v), u < v, the common neighbours w > v are found by merging N(u) and
 * N(v).  A triangle goes to *t_heavy iff heavy[u], heavy[v] and heavy[w]
 * are all set, otherwise to *t_light (Section 3.2).  Returns 0, or -2 if
 * memory runs out.
 */
int oracle_count_classes(const uint32_t *pairs, uint64_t m, uint32_t n, const uint8_t *heavy,
                         uint64_t *t_light, uint64_t *t_heavy)
{
    uint64_t *start = (uint64_t *)calloc((size_t)n + 1, sizeof(uint64_t));
    uint64_t *fill = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    uint32_t *adj = (uint32_t *)malloc((m ? 2 * m : 1) * sizeof(uint32_t));
    if (!start || !fill || !adj) { free(start); free(fill); free(adj); return -2; }
    /* full symmetric adjacency N(u), by counting sort, each list sorted */
    for (uint64_t i = 0; i < m; ++i) {
        start[pairs[2 * i] + 1]++;
        start[pairs[2 * i + 1] + 1]++;
    }
    for (uint32_t u = 0; u < n; ++u) start[u + 1] += start[u];
    memcpy(fill, start, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < m; ++i) {
        uint32_t a = pairs[2 * i], b = pairs[2 * i + 1];
        adj[fill[a]++] = b;
        adj[fill[b]++] = a;
    }
    free(fill);
    for (uint32_t u = 0; u < n; ++u)
        qsort(adj + start[u], start[u + 1] - start[u], sizeof(uint32_t), cmp_u32);

    uint64_t tl = 0, th = 0;
    for (uint32_t u = 0; u < n; ++u) {
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
    free(start);
    free(adj);
    *t_light = tl;
    *t_heavy = th;
    return 0;
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
int oracle_run(const uint32_t *pairs, uint64_t m, uint32_t n, double p, uint64_t seed,
               uint32_t *kept_out, uint8_t *heavy_out, oracle_result *res)
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
    oracle_degrees(kept, res->m_sampled, n, deg);
    res->n_heavy = oracle_partition(deg, n, res->m_sampled, heavy);
    rc = oracle_count_classes(kept, res->m_sampled, n, heavy, &res->t_light, &res->t_heavy);
    res->estimate = oracle_estimate(res->t_light, res->t_heavy, p);
done:
    if (!kept_out) free(kept);
    if (!heavy_out) free(heavy);
    free(deg);
    return rc;
}
