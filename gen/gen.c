/*
 * Seeded synthetic graph generators (input data only).
 *
 * These produce the simple undirected graphs that stand in for the paper's
 * real networks (Table 1 of the paper: social and web graphs with 1-10 M
 * vertices and 3-117 M edges), which are not available here.  Every
 * generator is a pure function of its arguments: randomness comes from a
 * counter-based stream (MurmurHash3's 64-bit finaliser applied to a
 * seed/stream/counter triple), so the output does not depend on threads or
 * call order.
 *
 * This module contains none of the triangle-counting method: no edge
 * sampling, no degree partition, no counting.  Its outputs feed both the
 * CPU oracle and the CUDA library.  Every generator returns a canonical
 * edge list: pairs (u, v) with u < v, sorted by (u, v), without duplicates
 * or self-loops, packed as uint32 pairs {u, v}.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ---------------------------------------------------------------- random */

static inline uint64_t g_fmix64(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdULL;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ULL;
    k ^= k >> 33;
    return k;
}

/* 64 random bits for (seed, stream, counter). */
static inline uint64_t g_rand(uint64_t seed, uint64_t stream, uint64_t ctr)
{
    uint64_t s = g_fmix64(seed * 0xd1b54a32d192ed03ULL + stream * 0x8cb92ba72f3d8dd7ULL + 1);
    return g_fmix64(s ^ (ctr * 0x9fb21c651e98df25ULL + 0x632be59bd9b4e019ULL));
}

/* ------------------------------------------------ portable log / exp / pow
   Built from IEEE basic operations only (compiled without FMA contraction),
   so every platform produces bit-identical graphs; libm's pow may differ in
   the last ulp between C libraries. */

/* natural log: x = f 2^e with f in [sqrt(1/2), sqrt(2)), then
   log f = 2 atanh(s), s = (f - 1)/(f + 1), by its odd power series */
static double g_log(double x)
{
    int e;
    double f = frexp(x, &e); /* exact: f in [0.5, 1) */
    if (f < 0.70710678118654752440) { f *= 2.0; e -= 1; }
    const double s = (f - 1.0) / (f + 1.0), s2 = s * s;
    double term = s, sum = 0.0;
    for (int k = 1; k <= 41; k += 2) { sum += term / k; term *= s2; }
    return 2.0 * sum + e * 0.69314718055994530942;
}

/* exp: y = k ln2 + r, |r| <= ln2 / 2, exp(r) by its Taylor series */
static double g_exp(double y)
{
    const double k = floor(y / 0.69314718055994530942 + 0.5);
    const double r = y - k * 0.69314718055994530942;
    double term = 1.0, sum = 1.0;
    for (int i = 1; i <= 24; ++i) { term = term * r / i; sum += term; }
    return ldexp(sum, (int)k);
}

static double g_pow(double x, double y) { return g_exp(y * g_log(x)); }

/* uniform in [0, 1) with 53 random bits */
static inline double g_unit(uint64_t r) { return (double)(r >> 11) * (1.0 / 9007199254740992.0); }

/* uniform integer in [0, n) from 32 random bits (multiply-shift) */
static inline uint32_t g_below(uint32_t r32, uint32_t n) { return (uint32_t)(((uint64_t)r32 * n) >> 32); }

/* ------------------------------------------------------- sort and dedup */

/* LSD radix sort of 64-bit keys restricted to the low `bits` bits. */
static int g_radix_sort_u64(uint64_t *a, uint64_t n, int bits)
{
    if (n < 2) return 0;
    uint64_t *tmp = (uint64_t *)malloc(n * sizeof(uint64_t));
    if (!tmp) return -1;
    uint64_t *src = a, *dst = tmp;
    for (int shift = 0; shift < bits; shift += 11) {
        uint64_t cnt[2048];
        memset(cnt, 0, sizeof(cnt));
        for (uint64_t i = 0; i < n; ++i) cnt[(src[i] >> shift) & 2047]++;
        uint64_t sum = 0;
        for (int d = 0; d < 2048; ++d) { uint64_t c = cnt[d]; cnt[d] = sum; sum += c; }
        for (uint64_t i = 0; i < n; ++i) dst[cnt[(src[i] >> shift) & 2047]++] = src[i];
        uint64_t *t = src; src = dst; dst = t;
    }
    if (src != a) memcpy(a, src, n * sizeof(uint64_t));
    free(tmp);
    return 0;
}

static int g_bits_for(uint64_t n)
{
    int b = 1;
    while (b < 64 && (1ULL << b) < n) ++b;
    return b;
}

/* keys (u << 32 | v) with u < v: sort, remove duplicates, unpack to pairs */
static int64_t g_finish(uint64_t *keys, uint64_t cnt, uint32_t n, uint32_t *out_pairs, uint64_t cap)
{
    int vb = g_bits_for(n);
    /* pack as (u << vb | v) so the sort only touches 2*vb bits */
    for (uint64_t i = 0; i < cnt; ++i) {
        uint64_t u = keys[i] >> 32, v = keys[i] & 0xffffffffULL;
        keys[i] = (u << vb) | v;
    }
    if (g_radix_sort_u64(keys, cnt, 2 * vb)) return -1;
    uint64_t m = 0;
    for (uint64_t i = 0; i < cnt; ++i) {
        if (i > 0 && keys[i] == keys[i - 1]) continue;
        if (m >= cap) return -2;
        out_pairs[2 * m] = (uint32_t)(keys[i] >> vb);
        out_pairs[2 * m + 1] = (uint32_t)(keys[i] & ((1ULL << vb) - 1));
        ++m;
    }
    return (int64_t)m;
}

/* open-addressing set of nonzero 64-bit keys */
typedef struct {
    uint64_t *slot;
    uint64_t mask;
} g_set;

static int g_set_init(g_set *s, uint64_t expect)
{
    uint64_t cap = 16;
    while (cap < 2 * expect + 16) cap <<= 1;
    s->slot = (uint64_t *)calloc(cap, sizeof(uint64_t));
    s->mask = cap - 1;
    return s->slot ? 0 : -1;
}

/* returns 1 if inserted, 0 if present; key must be nonzero */
static int g_set_insert(g_set *s, uint64_t key)
{
    uint64_t i = g_fmix64(key) & s->mask;
    for (;;) {
        if (s->slot[i] == 0) { s->slot[i] = key; return 1; }
        if (s->slot[i] == key) return 0;
        i = (i + 1) & s->mask;
    }
}

/* Stored keys are (u << 32 | v) + 1 so that the edge (0, 0) never collides
   with the empty marker; self-loops are rejected before insertion anyway. */
static inline uint64_t g_key(uint32_t a, uint32_t b)
{
    uint32_t u = a < b ? a : b, v = a < b ? b : a;
    return ((uint64_t)u << 32) | v;
}

/* ------------------------------------------------------- Erdos-Renyi */

/*
 * G(n, m): draw uniform vertex pairs, reject self-loops and repeats, stop at
 * m distinct edges.  out_pairs holds 2*m uint32.  Returns m, or a negative
 * value on bad arguments / allocation failure.
 */
int64_t gen_er(uint32_t n, uint64_t m, uint64_t seed, uint32_t *out_pairs)
{
    if (n < 2) return m == 0 ? 0 : -1;
    if (m > (uint64_t)n * (n - 1) / 2) return -1;
    g_set set;
    if (g_set_init(&set, m)) return -3;
    uint64_t *keys = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    if (!keys) { free(set.slot); return -3; }
    uint64_t got = 0;
    for (uint64_t ctr = 0; got < m; ++ctr) {
        uint64_t r = g_rand(seed, 1, ctr);
        uint32_t a = g_below((uint32_t)(r >> 32), n), b = g_below((uint32_t)r, n);
        if (a == b) continue;
        uint64_t k = g_key(a, b);
        if (g_set_insert(&set, k + 1)) keys[got++] = k;
    }
    free(set.slot);
    int64_t res = g_finish(keys, got, n, out_pairs, m);
    free(keys);
    return res;
}

/* ------------------------------------------------------- Chung-Lu */

/*
 * Walker's alias table (Vose's construction) for weights w[0..n) summing to
 * total: afterwards drawing i uniformly and keeping it with probability
 * w'[i] (stored back into w) else taking alias[i] samples proportionally to
 * w.  Deterministic: only IEEE basic operations and a fixed visiting order.
 */
static int g_alias_build(double *w, uint32_t *alias, uint32_t n, double total)
{
    uint32_t *small = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *large = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!small || !large) { free(small); free(large); return -1; }
    uint32_t ns = 0, nl = 0;
    for (uint32_t i = 0; i < n; ++i) {
        w[i] = w[i] * (double)n / total;
        alias[i] = i;
        if (w[i] < 1.0) small[ns++] = i; else large[nl++] = i;
    }
    while (ns > 0 && nl > 0) {
        uint32_t s = small[--ns], l = large[nl - 1];
        alias[s] = l;
        w[l] = (w[l] + w[s]) - 1.0;
        if (w[l] < 1.0) { --nl; small[ns++] = l; }
    }
    while (nl > 0) w[large[--nl]] = 1.0;
    while (ns > 0) w[small[--ns]] = 1.0;
    free(small);
    free(large);
    return 0;
}

/* seeded Fisher-Yates permutation of [0, n) */
static void g_perm(uint32_t *perm, uint32_t n, uint64_t seed, uint64_t stream)
{
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    for (uint32_t i = n - 1; i > 0; --i) {
        uint32_t j = g_below((uint32_t)(g_rand(seed, stream, i) >> 32), i + 1);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
}

/*
 * Chung-Lu power-law graph.  Expected-degree weights follow
 * w(x) = c (x + i0)^(-1/(gamma-1)) over positions x in [0, n); i0 and c are
 * chosen so that w(0) = wmax and the weights sum to 2*m.  Endpoints are drawn
 * independently with probability proportional to w (inverse of the
 * continuous CDF), positions are mapped through a seeded vertex permutation,
 * self-loops and repeats are rejected, and drawing stops at exactly m
 * distinct edges.  Returns m, or a negative value on error.
 */
int64_t gen_chung_lu(uint32_t n, uint64_t m, double gamma, double wmax, uint64_t seed,
                     uint32_t *out_pairs)
{
    if (n < 2 || gamma <= 2.0 || wmax <= 1.0) return -1;
    if (m > (uint64_t)n * (n - 1) / 4) return -1; /* keep far from complete */
    const double a = 1.0 / (gamma - 1.0), e = 1.0 - a; /* 0 < e < 1 */
    /* f(i0) = 2 m e / (i0^a ((n+i0)^e - i0^e)) decreases in i0; solve f = wmax */
    double lo = 1e-9, hi = 1e12;
    for (int it = 0; it < 200; ++it) {
        double mid = sqrt(lo * hi);
        double D = g_pow((double)n + mid, e) - g_pow(mid, e);
        double f = 2.0 * (double)m * e / (g_pow(mid, a) * D);
        if (f > wmax) lo = mid; else hi = mid;
    }
    const double i0 = sqrt(lo * hi);
    /* vertex i carries the weight of [i, i+1) under w: F(i+1) - F(i) with
       F(x) = (x + i0)^e up to a constant factor */
    double *prob = (double *)malloc((size_t)n * sizeof(double));
    uint32_t *alias = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint32_t *perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    g_set set;
    uint64_t *keys = (uint64_t *)malloc((m ? m : 1) * sizeof(uint64_t));
    if (!prob || !alias || !perm || !keys || g_set_init(&set, m)) {
        free(prob); free(alias); free(perm); free(keys);
        return -3;
    }
    double prev = g_pow(i0, e), total = 0.0;
    for (uint32_t i = 0; i < n; ++i) {
        double cur = g_pow((double)i + 1.0 + i0, e);
        prob[i] = cur - prev;
        total += prob[i];
        prev = cur;
    }
    if (g_alias_build(prob, alias, n, total)) { free(prob); free(alias); free(perm); free(keys); free(set.slot); return -3; }
    g_perm(perm, n, seed, 7);
    uint64_t got = 0;
    for (uint64_t ctr = 0; got < m; ++ctr) {
        uint32_t ends[2];
        for (int s = 0; s < 2; ++s) {
            uint64_t r = g_rand(seed, 2 + s, ctr);
            uint32_t i = g_below((uint32_t)(r >> 32), n);
            double u = ((double)(uint32_t)r + 0.5) * (1.0 / 4294967296.0);
            ends[s] = perm[u < prob[i] ? i : alias[i]];
        }
        if (ends[0] == ends[1]) continue;
        uint64_t k = g_key(ends[0], ends[1]);
        if (g_set_insert(&set, k + 1)) keys[got++] = k;
    }
    free(set.slot);
    free(perm);
    free(prob);
    free(alias);
    int64_t res = g_finish(keys, got, n, out_pairs, m);
    free(keys);
    return res;
}

/* ------------------------------------------------------- planted core */

/*
 * A dense core planted in a sparse graph: `core` vertices joined pairwise
 * with probability q (one counter-based draw per pair), plus m_rest uniform
 * random edges among all n vertices; vertex ids are scrambled by a seeded
 * permutation.  out_pairs must hold core*(core-1)/2 + m_rest pairs.  Returns
 * the number of distinct edges.
 */
int64_t gen_planted_core(uint32_t n, uint32_t core, double q, uint64_t m_rest, uint64_t seed, uint32_t *out_pairs)
{
    if (core > n || q < 0.0 || q > 1.0 || n < 2) return -1;
    const uint64_t cap = (uint64_t)core * (core - 1) / 2 + m_rest;
    uint64_t *keys = (uint64_t *)malloc((cap ? cap : 1) * sizeof(uint64_t));
    uint32_t *perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    if (!keys || !perm) { free(keys); free(perm); return -3; }
    g_perm(perm, n, seed, 13);
    const uint64_t thr = q >= 1.0 ? ~0ULL : (uint64_t)(q * 18446744073709551616.0);
    uint64_t cnt = 0;
    for (uint32_t i = 0; i < core; ++i)
        for (uint32_t j = i + 1; j < core; ++j)
            if (g_rand(seed, 17, (uint64_t)i * core + j) < thr || q >= 1.0) keys[cnt++] = g_key(perm[i], perm[j]);
    for (uint64_t e = 0; e < m_rest; ++e) {
        uint64_t r = g_rand(seed, 19, e);
        uint32_t a = g_below((uint32_t)(r >> 32), n), b = g_below((uint32_t)r, n);
        if (a == b) continue;
        keys[cnt++] = g_key(perm[a], perm[b]);
    }
    free(perm);
    int64_t res = g_finish(keys, cnt, n, out_pairs, cap);
    free(keys);
    return res;
}

/* ------------------------------------------------------- R-MAT */

/* quadrant thresholds on 16-bit uniforms: four levels per 64-bit draw */
typedef struct {
    uint32_t ta, tb, tc;
} g_rmat_t;

static int g_rmat_thresholds(double a, double b, double c, g_rmat_t *t)
{
    if (a < 0 || b < 0 || c < 0 || a + b + c > 1.0) return -1;
    t->ta = (uint32_t)(a * 65536.0);
    t->tb = (uint32_t)((a + b) * 65536.0);
    t->tc = (uint32_t)((a + b + c) * 65536.0);
    return 0;
}

/* Draw e: `scale` levels of the adjacency quadtree, each taking quadrant
   (0,0), (0,1), (1,0), (1,1) with probabilities a, b, c, 1-a-b-c; the
   positions before the vertex permutation. */
static inline void g_rmat_draw(uint32_t scale, const g_rmat_t *t, uint64_t seed, uint64_t e, uint32_t *pu,
                               uint32_t *pv)
{
    uint32_t u = 0, v = 0;
    uint64_t r = 0;
    for (uint32_t l = 0; l < scale; ++l) {
        if ((l & 3) == 0) r = g_rand(seed, 3 + l / 4, e);
        uint32_t x = (uint32_t)(r & 0xffff);
        r >>= 16;
        uint32_t ubit = x >= t->tb, vbit = (x >= t->ta && x < t->tb) || x >= t->tc;
        u = (u << 1) | ubit;
        v = (v << 1) | vbit;
    }
    *pu = u;
    *pv = v;
}

/* The seeded vertex permutation of an R-MAT graph (perm holds 2^scale). */
int gen_rmat_perm(uint32_t scale, uint64_t seed, uint32_t *perm)
{
    if (scale < 1 || scale > 31) return -1;
    g_perm(perm, 1u << scale, seed, 11);
    return 0;
}

/*
 * Draws [e0, e1) of the R-MAT graph as raw pairs (perm[u], perm[v]) in draw
 * order, self-loops and repeats included (out_pairs holds 2 (e1 - e0)
 * uint32).  Symmetrising, deduplicating and dropping self-loops over all
 * edge_factor 2^scale draws gives exactly gen_rmat's graph.  Disjoint ranges
 * may be filled concurrently.
 */
int gen_rmat_draws(uint32_t scale, double a, double b, double c, uint64_t seed, const uint32_t *perm,
                   uint64_t e0, uint64_t e1, uint32_t *out_pairs)
{
    g_rmat_t t;
    if (scale < 1 || scale > 31 || g_rmat_thresholds(a, b, c, &t)) return -1;
    for (uint64_t e = e0; e < e1; ++e) {
        uint32_t u, v;
        g_rmat_draw(scale, &t, seed, e, &u, &v);
        out_pairs[2 * (e - e0)] = perm[u];
        out_pairs[2 * (e - e0) + 1] = perm[v];
    }
    return 0;
}

/*
 * R-MAT graph with 2^scale vertices and edge_factor * 2^scale generated
 * edges (g_rmat_draw).  Vertex ids are then scrambled by a seeded
 * permutation (as Graph500 does), the result is symmetrised (u, v) ->
 * (min, max) and deduplicated, and self-loops are dropped.  out_pairs must
 * hold 2 * edge_factor * 2^scale uint32.  Returns the number of distinct
 * undirected edges.
 */
int64_t gen_rmat(uint32_t scale, uint32_t edge_factor, double a, double b, double c,
                 uint64_t seed, uint32_t *out_pairs)
{
    g_rmat_t t;
    if (scale < 1 || scale > 31 || g_rmat_thresholds(a, b, c, &t)) return -1;
    const uint32_t n = 1u << scale;
    const uint64_t draws = (uint64_t)edge_factor << scale;
    uint32_t *perm = (uint32_t *)malloc((size_t)n * sizeof(uint32_t));
    uint64_t *keys = (uint64_t *)malloc((draws ? draws : 1) * sizeof(uint64_t));
    if (!perm || !keys) { free(perm); free(keys); return -3; }
    g_perm(perm, n, seed, 11);
    uint64_t cnt = 0;
    for (uint64_t e = 0; e < draws; ++e) {
        uint32_t u, v;
        g_rmat_draw(scale, &t, seed, e, &u, &v);
        u = perm[u];
        v = perm[v];
        if (u == v) continue;
        keys[cnt++] = g_key(u, v);
    }
    free(perm);
    int64_t res = g_finish(keys, cnt, n, out_pairs, draws);
    free(keys);
    return res;
}
