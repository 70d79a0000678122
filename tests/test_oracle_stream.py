"""Pins for the oracle's semi-streaming triple sampler (Section 5.2): the
heavy vertices found from sampled stream entries (the lemma's guarantee
and the exact partition when every entry is sampled), the size of U and
the 3 t weight of its closed triples written out here from the definition,
exactness on graphs whose every triple closes, zero on triangle-free
graphs, and unbiasedness against the exact variance of s uniform draws."""
import math

import numpy as np
import pytest

import gen
import oracle
from test_oracle_pins import adjacency, brute_classes

ALL = 1e12  # a factor that samples every stream entry (q = 1)


def brute_stream_universe(edges, n, heavy):
    """U of Section 5.2 written out: the wedges {N[a], N[b]} (b = 1.., a < b)
    of every vertex outside `heavy` in id order, then the pairs (edge e,
    heavy vertex h) for the edges u < v in order and the heavy vertices in
    id order.  Returns a list of closed flags."""
    A = adjacency(edges, n)
    nbrs = [sorted(int(x) for x in np.nonzero(A[u])[0]) for u in range(n)]
    H = sorted(int(h) for h in np.nonzero(heavy)[0])
    out = []
    for u in range(n):
        if heavy[u]:
            continue
        d = len(nbrs[u])
        for b in range(1, d):
            for a in range(b):
                out.append(bool(A[nbrs[u][a], nbrs[u][b]]))
    for u in range(n):
        for v in nbrs[u]:
            if v <= u:
                continue
            for h in H:
                out.append(h != u and h != v and bool(A[h, u]) and bool(A[h, v]))
    return out


def small_graphs():
    yield gen.wheel(5), 6
    yield gen.complete(6), 6
    g, n = gen.disjoint_union(gen.complete(4), gen.wheel(7), gen.star(5))
    yield g, n
    yield gen.er(30, 90, 3), 30
    yield gen.chung_lu(60, 250, 2.1, 25.0, 4), 60


@pytest.mark.parametrize("edges,n", list(small_graphs()))
def test_universe_and_three_t(edges, n):
    """With every entry sampled the heavy set is the exact partition
    (deg^2 > m); |U| and the closed count of U (3 t) match the brute-force
    enumeration of the definition."""
    deg, heavy, tl, th = brute_classes(edges, n)
    off, adj = gen.adjacency_stream(edges, n)
    r = oracle.stream_triples(off, adj, n, 1, 10, c=ALL)
    assert r["n_heavy"] == int(heavy.sum())
    assert r["candidates"] == int((deg > 0).sum())
    U = brute_stream_universe(edges, n, heavy)
    assert r["universe"] == len(U)
    assert sum(U) == 3 * (tl + th)


def test_every_triple_closes_in_unions_of_small_cliques():
    """50 disjoint K_4: every vertex is light (9 <= 300) and every wedge
    closes, so every sample closes and the estimate is |U| / 3 = 200."""
    g, n = gen.disjoint_union(*[gen.complete(4)] * 50)
    off, adj = gen.adjacency_stream(g, n)
    for seed, s in ((1, 7), (2, 5000), (3, 0)):
        r = oracle.stream_triples(off, adj, n, seed, s)
        assert r["n_heavy"] == 0 and r["closed_wedge"] == r["samples"] and r["closed_pair"] == 0
        assert r["estimate"] == 200.0


@pytest.mark.parametrize("g,n", [(gen.star(20), 21), (gen.random_tree(80, 2), 80), (gen.complete_bipartite(7, 9), 16),
                                 (np.zeros((0, 2), np.uint32), 4)])
def test_triangle_free_and_empty(g, n):
    off, adj = gen.adjacency_stream(g, n)
    for c in (3.0, ALL):
        r = oracle.stream_triples(off, adj, n, 5, 300, c=c)
        assert r["closed_wedge"] == r["closed_pair"] == 0 and r["estimate"] == 0.0


def test_heavy_vertices_found_with_high_probability():
    """Section 5.2's lemma: with about c m^(1/2) ln n sampled entries every
    vertex of degree > m^(1/2) is a candidate except with probability about
    n^(1 - c); over 40 seeds (c = 3) all are found, and the sampled entries
    stay within 6 sigma of their expectation."""
    e, n = gen.chung_lu(5000, 40000, 2.1, 900.0, 6), 5000
    deg = oracle.degrees(e, n)  # the heavy vertices by Section 3.2's definition, deg^2 > m
    m = len(e)
    want = int(((deg.astype(np.int64) ** 2) > m).sum())
    off, adj = gen.adjacency_stream(e, n)
    q = min(1.0, 3.0 * math.sqrt(m) * math.log(n) / (2.0 * m))
    for seed in range(1, 41):
        r = oracle.stream_triples(off, adj, n, seed, 10)
        assert r["n_heavy"] == want > 0
        mu = q * 2 * m
        assert abs(r["sampled_entries"] - mu) <= 6 * math.sqrt(mu * (1 - q))


def test_stream_estimator_unbiased_with_exact_variance():
    """With the heavy set fixed (every entry sampled) the s draws are
    independent with P(closed) = 3 t / |U|, so the estimate |U| c / (3 s)
    has mean t and variance (|U| / 3)^2 P (1 - P) / s."""
    e, n = gen.chung_lu(80, 330, 2.1, 30.0, 7), 80
    _, heavy, tl, th = brute_classes(e, n)
    t = tl + th
    size = len(brute_stream_universe(e, n, heavy))
    pr = 3 * t / size
    s = 60
    var = (size / 3.0) ** 2 * pr * (1 - pr) / s
    off, adj = gen.adjacency_stream(e, n)
    ests = np.array([oracle.stream_triples(off, adj, n, seed, s, c=ALL)["estimate"] for seed in range(1, 201)])
    assert abs(ests.mean() - t) <= 5 * math.sqrt(var / len(ests))
    assert 0.6 * var <= ests.var(ddof=1) <= 1.6 * var


def test_stream_estimate_tracks_the_count():
    e, n = gen.chung_lu(20000, 150000, 2.1, 2500.0, 2), 20000
    t = oracle.run(e, n, 1.0, 1)["estimate"]
    off, adj = gen.adjacency_stream(e, n)
    r = oracle.stream_triples(off, adj, n, 3, 400000)
    assert abs(r["estimate"] - t) <= 0.05 * t
