"""Pins for the oracle's triple sampling (Sections 3.2-3.3), its choice of p
(Section 3.3) and its partition on the original degrees (the alternative
reading of which graph Section 3.2 splits).

Each test ties the oracle to something outside its own code: a brute-force
enumeration of the triple set U written here from the definition, the
identity that the weights of U's closed triples sum to 3 t, closed forms
(complete graphs, triangle-free graphs), the exact variance of the
with-replacement estimator, and the balance equation that defines the
suggested p.
"""
import itertools
import math

import numpy as np
import pytest

import gen
import oracle
from test_oracle_pins import adjacency, brute_classes, brute_enumerate


# ------------------------------------------------------------ brute force of U

def brute_universe(edges, n, mode):
    """U of the whole graph written out from the definition: vertices in id
    order; a light vertex (every vertex in the simple mode) lists its wedges
    {N[a], N[b]} for b = 1, 2, ... and a = 0 .. b - 1 over its sorted
    neighbour list; a heavy vertex (deg^2 > m, hybrid mode) lists the 2-paths
    u - v - w for v in N(u), w in N(v), both in sorted order.  Returns a list
    of (u, v, w, closed, weight)."""
    A = adjacency(edges, n)
    m = int(round(A.sum())) // 2
    nbrs = [sorted(int(x) for x in np.nonzero(A[u])[0]) for u in range(n)]
    out = []
    for u in range(n):
        d = len(nbrs[u])
        heavy = mode == "hybrid" and d * d > m
        if not heavy:
            for b in range(1, d):
                for a in range(b):
                    v, w = nbrs[u][a], nbrs[u][b]
                    out.append((u, v, w, bool(A[v, w]), 1.0))
        else:
            for v in nbrs[u]:
                for w in nbrs[v]:
                    out.append((u, v, w, w != u and bool(A[u, w]), 0.5))
    return out


def tiny_graphs():
    yield "wheel5", gen.wheel(5), 6
    yield "wheel4", gen.wheel(4), 5
    yield "k5", gen.complete(5), 5
    g, n = gen.disjoint_union(gen.complete(4), gen.wheel(6), gen.star(4))
    yield "union", g, n
    for s in range(3):
        g = gen.er(14, 34, 100 + s)
        yield "er%d" % s, g, 14
    g = gen.chung_lu(40, 120, 2.1, 15.0, 9)
    yield "chung_lu", g, 40


@pytest.mark.parametrize("mode", ["simple", "hybrid"])
@pytest.mark.parametrize("name,edges,n", list(tiny_graphs()))
def test_triple_index_map_matches_brute_force(name, edges, n, mode):
    """The oracle's map from an index of U to its triple visits U exactly in
    the order of the definition, and decides closure like the adjacency
    matrix does."""
    want = brute_universe(edges, n, mode)
    u, v, w, c = oracle.triple_enumerate(edges, n, mode)
    got = [(int(a), int(b), int(x), bool(y)) for a, b, x, y in zip(u, v, w, c)]
    assert got == [t[:4] for t in want]


@pytest.mark.parametrize("mode", ["simple", "hybrid"])
@pytest.mark.parametrize("name,edges,n", list(tiny_graphs()))
def test_closed_weights_sum_to_three_t(name, edges, n, mode):
    """Every triangle is in U once per light corner and twice per heavy
    corner, so the closed weights sum to 3 t (t from trace(A^3) / 6)."""
    _, _, tl, th = brute_classes(edges, n)
    t = tl + th
    U = brute_universe(edges, n, mode)
    assert sum(wt for *_, closed, wt in U if closed) == 3 * t
    res = oracle.triples(edges, n, 1.0, 1, samples=1, mode=mode)
    assert res["universe"] == len(U)


@pytest.mark.parametrize("k", [3, 4, 7, 12])
def test_simple_mode_is_exact_on_complete_graphs(k):
    """In K_k every wedge is closed, so every sample closes and the estimate
    is |U| / 3 = k C(k - 1, 2) / 3 = C(k, 3) for any seed and sample count."""
    e = gen.complete(k)
    for seed, s in ((1, 17), (99, 1000)):
        r = oracle.triples(e, k, 1.0, seed, samples=s, mode="simple")
        assert r["closed_wedge"] == s and r["closed_path"] == 0
        assert r["universe"] == k * math.comb(k - 1, 2)
        assert r["estimate"] == math.comb(k, 3)


@pytest.mark.parametrize("g,n", [(gen.star(9), 10), (gen.random_tree(60, 3), 60),
                                 (gen.complete_bipartite(5, 7), 12), (gen.cycle(8), 8)])
@pytest.mark.parametrize("mode", ["simple", "hybrid"])
def test_triangle_free_graphs_estimate_zero(g, n, mode):
    for p in (1.0, 0.6):
        r = oracle.triples(g, n, p, 3, samples=500, mode=mode)
        assert r["closed_wedge"] == 0 and r["closed_path"] == 0 and r["estimate"] == 0.0


def test_default_sample_count_is_m_p():
    e = gen.er(200, 1500, 4)
    for p in (1.0, 0.3):
        r = oracle.triples(e, 200, p, 8, samples=0, mode="hybrid")
        assert r["samples"] == r["m_sampled"] == len(oracle.sample(e, p, 8))


def test_hybrid_heavy_vertices_are_the_partition_of_the_sample():
    e = gen.chung_lu(3000, 20000, 2.1, 600.0, 5)
    for p in (1.0, 0.5):
        r = oracle.triples(e, 3000, p, 11, samples=10, mode="hybrid")
        kept = oracle.sample(e, p, 11)
        flags = oracle.partition_flags(oracle.degrees(kept, 3000), len(kept))
        assert r["n_heavy"] == int(flags.sum()) > 0


@pytest.mark.parametrize("mode", ["simple", "hybrid"])
def test_triple_estimator_unbiased_with_exact_variance(mode):
    """Samples are independent uniform draws from U, so over seeds the
    estimate |U| (2 c_w + c_p) / (6 s) has mean t and variance
    (|U| / 3)^2 Var(Y) / s, Y the weight of one draw (1 closed wedge,
    1/2 closed 2-path, else 0), computed here from the brute-force U."""
    e = gen.chung_lu(60, 260, 2.1, 25.0, 17)
    n = 60
    _, _, tl, th = brute_classes(e, n)
    t = tl + th
    U = brute_universe(e, n, mode)
    size = len(U)
    ey = sum(wt for *_, c, wt in U if c) / size
    ey2 = sum(wt * wt for *_, c, wt in U if c) / size
    s = 50
    var = (size / 3.0) ** 2 * (ey2 - ey * ey) / s
    ests = np.array([oracle.triples(e, n, 1.0, seed, samples=s, mode=mode)["estimate"] for seed in range(1, 201)])
    assert abs(ests.mean() - t) <= 5 * math.sqrt(var / len(ests))
    assert 0.6 * var <= ests.var(ddof=1) <= 1.6 * var


def test_hybrid_after_sparsification_is_unbiased():
    """Section 3.3: sparsify with p, sample triples of the kept graph, divide
    by p^3; over seeds (both draws change) the mean is t."""
    e = gen.chung_lu(400, 3000, 2.1, 80.0, 21)
    n = 400
    t = sum(brute_classes(e, n)[2:])
    ests = np.array([oracle.triples(e, n, 0.5, seed, samples=0, mode="hybrid")["estimate"]
                     for seed in range(1, 201)])
    se = ests.std(ddof=1) / math.sqrt(len(ests))
    assert abs(ests.mean() - t) <= 5 * se


def test_triple_draws_are_uniform_over_u():
    """The map of a 64-bit hash to floor(h |U| / 2^64): with |U| = 30 (the
    wheel W_5) and 30,000 draws every triple's frequency is within 6 sigma
    of uniform.  The closed fraction of the wheel's U is 20 / 30."""
    e = gen.wheel(5)
    r = oracle.triples(e, 6, 1.0, 5, samples=30000, mode="hybrid")
    assert r["universe"] == 30
    closed = r["closed_wedge"] + r["closed_path"]
    q = 20 / 30
    assert abs(closed - q * 30000) <= 6 * math.sqrt(30000 * q * (1 - q))


# ------------------------------------------------------------ choice of p

@pytest.mark.parametrize("m,n,t,eps", [(10 ** 6, 10 ** 5, 1e7, 0.1), (48709772, 5284457, 3.1e8, 0.05),
                                       (3852985, 875713, 1.3e7, 0.02), (20000, 2000, 1300.0, 0.2)])
def test_suggested_p_balances_the_two_terms(m, n, t, eps):
    """Section 3.3 picks p where the pass over the kept edges (p m) equals
    the triple-sampling term m^(3/2) ln n / (p^(3/2) t eps^2)."""
    p = oracle.suggest_p(m, n, t, eps)
    assert 0 < p <= 1
    if p < 1:
        lhs = p * m
        rhs = m ** 1.5 * math.log(n) / (p ** 1.5 * t * eps * eps)
        assert abs(lhs - rhs) <= 1e-9 * lhs
    else:  # clamped: at p = 1 the triple term still exceeds the pass
        assert m ** 1.5 * math.log(n) / (t * eps * eps) >= m


def test_suggested_p_edge_cases():
    assert oracle.suggest_p(1000, 100, 0.0, 0.1) == 1.0  # no triangle seen: no sparsification
    assert oracle.suggest_p(1000, 100, 1e-3, 0.1) == 1.0  # clamped
    for bad in ((0, 100, 10.0, 0.1), (1000, 1, 10.0, 0.1), (1000, 100, 10.0, 0.0)):
        with pytest.raises(ValueError):
            oracle.suggest_p(*bad)
    # more triangles allow a smaller p, a tighter eps needs a larger one
    assert oracle.suggest_p(10 ** 7, 10 ** 6, 1e9, 0.1) < oracle.suggest_p(10 ** 7, 10 ** 6, 1e8, 0.1)
    assert oracle.suggest_p(10 ** 7, 10 ** 6, 1e9, 0.05) > oracle.suggest_p(10 ** 7, 10 ** 6, 1e9, 0.1)


# ------------------------------------------------------------ original-degree partition

def brute_original_classes(edges, n, kept):
    """(T_L, T_H) of the kept graph with flags deg^2 > m of the whole graph."""
    deg, _, _, _ = brute_classes(edges, n)
    m = len(edges)
    flags = deg * deg > m
    return brute_enumerate(kept, n, flags), int(flags.sum())


@pytest.mark.parametrize("seed", range(4))
def test_original_partition_matches_brute_force(seed):
    e = gen.chung_lu(50, 220, 2.1, 20.0, 30 + seed)
    for p in (1.0, 0.7, 0.4):
        kept = oracle.sample(e, p, seed + 1)
        (tl, th), h = brute_original_classes(e, 50, kept)
        r = oracle.run(e, 50, p, seed + 1, partition="original")
        assert (r["t_light"], r["t_heavy"], r["n_heavy"]) == (tl, th, h)
        assert r["m_sampled"] == len(kept)
        assert r["estimate"] == oracle.estimate(tl, th, p)


def test_original_partition_on_wheels():
    """W_4 is all heavy in the whole graph (9 > 8), so with the original
    partition every kept triangle is heavy at any p; the rim of W_6 is light
    (9 <= 12), so none is."""
    for seed in range(1, 30):
        r4 = oracle.run(gen.wheel(4), 5, 0.8, seed, partition="original")
        assert r4["t_light"] == 0 and r4["n_heavy"] == 5
        r6 = oracle.run(gen.wheel(6), 7, 0.8, seed, partition="original")
        assert r6["t_heavy"] == 0 and r6["n_heavy"] == 1


def test_partitions_agree_at_p_one():
    e = gen.chung_lu(3000, 20000, 2.1, 600.0, 5)
    a = oracle.run(e, 3000, 1.0, 1)
    b = oracle.run(e, 3000, 1.0, 1, partition="original")
    assert a == b
