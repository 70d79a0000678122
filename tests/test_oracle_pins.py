"""Pins for the CPU oracle against facts fixed outside it.

Each test ties one part of the oracle to something other than its own code:
published generator outputs, exact rational arithmetic, closed-form triangle
counts, brute-force enumeration, the adjacency-matrix identity for triangles
(t = trace(A^3) / 6, Section 5.1 of the paper), and the exact mean and
variance of the edge-sparsification estimator (Section 3.1).
"""
import itertools
import math
import os
from fractions import Fraction

import numpy as np
import pytest

import gen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
GAMMA = 0x9E3779B97F4A7C15
MASK = (1 << 64) - 1


# ------------------------------------------------------------ helpers (brute)

def adjacency(edges, n):
    A = np.zeros((n, n), dtype=np.float64)
    for u, v in np.asarray(edges, dtype=np.int64).reshape(-1, 2):
        A[u, v] = A[v, u] = 1
    return A


def brute_classes(edges, n):
    """Degrees, heavy flags (deg^2 > m) and (T_L, T_H) from the adjacency
    matrix: t = trace(A^3)/6, and the all-heavy count is the same identity on
    the heavy-induced submatrix."""
    A = adjacency(edges, n)  # float64: every entry of A^3 is an exact integer
    m = int(round(A.sum())) // 2
    deg = A.sum(axis=1).astype(np.int64)
    heavy = deg * deg > m
    t = int(round(np.trace(A @ A @ A))) // 6
    H = A[np.ix_(heavy, heavy)]
    th = int(round(np.trace(H @ H @ H))) // 6 if len(H) else 0
    return deg, heavy, t - th, th


def brute_enumerate(edges, n, heavy):
    """Explicit O(n^3) enumeration of triangles, classified by heavy flags."""
    A = adjacency(edges, n)
    tl = th = 0
    for a, b, c in itertools.combinations(range(n), 3):
        if A[a, b] and A[b, c] and A[a, c]:
            if heavy[a] and heavy[b] and heavy[c]:
                th += 1
            else:
                tl += 1
    return tl, th


# ------------------------------------------------------------ splitmix64

def test_splitmix64_published_outputs():
    rows = [l.split() for l in open(os.path.join(GOLDEN, "splitmix64_state0.txt"))
            if l.strip() and not l.startswith("#")]
    assert len(rows) == 4
    for k, hexval in rows:
        assert oracle.splitmix64((int(k) * GAMMA) & MASK) == int(hexval, 16)


def test_threshold_is_floor_of_p_times_2_53():
    for p in [1.0, 0.5, 0.1, 0.01, 0.05, 1e-9, 0.3333333333333333, 0.9999999999999999, 2.0 ** -53]:
        assert oracle.threshold(p) == math.floor(Fraction(p) * 2 ** 53)


def test_p_one_keeps_everything():
    e = gen.er(300, 3000, 5)
    for seed in (0, 1, 2 ** 63, MASK):
        assert np.array_equal(oracle.sample(e, 1.0, seed), e)


def test_tiny_p_keeps_nothing():
    e = gen.er(300, 3000, 5)
    assert len(oracle.sample(e, 2.0 ** -53, 3)) == 0


def test_kept_fraction_within_6_sigma():
    e = gen.er(20000, 1_000_000, 9)
    m = len(e)
    for p in (0.5, 0.1, 0.01):
        for seed in (1, 2):
            k = len(oracle.sample(e, p, seed))
            sigma = math.sqrt(m * p * (1 - p))
            assert abs(k - m * p) <= 6 * sigma, (p, seed, k)


def test_seeds_draw_independent_samples():
    # Two seeds keep an edge together with probability p^2 (pairwise
    # independence across seeds), and one seed's draws of the two edges of a
    # pair are independent too.
    e = gen.er(20000, 1_000_000, 9)
    p, m = 0.3, len(e)
    keys = lambda s: set(map(tuple, oracle.sample(e, p, s).tolist()))
    both = len(keys(11) & keys(12))
    sigma = math.sqrt(m * p * p * (1 - p * p))
    assert abs(both - m * p * p) <= 6 * sigma


def test_sample_preserves_order_and_subset():
    e = gen.er(500, 5000, 2)
    k = oracle.sample(e, 0.37, 77)
    s = set(map(tuple, e.tolist()))
    assert all(tuple(x) in s for x in k.tolist())
    kk = k.astype(np.int64)
    keys = kk[:, 0] * (1 << 32) + kk[:, 1]
    assert np.all(np.diff(keys) > 0)


# ------------------------------------------------------------ canonical input

def test_canonicalize_drops_loops_and_repeats():
    raw = np.array([[3, 1], [1, 3], [2, 2], [0, 4], [4, 0], [1, 2], [1, 3]], dtype=np.uint32)
    c = oracle.canonicalize(raw, 5)
    assert c.tolist() == [[0, 4], [1, 2], [1, 3]]


def test_canonicalize_rejects_out_of_range():
    with pytest.raises(ValueError):
        oracle.canonicalize(np.array([[0, 5]], dtype=np.uint32), 5)


def test_canonicalize_matches_generator_canonical_form():
    rng = np.random.default_rng(4)
    raw = rng.integers(0, 50, size=(400, 2))
    assert np.array_equal(oracle.canonicalize(raw, 50), gen.canonical(raw))


# ------------------------------------------------------------ closed forms

def run1(edges, n=None, p=1.0, seed=1):
    n = gen.num_vertices(edges) if n is None else n
    return oracle.run(edges, n, p, seed)


@pytest.mark.parametrize("k", range(3, 13))
def test_complete_graph(k):
    r = run1(gen.complete(k))
    # deg = k-1, m = k(k-1)/2, (k-1)^2 > m for k >= 3: every vertex heavy
    assert r["n_heavy"] == k
    assert (r["t_light"], r["t_heavy"]) == (0, math.comb(k, 3))
    assert r["estimate"] == math.comb(k, 3)


@pytest.mark.parametrize("k", range(4, 20))
def test_wheel(k):
    r = run1(gen.wheel(k))
    assert r["t_light"] + r["t_heavy"] == k
    if k == 4:
        # hub 4^2 = 16 > 8 and rim 3^2 = 9 > 8: all heavy
        assert (r["n_heavy"], r["t_heavy"]) == (5, 4)
    else:
        # rim 9 <= 2k: light, so every triangle has a light vertex
        assert (r["n_heavy"], r["t_light"], r["t_heavy"]) == (1, k, 0)


def test_heavy_threshold_is_strict():
    # K4 plus three separate edges: m = 9, K4 degrees 3, 3^2 = 9 is not > 9.
    g, n = gen.disjoint_union(gen.complete(4), [[0, 1]], [[0, 1]], [[0, 1]])
    r = run1(g, n)
    assert r["m"] == 9 and r["n_heavy"] == 0
    assert (r["t_light"], r["t_heavy"]) == (4, 0)
    # with one separate edge fewer, m = 8 < 9 and the K4 vertices are heavy
    g2, n2 = gen.disjoint_union(gen.complete(4), [[0, 1]], [[0, 1]])
    r2 = run1(g2, n2)
    assert r2["m"] == 8 and r2["n_heavy"] == 4
    assert (r2["t_light"], r2["t_heavy"]) == (0, 4)


@pytest.mark.parametrize("g", [gen.star(50), gen.cycle(10), gen.cycle(4), gen.random_tree(200, 3),
                               gen.complete_bipartite(7, 9), gen.complete_bipartite(1, 30)])
def test_triangle_free(g):
    r = run1(g)
    assert (r["t_light"], r["t_heavy"], r["estimate"]) == (0, 0, 0.0)


def test_single_triangle():
    r = run1(gen.cycle(3))
    assert r["t_light"] + r["t_heavy"] == 1


def test_disjoint_union_adds():
    parts = [gen.complete(6), gen.wheel(9), gen.er(60, 400, 3), gen.complete_bipartite(5, 5)]
    g, n = gen.disjoint_union(*parts)
    total = sum(sum(brute_classes(p, gen.num_vertices(p))[2:]) for p in parts)
    r = run1(g, n)
    assert r["t_light"] + r["t_heavy"] == total


def test_planted_clique_in_bipartite():
    k = 9
    bip = gen.complete_bipartite(20, 25)
    clique = gen.complete(k, offset=0)  # vertices 0..8 all on the left side
    g = gen.canonical(np.concatenate([bip, clique]))
    r = run1(g, 45)
    # the left side is independent in K_{20,25}; the only triangles are the
    # clique's own and clique-edge + right vertex: C(9,3) + C(9,2) * 25
    assert r["t_light"] + r["t_heavy"] == math.comb(k, 3) + math.comb(k, 2) * 25


def test_empty_and_edgeless():
    r = oracle.run(np.zeros((0, 2), dtype=np.uint32), 10, 0.5, 1)
    assert (r["m"], r["m_sampled"], r["n_heavy"], r["t_light"], r["t_heavy"]) == (0, 0, 0, 0, 0)


def test_bad_p_rejected():
    for p in (0.0, -0.1, 1.5, float("nan")):
        with pytest.raises(ValueError):
            oracle.run(gen.complete(4), 4, p, 1)


# ------------------------------------------------------------ brute force

@pytest.mark.parametrize("seed", range(40))
def test_brute_force_random_tiny(seed):
    rng = np.random.default_rng(seed)
    n = int(rng.integers(3, 40))
    dens = float(rng.choice([0.05, 0.2, 0.5, 0.9]))
    A = np.triu(rng.random((n, n)) < dens, 1)
    g = np.argwhere(A).astype(np.uint32)
    p = float(rng.choice([1.0, 0.7, 0.4]))
    s = int(rng.integers(0, 2 ** 63))
    r = oracle.run(g, n, p, s, want_sample=True)
    kept = r["kept"]
    deg, heavy, tl, th = brute_classes(kept, n)
    assert np.array_equal(oracle.degrees(kept, n), deg)
    assert np.array_equal(r["heavy"].astype(bool), heavy)
    assert r["n_heavy"] == int(heavy.sum())
    assert (r["t_light"], r["t_heavy"]) == (tl, th)
    assert r["estimate"] == tl / p ** 3 + th / p ** 3


@pytest.mark.parametrize("seed", range(8))
def test_explicit_enumeration_with_mixed_flags(seed):
    # arbitrary (not degree-derived) flags exercise the classifier on every
    # heavy/light combination of a triangle
    rng = np.random.default_rng(100 + seed)
    n = 22
    A = np.triu(rng.random((n, n)) < 0.45, 1)
    g = np.argwhere(A).astype(np.uint32)
    flags = (rng.random(n) < 0.5).astype(np.uint8)
    assert oracle.count_classes(g, n, flags) == brute_enumerate(g, n, flags)


def test_heavy_bound_invariant():
    # Section 3.2: at most 2 m^(1/2) vertices have degree above m^(1/2)
    for seed in range(5):
        g = gen.chung_lu(20000, 200000, 2.1, 3000.0, seed)
        for p in (1.0, 0.3):
            r = oracle.run(g, 20000, p, seed)
            assert r["n_heavy"] <= 2 * math.sqrt(r["m_sampled"])


# ------------------------------------------------------------ estimator

def exact_moments(edges, n, p):
    """Section 3.1: E[T_p] = p^3 t and, from the independence of the edge
    draws, Var[T_p] = t (p^3 - p^6) + 2 S (p^5 - p^6) where S counts pairs of
    triangles that share an edge (two triangles share at most one edge)."""
    A = adjacency(edges, n)
    t = int(round(np.trace(A @ A @ A))) // 6
    common = (A @ A) * A  # common[u, v] = #triangles on edge uv
    tri_per_edge = np.rint(common[np.triu_indices(n, 1)]).astype(np.int64)
    S = int(sum(c * (c - 1) // 2 for c in tri_per_edge))
    var_tp = t * (p ** 3 - p ** 6) + 2 * S * (p ** 5 - p ** 6)
    return t, var_tp / p ** 6


@pytest.mark.parametrize("graph,p", [("er", 0.1), ("er", 0.5), ("dense", 0.3)])
def test_estimator_unbiased_with_exact_variance(graph, p):
    if graph == "er":
        g, n = gen.er(2000, 20000, 1), 2000
    else:
        g, n = gen.er(120, 2500, 7), 120
    t, var_est = exact_moments(g, n, p)
    ests = np.array([oracle.run(g, n, p, s)["estimate"] for s in range(1, 201)])
    sd_mean = math.sqrt(var_est / len(ests))
    assert abs(ests.mean() - t) <= 5 * sd_mean, (ests.mean(), t, sd_mean)
    # the sample variance of 200 draws lies within a wide band of the exact one
    ratio = ests.var(ddof=1) / var_est
    assert 0.6 < ratio < 1.6, ratio


def test_p_one_is_exact_on_c1():
    g = gen.er(2000, 20000, 1)
    r = oracle.run(g, 2000, 1.0, 1)
    t = brute_classes(g, 2000)
    assert r["t_light"] + r["t_heavy"] == t[2] + t[3]
    assert r["estimate"] == float(r["t_light"] + r["t_heavy"])
    assert r["n_heavy"] == 0  # max degree well below sqrt(20000)
