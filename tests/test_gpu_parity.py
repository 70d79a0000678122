"""GPU parity: libtc (through its C ABI) against the CPU oracle.

Integer outputs (kept edge set, sampled degrees, heavy flags, m_p, n_heavy,
T_L, T_H) must be bit-exact; the float64 estimate must agree to a relative
1e-12 (both sides compute T_L/p^3 + T_H/p^3 with IEEE round-to-nearest
operations in the same order, so in practice it is identical).
"""
import math

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

INT_KEYS = ("m", "m_sampled", "n", "n_heavy", "t_light", "t_heavy")


@pytest.fixture(scope="module")
def tc():
    from paper_1011_0468_gb300 import _build, tc as _tc
    _build.build()
    return _tc


def assert_same(got, want, ctx=""):
    for k in INT_KEYS:
        assert got[k] == want[k], (ctx, k, got[k], want[k])
    e, w = got["estimate"], want["estimate"]
    assert e == w or abs(e - w) <= 1e-12 * abs(w), (ctx, e, w)


def check_graph(tc, edges, n, runs, sample=True):
    with tc.Graph(edges, n) as g:
        assert g.m == len(edges)
        for p, seed in runs:
            want = oracle.run(edges, n, p, seed, want_sample=sample)
            got = g.count(p, seed)
            assert_same(got, want, (p, seed))
            if sample:
                kept, heavy, deg = g.export_sample(p, seed)
                assert np.array_equal(kept, want["kept"]), (p, seed)
                assert np.array_equal(heavy, want["heavy"]), (p, seed)
                assert np.array_equal(deg, oracle.degrees(want["kept"], n)), (p, seed)


# ------------------------------------------------------------ configs

def test_er_2000_20000_exact_and_sampled(tc):
    """Erdos-Renyi G(2000, 20000), seed 1: p = 1 and p = 0.1 with seeds 1..10."""
    e = gen.er(2000, 20000, 1)
    check_graph(tc, e, 2000, [(1.0, 1)] + [(0.1, s) for s in range(1, 11)])


@pytest.mark.parametrize("n,m,wmax", [(100_000, 1_000_000, 5000.0), (300_000, 3_000_000, 20000.0)])
def test_chung_lu_power_law(tc, n, m, wmax):
    """Power-law graphs with heavy vertices; many radix tiles, ragged tails."""
    e = gen.chung_lu(n, m, 2.1, wmax, 5)
    check_graph(tc, e, n, [(1.0, 1), (0.5, 2), (0.1, 3), (0.01, 4)])


def test_rmat_small(tc):
    e = gen.rmat(16, 16, seed=3)
    check_graph(tc, e, 1 << 16, [(1.0, 1), (0.05, 2)])


def test_dense_core_heavy_block(tc):
    """A dense core (many heavy vertices, large T_H) inside a sparse graph.
    Core vertices of a c-vertex core at density q have degree ~ c q and are
    heavy when (c q)^2 > c^2 q / 2 + m_rest, which needs q > 1/2."""
    core = gen.er(1500, 1500 * 1499 * 4 // 10, 11)  # density 0.8
    rest = gen.er(200_000, 200_000, 12).astype(np.int64) + 1500
    e = gen.canonical(np.concatenate([core.astype(np.int64), rest,
                                      np.stack([np.arange(1500), 1500 + np.arange(1500) * 7], 1)]))
    n = 201_500
    r = oracle.run(e, n, 1.0, 1)
    assert r["n_heavy"] > 100 and r["t_heavy"] > 0
    check_graph(tc, e, n, [(1.0, 1), (0.7, 2)], sample=False)
    with tc.Graph(e, n) as g:
        assert g.count(1.0, 1)["heavy_mma_flops"] > 0  # the tensor-core path ran


def test_planted_core_spans_many_tensor_tiles(tc):
    """2048 heavy vertices: the dense block is 16 x 16 tiles of 128, with a
    ragged edge once sampling thins the core (p = 0.9)."""
    n = 100_000
    e = gen.planted_core(n, 2048, 0.7, 200_000, 21)
    r = oracle.run(e, n, 1.0, 1)
    assert r["n_heavy"] >= 2000
    check_graph(tc, e, n, [(1.0, 1), (0.9, 5)], sample=False)
    with tc.Graph(e, n) as g:
        assert g.count(1.0, 1)["heavy_mma_flops"] > 0


# ------------------------------------------------------------ closed forms

@pytest.mark.parametrize("k", [3, 4, 5, 17, 33, 34, 65, 130])
def test_complete_graphs(tc, k):
    e = gen.complete(k)
    with tc.Graph(e, k) as g:
        r = g.count(1.0, 1)
    assert (r["t_light"], r["t_heavy"], r["n_heavy"]) == (0, math.comb(k, 3), k)


@pytest.mark.parametrize("k", [4, 5, 6, 40, 100])
def test_wheels(tc, k):
    with tc.Graph(gen.wheel(k), k + 1) as g:
        r = g.count(1.0, 9)
    assert r["t_light"] + r["t_heavy"] == k
    assert r["t_heavy"] == (4 if k == 4 else 0)


def test_strict_threshold(tc):
    e, n = gen.disjoint_union(gen.complete(4), [[0, 1]], [[0, 1]], [[0, 1]])
    with tc.Graph(e, n) as g:
        r = g.count(1.0, 1)
    assert (r["m"], r["n_heavy"], r["t_light"], r["t_heavy"]) == (9, 0, 4, 0)


@pytest.mark.parametrize("edges", [gen.star(1000), gen.random_tree(5000, 2), gen.complete_bipartite(40, 60),
                                   gen.cycle(1000)])
def test_triangle_free(tc, edges):
    n = gen.num_vertices(edges)
    with tc.Graph(edges, n) as g:
        r = g.count(1.0, 3)
    assert (r["t_light"], r["t_heavy"], r["estimate"]) == (0, 0, 0.0)


# ------------------------------------------------------------ edges / inputs

def test_raw_input_is_canonicalised(tc):
    rng = np.random.default_rng(7)
    n = 3000
    raw = rng.integers(0, n, size=(60_000, 2)).astype(np.uint32)  # repeats, loops, both orders
    want_edges = oracle.canonicalize(raw, n)
    with tc.Graph(raw, n) as g:
        assert np.array_equal(g.export_edges(), want_edges)
        for p, s in ((1.0, 1), (0.3, 2)):
            assert_same(g.count(p, s), oracle.run(want_edges, n, p, s))


def test_device_input(tc):
    import torch
    rng = np.random.default_rng(8)
    n = 5000
    raw = rng.integers(0, n, size=(80_000, 2)).astype(np.int32)
    dev = torch.from_numpy(raw).cuda()
    want_edges = oracle.canonicalize(raw.astype(np.uint32), n)
    with tc.Graph(dev, n) as g:
        assert np.array_equal(g.export_edges(), want_edges)
        assert_same(g.count(0.5, 5), oracle.run(want_edges, n, 0.5, 5))


def test_pinned_host_input(tc):
    """Pinned host pairs are read in place by the device (8-byte aligned, and
    4 bytes off alignment), raw and already canonical."""
    import torch
    rng = np.random.default_rng(9)
    n = 4000
    raw = rng.integers(0, n, size=(70_000, 2)).astype(np.uint32)
    canon = oracle.canonicalize(raw, n)
    for edges in (raw, canon):
        want_edges = oracle.canonicalize(edges, n)
        buf = torch.zeros(2 * len(edges) + 1, dtype=torch.int32).pin_memory()
        for off in (0, 1):  # in uint32 units
            buf[off:off + 2 * len(edges)] = torch.from_numpy(edges.reshape(-1).view(np.int32))
            g = tc.Graph.from_address(buf.data_ptr() + 4 * off, len(edges), n, on_device=False)
            try:
                assert np.array_equal(g.export_edges(), want_edges), off
                assert_same(g.count(0.7, 3), oracle.run(want_edges, n, 0.7, 3))
            finally:
                g.close()


def test_degree_candidates_and_fallback(tc):
    """Sampled in-degrees are counted only for the vertices that can be heavy
    (a lower bound on m_p decides them); a bound of 0 makes every vertex a
    candidate, a bound above m sends every sample p < 1 through the exact
    fallback.  All three give the oracle's counts."""
    n = 40000
    e = gen.chung_lu(n, 400_000, 2.1, 4000.0, 13)
    canon = oracle.canonicalize(e, n)
    want = {p: oracle.run(canon, n, p, 5) for p in (1.0, 0.5, 0.1)}
    with tc.Graph(e, n) as g:
        for floor in (-1, 0, len(canon) + 1, -1):
            g.set_sample_floor(floor)
            for p, w in want.items():
                assert_same(g.count(p, 5), w)


def test_bounded_device_wait_gives_up_and_context_stays_usable(tc):
    """The tensor kernels' mbarrier wait, on a barrier nothing arrives at,
    gives up after its limit with TC_ETIMEOUT; the next count is exact."""
    assert tc.lib().tc_check_bounded_wait(20000) == tc.TC_ETIMEOUT
    n = 2000
    e = gen.er(n, 20000, 1)
    with tc.Graph(e, n) as g:
        assert_same(g.count(0.5, 3), oracle.run(oracle.canonicalize(e, n), n, 0.5, 3))


def test_empty_and_tiny(tc):
    for edges, n in ((np.zeros((0, 2), np.uint32), 1), (np.zeros((0, 2), np.uint32), 100_000),
                     (np.array([[0, 1]], np.uint32), 2), (gen.complete(3), 3)):
        with tc.Graph(edges, n) as g:
            for p, s in ((1.0, 1), (0.5, 2)):
                assert_same(g.count(p, s), oracle.run(edges, n, p, s))


def test_everything_dropped(tc):
    e = gen.er(1000, 5000, 4)
    with tc.Graph(e, 1000) as g:
        r = g.count(2.0 ** -53, 1)
    assert (r["m_sampled"], r["t_light"], r["t_heavy"], r["n_heavy"]) == (0, 0, 0, 0)


def test_invalid_arguments(tc):
    e = gen.er(100, 300, 4)
    with tc.Graph(e, 100) as g:
        for p in (0.0, -1.0, 1.0000001, float("nan"), float("inf")):
            with pytest.raises(tc.TCError) as ei:
                g.count(p, 1)
            assert ei.value.status == tc.TC_EINVAL
        # the graph stays usable after rejected calls
        assert_same(g.count(1.0, 1), oracle.run(e, 100, 1.0, 1))
    with pytest.raises(tc.TCError) as ei:
        tc.Graph(np.array([[0, 1], [2, 100]], np.uint32), 100)
    assert ei.value.status == tc.TC_EINVAL


def test_async_matches_blocking(tc):
    import ctypes
    import torch
    e = gen.chung_lu(50_000, 400_000, 2.1, 2000.0, 9)
    buf = torch.empty(ctypes.sizeof(tc.tc_result), dtype=torch.uint8, pin_memory=True)
    with tc.Graph(e, 50_000) as g:
        want = g.count(0.4, 3)
        g.count_async(0.4, 3, buf.data_ptr())
        g.sync()
        got = tc.tc_result.from_address(buf.data_ptr()).as_dict()
    for k in INT_KEYS + ("estimate",):
        assert got[k] == want[k]


def test_small_graph_in_fresh_process():
    """Per-function launch limits start at their defaults in every process:
    a small graph counted first thing in a new process must work too."""
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    code = ("import sys; sys.path.insert(0, %r)\n"
            "import gen, oracle\n"
            "from paper_1011_0468_gb300 import tc\n"
            "e = gen.chung_lu(20000, 200000, 2.1, 3000.0, 3)\n"
            "with tc.Graph(e, 20000) as g:\n"
            "    r = g.count(1.0, 1)\n"
            "w = oracle.run(e, 20000, 1.0, 1)\n"
            "assert (r['t_light'], r['t_heavy']) == (w['t_light'], w['t_heavy'])\n" % root)
    out = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stdout + out.stderr


def test_repeat_is_deterministic(tc):
    e = gen.chung_lu(100_000, 800_000, 2.1, 4000.0, 10)
    with tc.Graph(e, 100_000) as g:
        a = [g.count(0.3, 5) for _ in range(3)]
    for r in a[1:]:
        for k in INT_KEYS + ("estimate",):
            assert r[k] == a[0][k]


# ------------------------------------------------------------ CSR properties

def test_csr_is_degree_oriented_and_sorted(tc):
    """The CSR is oriented by the rank (degree in the whole graph, id), fixed
    at creation, and every row lists its out-neighbours in rank order."""
    n = 100_000
    e = gen.chung_lu(n, 1_000_000, 2.1, 5000.0, 6)
    full = oracle.degrees(oracle.canonicalize(e, n), n).astype(np.int64)
    rank = np.empty(n, np.int64)
    rank[np.lexsort((np.arange(n), full))] = np.arange(n)
    for p, s in ((1.0, 1), (0.2, 2)):
        want = oracle.run(e, n, p, s, want_sample=True)
        kept = want["kept"]
        with tc.Graph(e, n) as g:
            rowptr, col = g.export_csr(p, s)
        assert rowptr[0] == 0 and rowptr[-1] == len(kept) == len(col)
        assert np.all(np.diff(rowptr.astype(np.int64)) >= 0)
        src = np.repeat(np.arange(n, dtype=np.int64), np.diff(rowptr.astype(np.int64)))
        dst = col.astype(np.int64)
        # every row strictly increasing in rank
        same = src[1:] == src[:-1]
        assert np.all(rank[dst[1:][same]] > rank[dst[:-1][same]])
        # orientation: the rank of src below that of dst
        assert np.all(rank[src] < rank[dst])
        # the undirected edge set is exactly the kept set
        keys = np.minimum(src, dst) * (1 << 32) + np.maximum(src, dst)
        kk = kept.astype(np.int64)
        assert np.array_equal(np.sort(keys), kk[:, 0] * (1 << 32) + kk[:, 1])
