"""Parity at the sizes that matter:
- the tensor-core contraction with accumulator entries above 2^14 (a
  20,000-vertex clique: every pair of clique vertices has 19,998 common
  neighbours), in the heavy block and in forced dense cores of 8192 to
  65536 ranks, against the closed form C(c, 3);
- the whole 10,000-graph batched workload against the single-graph path
  graph by graph, and a hundred of its graphs (the largest and a spread of
  the rest) against the oracle, plus a batch with large owners (out-degree
  above 1024);
- the served path with 2^23-edge Chung-Lu graphs in the mix.
"""
import math
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu
KEYS = ("m", "m_sampled", "n", "n_heavy", "t_light", "t_heavy", "estimate")


@pytest.fixture(scope="module")
def tc():
    from paper_1011_0468_gb300 import _build, tc as _tc
    _build.build()
    return _tc


def clique_pairs(c: int, offset: int = 0) -> np.ndarray:
    """Canonical edge list of K_c on vertices offset .. offset + c - 1."""
    lens = c - 1 - np.arange(c - 1, dtype=np.int64)  # row u holds u + 1 .. c - 1
    start = np.concatenate([[0], np.cumsum(lens)[:-1]])
    u = np.repeat(np.arange(c - 1, dtype=np.int64), lens)
    v = np.arange(len(u), dtype=np.int64) - np.repeat(start, lens) + u + 1
    return np.stack([u + offset, v + offset], axis=1).astype(np.uint32)


def test_clique_pairs_builder():
    for c in (2, 3, 7, 40):
        assert np.array_equal(clique_pairs(c, 5), gen.complete(c, offset=5))


def test_tensor_accumulator_above_2_14(tc):
    """K_20000 next to a triangle-free bipartite graph (n = 2^17): every
    clique vertex is heavy, the heavy block holds all 20,000 of them, and the
    entries of U U reach 19,998.  Every core size and no core give exactly
    C(20000, 3) heavy triangles and no light one."""
    c = 20000
    n = 1 << 17
    rng = np.random.default_rng(4)
    left = rng.integers(c, c + 40000, size=600000)
    right = rng.integers(c + 40000, n, size=600000)
    bip = gen.canonical(np.stack([left, right], axis=1))
    edges = np.concatenate([clique_pairs(c), bip])
    want = math.comb(c, 3)
    with tc.Graph(edges, n) as g:
        assert g.m == c * (c - 1) // 2 + len(bip)
        for ranks in (-1, 0, 8192, 32768, 65536):
            g.set_core_ranks(ranks)
            r = g.count(1.0, 1)
            assert r["n_heavy"] == c, ranks
            assert (r["t_light"], r["t_heavy"]) == (0, want), ranks
            assert r["estimate"] == float(want)
            assert r["heavy_mma_flops"] > 0
        # a sample of the clique: the count of the sampled graph is checked
        # against the same graph counted without any dense block
        g.set_core_ranks(0)
        a = g.count(0.9, 3)
        g.set_core_ranks(65536)
        b = g.count(0.9, 3)
        assert all(a[k] == b[k] for k in KEYS)


def test_full_batch_workload_equals_single_and_oracle(tc):
    """All 10,000 graphs of the batched workload in one batch: every graph's
    result equals its single-graph count; 100 of them (the 50 with the most
    edges, 50 spread over the rest) equal the oracle's."""
    specs = gen.batch_specs(10000, seed=1)
    with ThreadPoolExecutor(16) as ex:
        graphs = list(ex.map(gen.batch_graph, specs))
    k = len(graphs)
    p = np.array([s["p"] for s in specs])
    seed = np.array([s["seed"] for s in specs], dtype=np.uint64)
    with tc.Batch([(e, s["n"]) for e, s in zip(graphs, specs)]) as b:
        res = b.count(p, seed)
    objs = []
    try:
        for e, s in zip(graphs, specs):
            objs.append(tc.Graph(e, s["n"]))
        single = tc.tc_count_batch(objs, p, seed)  # resident graphs, one launch
        for j, o in enumerate(objs):
            if j % 10 == 0:
                r = o.count(float(p[j]), int(seed[j]))
                for key in KEYS:
                    assert res[key][j] == r[key], (j, key)
        for key in KEYS:
            assert np.array_equal(res[key], single[key]), key
    finally:
        for o in objs:
            o.close()
    by_m = np.argsort([len(e) for e in graphs])
    pick = list(by_m[-50:]) + list(by_m[:-50][:: (k - 50) // 50][:50])

    def run(j):
        return oracle.run(graphs[j], specs[j]["n"], float(p[j]), int(seed[j]))

    with ThreadPoolExecutor(16) as ex:
        wants = list(ex.map(run, pick))
    for j, want in zip(pick, wants):
        for key in KEYS:
            assert res[key][j] == want[key], (j, key, res[key][j], want[key])


def test_batch_with_large_owners(tc):
    """A batch whose graphs have owners with out-degree above 1024 (a planted
    3000-vertex core at density 0.9), so the large-owner kernel runs on a
    union: equal to the single-graph counts and to the oracle."""
    graphs = [(gen.planted_core(40000, 3000, 0.9, 200000, 3), 40000),
              (gen.er(2000, 20000, 1), 2000),
              (gen.planted_core(20000, 2200, 0.95, 50000, 8), 20000)]
    p = np.array([1.0, 0.5, 0.8])
    seed = np.array([1, 2, 3], dtype=np.uint64)
    with tc.Batch(graphs) as b:
        res = b.count(p, seed)
    for j, (e, n) in enumerate(graphs):
        want = oracle.run(e, n, float(p[j]), int(seed[j]))
        for key in KEYS:
            assert res[key][j] == want[key], (j, key)


def test_server_with_large_graphs_in_the_mix(tc):
    """Requests on two Chung-Lu graphs of 2^23 edges mixed with small ones
    (served in shared slot launches): each equals its graph counted alone."""
    small = []
    for spec in gen.batch_specs(40, seed=9):
        small.append((gen.batch_graph(spec), spec["n"]))
    large = [(gen.cached("chung_lu", gen.chung_lu, 1 << 20, 1 << 23, 2.1, 35000.0, 100 + i), 1 << 20)
             for i in range(2)]
    pool = small + large
    rng = np.random.default_rng(17)
    reqs = []
    for i in range(300):
        gid = len(small) + (i // 10) % 2 if i % 10 == 0 else int(rng.integers(0, len(small)))
        reqs.append((gid, float(rng.choice([0.1, 0.5, 1.0])), int(rng.integers(1, 2 ** 62))))
    with tc.Server(40 * 10 ** 9, slots=3, slot_edges=1 << 25, slot_vertices=1 << 23, slot_requests=1024) as srv:
        gids = [srv.add_graph(e, n) for e, n in pool]
        tickets = [srv.submit(gids[g], p, s) for g, p, s in reqs]
        got = [srv.wait(t, 600000) for t in tickets]
    alone = {}
    try:
        for (g, p, s), r in zip(reqs, got):
            if g not in alone:
                alone[g] = tc.Graph(*pool[g])
            want = alone[g].count(p, s)
            assert r["status"] == 0
            for key in KEYS:
                assert r[key] == want[key], (g, p, s, key)
        assert any(r["wave_size"] > 1 for r in got)
    finally:
        for o in alone.values():
            o.close()
