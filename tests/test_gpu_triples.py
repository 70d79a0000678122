"""Triple sampling on the GPU (tc_count_triples) against the oracle, field
by field: the sampled graph, the heavy rows, |U|, the number of samples,
the closed wedges and 2-paths among them (integers, bit-exact) and the
float64 estimate (the same IEEE operations in the same order, compared with
==).  Graphs span several warps per row, hubs whose 2-path rows span many
blocks, ragged tails, and the degenerate cases (no edges, no wedges, every
triple closed)."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

KEYS = ("m", "m_sampled", "n", "n_heavy", "universe", "samples", "closed_wedge", "closed_path", "estimate")


def _tc():
    from paper_1011_0468_gb300 import tc
    return tc


def check(g, edges, n, p, seed, samples, mode):
    got = g.count_triples(p, seed, samples, mode)
    want = oracle.triples(edges, n, p, seed, samples, mode)
    for k in KEYS:
        assert got[k] == want[k], (k, p, seed, samples, mode, got[k], want[k])
    assert got["mode"] == (1 if mode == "hybrid" else 0)
    return got


CASES = [
    ("er", lambda: (gen.er(2000, 20000, 1), 2000)),
    ("chung_lu", lambda: (gen.chung_lu(20000, 200000, 2.1, 3000.0, 3), 20000)),
    ("planted_core", lambda: (gen.planted_core(30000, 600, 0.8, 120000, 4), 30000)),
    ("rmat16", lambda: (gen.rmat(16, 16, seed=2), 1 << 16)),
]


@pytest.mark.parametrize("mode", ["simple", "hybrid"])
@pytest.mark.parametrize("name,make", CASES)
def test_triples_match_the_oracle(name, make, mode):
    tc = _tc()
    edges, n = make()
    with tc.Graph(edges, n) as g:
        for p, seed, s in ((1.0, 1, 0), (1.0, 7, 100003), (0.3, 2, 0), (0.1, 5, 50000), (0.55, 9, 1)):
            r = check(g, edges, n, p, seed, s, mode)
            assert r["universe"] > 0
        # the exact count of the same sample is what the estimates target
        exact = g.count(1.0, 1)["estimate"]
        est = g.count_triples(1.0, 11, 400000, mode)["estimate"]
        assert abs(est - exact) <= 0.25 * exact


def test_triples_degenerate_graphs():
    tc = _tc()
    for edges, n in ((np.zeros((0, 2), np.uint32), 5), (gen.star(40), 41), (gen.complete_bipartite(6, 9), 15),
                     (gen.cycle(50), 50)):
        with tc.Graph(edges, n) as g:
            for mode in ("simple", "hybrid"):
                r = check(g, edges, n, 1.0, 3, 1000, mode)
                assert r["closed_wedge"] == r["closed_path"] == 0 and r["estimate"] == 0.0
                check(g, edges, n, 0.5, 4, 0, mode)


def test_simple_mode_exact_on_complete_graph():
    tc = _tc()
    k = 300  # rows of 299 entries: several warps per row in the compaction
    edges = gen.complete(k)
    with tc.Graph(edges, k) as g:
        r = check(g, edges, k, 1.0, 5, 12345, "simple")
        assert r["closed_wedge"] == 12345 and r["estimate"] == k * (k - 1) * (k - 2) // 6
        check(g, edges, k, 1.0, 5, 12345, "hybrid")  # every vertex heavy: 2-paths only
        check(g, edges, k, 0.7, 6, 0, "hybrid")


def test_triples_reject_bad_arguments():
    tc = _tc()
    edges = gen.er(100, 300, 1)
    with tc.Graph(edges, 100) as g:
        for p in (0.0, 1.5, float("nan")):
            with pytest.raises(tc.TCError) as ei:
                g.count_triples(p, 1)
            assert ei.value.status == tc.TC_EINVAL
        import ctypes
        r = tc.tc_triple_result()
        assert tc.lib().tc_count_triples(g.handle, 1.0, 1, 0, 7, ctypes.byref(r)) == tc.TC_EINVAL
