"""Batched counting (tc_batch_*): every graph of a batch must get exactly
the result of counting it alone (tc_graph_create + tc_count), and the
oracle's result on a sample of graphs."""
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


def mixed_graphs():
    """Uneven small graphs: ER and power-law, tiny and empty ones, raw pairs."""
    rng = np.random.default_rng(3)
    graphs = []
    for i, spec in enumerate(gen.batch_specs(40, seed=7)):
        spec = dict(spec, n=min(spec["n"], 6000), m=min(spec["m"], 60000))
        graphs.append((gen.batch_graph(spec), spec["n"]))
    graphs.append((np.zeros((0, 2), np.uint32), 1))
    graphs.append((np.zeros((0, 2), np.uint32), 500))
    graphs.append((gen.complete(20), 20))
    graphs.append((gen.wheel(9), 10))
    raw = rng.integers(0, 800, size=(9000, 2)).astype(np.uint32)  # repeats, loops
    graphs.append((raw, 800))
    graphs.append((gen.chung_lu(30000, 300000, 2.1, 3000.0, 9), 30000))
    return graphs


def single(tc, edges, n, p, seed):
    with tc.Graph(edges, n) as g:
        return g.count(p, seed)


def test_batch_equals_single_graph_counts(tc):
    graphs = mixed_graphs()
    k = len(graphs)
    rng = np.random.default_rng(11)
    p = rng.choice([0.1, 0.5, 1.0], size=k)
    seed = rng.integers(1, 2 ** 62, size=k, dtype=np.uint64)
    with tc.Batch(graphs) as b:
        for rep in range(2):  # second call replays the captured launch
            pr = p if rep == 0 else np.roll(p, 1)
            res = b.count(pr, seed + rep)
            for g, (e, n) in enumerate(graphs):
                want = single(tc, e, n, float(pr[g]), int(seed[g]) + rep)
                for key in KEYS:
                    assert res[key][g] == want[key], (rep, g, key, res[key][g], want[key])


def test_batch_against_oracle_sample(tc):
    graphs = mixed_graphs()
    k = len(graphs)
    p = np.array([[1.0, 0.5, 0.1][g % 3] for g in range(k)])
    seed = np.arange(1, k + 1, dtype=np.uint64)
    with tc.Batch(graphs) as b:
        res = b.count(p, seed)
    for g in range(0, k, 5):
        e, n = graphs[g]
        canon = oracle.canonicalize(e, n)
        want = oracle.run(canon, n, float(p[g]), int(seed[g]))
        for key in ("m", "m_sampled", "n_heavy", "t_light", "t_heavy", "estimate"):
            assert res[key][g] == want[key], (g, key)


def test_autotuned_schedule_gives_identical_counts(tc):
    graphs = mixed_graphs()
    k = len(graphs)
    p = np.full(k, 0.5)
    seed = np.arange(7, 7 + k, dtype=np.uint64)
    with tc.Batch(graphs) as b:
        before = b.count(p, seed)
        desc = b.autotune(p, seed)
        assert "warp_max=" in desc and "mid_max=" in desc
        assert "warp per owner" in desc and ("hash set" in desc or "binary search" in desc)
        after = b.count(p, seed)
    for key in KEYS:
        assert np.array_equal(before[key], after[key]), key


def test_batch_rejects_bad_input(tc):
    with pytest.raises(tc.TCError) as e:
        tc.Batch([(np.array([[0, 1]], np.uint32), 2), (np.array([[0, 5]], np.uint32), 5)])
    assert e.value.status == tc.TC_EINVAL
    with tc.Batch([(gen.complete(5), 5)]) as b:
        with pytest.raises(tc.TCError):
            b.count([0.0], [1])
        assert b.count([1.0], [1])["t_heavy"][0] + b.count([1.0], [1])["t_light"][0] == 10
