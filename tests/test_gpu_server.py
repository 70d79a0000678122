"""Served counting (tc_server_*): each request's result must be the same
counted alone (tc_graph_create + tc_count on its graph) and in the mix of
requests that share slot launches, including after its graph was evicted by
the HBM budget and uploaded again."""
import threading

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


def pool():
    """Uneven graphs: batch-style ER / power-law, tiny, empty, raw pairs and
    one larger Chung-Lu graph."""
    graphs = []
    for spec in gen.batch_specs(24, seed=21):
        spec = dict(spec, n=min(spec["n"], 8000), m=min(spec["m"], 80000))
        graphs.append((gen.batch_graph(spec), spec["n"]))
    rng = np.random.default_rng(5)
    graphs.append((np.zeros((0, 2), np.uint32), 7))
    graphs.append((np.array([[3, 3], [4, 4]], np.uint32), 9))  # self-loops only
    graphs.append((gen.complete(24), 24))
    graphs.append((gen.wheel(12), 13))
    graphs.append((rng.integers(0, 900, size=(12000, 2)).astype(np.uint32), 900))
    graphs.append((gen.chung_lu(40000, 400000, 2.1, 4000.0, 13), 40000))
    return graphs


class Alone:
    """tc_count on each graph by itself, cached per graph."""

    def __init__(self, tc, graphs):
        self.tc, self.graphs, self.g = tc, graphs, {}

    def __call__(self, gid, p, seed):
        if gid not in self.g:
            e, n = self.graphs[gid]
            self.g[gid] = self.tc.Graph(e, n)
        return self.g[gid].count(p, seed)

    def close(self):
        for g in self.g.values():
            g.close()


def requests(k, n_graphs, seed):
    rng = np.random.default_rng(seed)
    gids = rng.integers(0, n_graphs, size=k)
    ps = rng.choice([0.1, 0.5, 1.0], size=k)
    seeds = rng.integers(1, 2 ** 63, size=k, dtype=np.uint64)
    return [(int(g), float(p), int(s)) for g, p, s in zip(gids, ps, seeds)]


def check_same(got, want, what):
    assert got["status"] == 0, what
    for key in KEYS:
        assert got[key] == want[key], (what, key, got[key], want[key])


def test_each_result_same_alone_and_in_the_mix(tc):
    graphs = pool()
    reqs = requests(400, len(graphs), 1)
    alone = Alone(tc, graphs)
    with tc.Server(8 << 30, slots=2, slot_edges=1 << 21, slot_vertices=1 << 20, slot_requests=128) as srv:
        gids = [srv.add_graph(e, n) for e, n in graphs]
        assert gids == list(range(len(graphs)))
        tickets = [srv.submit(g, p, s) for g, p, s in reqs]  # a burst: requests share launches
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(reqs) and st["queued"] == 0
    assert st["max_wave"] > 1 and st["waves"] < len(reqs)
    for i, (g, p, s) in enumerate(reqs):
        check_same(got[i], alone(g, p, s), ("request", i, g, p))
        assert got[i]["t_submit_us"] <= got[i]["t_admit_us"] <= got[i]["t_done_us"]
        assert 1 <= got[i]["wave_size"] <= 128
    # the same requests one at a time (every launch holds a single request)
    with tc.Server(8 << 30, slots=1, slot_edges=1 << 21, slot_vertices=1 << 20, slot_requests=1) as srv:
        for e, n in graphs:
            srv.add_graph(e, n)
        for i, (g, p, s) in enumerate(reqs[:60]):
            r = srv.wait(srv.submit(g, p, s))
            assert r["wave_size"] == 1
            check_same(r, got[i], ("single-request launch", i))
    alone.close()


def test_server_against_oracle_sample(tc):
    graphs = pool()
    reqs = requests(40, len(graphs), 2)
    with tc.Server(4 << 30, slots=2, slot_edges=1 << 21, slot_vertices=1 << 20, slot_requests=64) as srv:
        for e, n in graphs:
            srv.add_graph(e, n)
        tickets = [srv.submit(g, p, s) for g, p, s in reqs]
        got = [srv.wait(t) for t in tickets]
    for i in range(0, len(reqs), 4):
        g, p, s = reqs[i]
        e, n = graphs[g]
        want = oracle.run(oracle.canonicalize(e, n), n, p, s)
        for key in ("m", "m_sampled", "n_heavy", "t_light", "t_heavy", "estimate"):
            assert got[i][key] == want[key], (i, key)


def test_budget_evicts_and_results_stay_the_same(tc):
    graphs = pool()
    slot = dict(slots=2, slot_edges=1 << 21, slot_vertices=1 << 20, slot_requests=32)
    with tc.Server(1 << 40, **slot) as probe:
        slot_bytes = probe.stats()["slot_bytes"]
    # room for the largest graph and a little more: most graphs must be
    # evicted and uploaded again as the requests cycle through them (a
    # resident graph holds 16 bytes per canonical edge)
    sizes = [len(oracle.canonicalize(e, n)) * 16 for e, n in graphs]
    room = max(sizes) + 200_000
    reqs = requests(300, len(graphs), 3)
    alone = Alone(tc, graphs)
    with tc.Server(slot_bytes + room, **slot) as srv:
        for e, n in graphs:
            srv.add_graph(e, n)
        assert srv.stats()["resident_bytes"] <= room
        tickets = [srv.submit(g, p, s) for g, p, s in reqs]
        got = [srv.wait(t) for t in tickets]
        st = srv.stats()
    assert st["evictions"] > 0 and st["uploads"] > 0
    assert st["resident_bytes"] <= room
    for i, (g, p, s) in enumerate(reqs):
        check_same(got[i], alone(g, p, s), ("budget", i))
    alone.close()


def test_concurrent_submitters(tc):
    graphs = pool()
    alone = Alone(tc, graphs)
    out = {}
    with tc.Server(4 << 30, slots=3, slot_edges=1 << 21, slot_vertices=1 << 20, slot_requests=64) as srv:
        for e, n in graphs:
            srv.add_graph(e, n)

        def client(c):
            for j, (g, p, s) in enumerate(requests(60, len(graphs), 100 + c)):
                out[(c, j)] = ((g, p, s), srv.wait(srv.submit(g, p, s)))

        threads = [threading.Thread(target=client, args=(c,)) for c in range(4)]
        for t in threads:
            t.start()
        for t in threads:
            t.join()
    assert len(out) == 240
    for key, ((g, p, s), r) in out.items():
        check_same(r, alone(g, p, s), key)
    alone.close()


def test_server_errors(tc):
    with pytest.raises(tc.TCError) as e:
        tc.Server(1 << 20, slots=2, slot_edges=1 << 22, slot_vertices=1 << 20, slot_requests=64)
    assert e.value.status == tc.TC_ENOMEM  # the slots alone exceed the budget
    with tc.Server(1 << 30, slots=1, slot_edges=1000, slot_vertices=5000, slot_requests=8) as srv:
        with pytest.raises(tc.TCError) as e:
            srv.add_graph(gen.complete(60), 60)  # 1770 edges > slot_edges
        assert e.value.status == tc.TC_EINVAL
        with pytest.raises(tc.TCError) as e:
            srv.add_graph(np.array([[0, 1]], np.uint32), 6000)  # n > slot_vertices
        assert e.value.status == tc.TC_EINVAL
        with pytest.raises(tc.TCError) as e:
            srv.add_graph(np.array([[0, 9]], np.uint32), 5)  # endpoint >= n
        assert e.value.status == tc.TC_EINVAL
        gid = srv.add_graph(gen.complete(10), 10)
        for bad_p in (0.0, 1.5, float("nan")):
            with pytest.raises(tc.TCError):
                srv.submit(gid, bad_p, 1)
        with pytest.raises(tc.TCError):
            srv.submit(gid + 1, 0.5, 1)  # unknown graph
        with pytest.raises(tc.TCError):
            srv.poll(12345)  # unknown ticket
        t = srv.submit(gid, 1.0, 1)
        r = srv.wait(t)
        assert r["t_light"] + r["t_heavy"] == 120 and r["estimate"] == 120.0
        with pytest.raises(tc.TCError):
            srv.poll(t)  # released by wait
    with tc.Server(1 << 30, slots=1, slot_edges=1 << 16, slot_vertices=1 << 16, slot_requests=8) as probe:
        slot_bytes = probe.stats()["slot_bytes"]
    with tc.Server(slot_bytes + 2000, slots=1, slot_edges=1 << 16, slot_vertices=1 << 16, slot_requests=8) as srv:
        with pytest.raises(tc.TCError) as e:
            srv.add_graph(gen.complete(40), 40)  # 780 edges * 16 bytes > the 2000 left
        assert e.value.status == tc.TC_ENOMEM
        gid = srv.add_graph(gen.complete(12), 12)  # 66 edges * 16 bytes fit
        assert srv.wait(srv.submit(gid, 1.0, 3))["estimate"] == 220.0
