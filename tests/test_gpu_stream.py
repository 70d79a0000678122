"""The semi-streaming count (tc_stream_count, Section 5.2) against the
oracle, field by field: the heavy vertices found from sampled entries, |U|,
the samples' closed wedges and pairs (bit-exact) and the estimate (==).
The stream is read both in place (pinned, mapped) and copied in chunks of
many sizes, including chunks that cut lists and a last chunk of one entry."""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

KEYS = ("m", "n", "n_heavy", "candidates", "sampled_entries", "universe", "samples", "closed_wedge", "closed_pair",
        "estimate")


def _tc():
    from paper_1011_0468_gb300 import tc
    return tc


def check(off, adj, n, seed, s, c, chunk, pinned=False):
    import torch
    tc = _tc()
    if pinned:
        o = torch.from_numpy(off.view(np.int64)).pin_memory()
        a = torch.from_numpy(adj.view(np.int32)).pin_memory()
        got = tc.tc_stream_count(o, a, n, seed, s, c, chunk)
    else:
        got = tc.tc_stream_count(off, adj, n, seed, s, c, chunk)
    want = oracle.stream_triples(off, adj, n, seed, s, c)
    for k in KEYS:
        assert got[k] == want[k], (k, seed, s, c, chunk, pinned, got[k], want[k])
    assert got["passes"] == (3 if want["universe"] and want["samples"] else 1)
    return got


@pytest.mark.parametrize("name,make", [
    ("chung_lu", lambda: (gen.chung_lu(20000, 200000, 2.1, 3000.0, 3), 20000)),
    ("er", lambda: (gen.er(3000, 30000, 2), 3000)),
    ("planted_core", lambda: (gen.planted_core(20000, 500, 0.8, 80000, 4), 20000)),
    ("rmat15", lambda: (gen.rmat(15, 16, seed=3), 1 << 15)),
])
def test_stream_matches_the_oracle(name, make):
    e, n = make()
    off, adj = gen.adjacency_stream(e, n)
    len_ = len(adj)
    for seed, s, c, chunk in ((1, 0, 3.0, 0), (2, 100000, 3.0, 4099), (3, 50000, 1.0, len_ - 1), (4, 7, 3.0, 1 << 16),
                              (5, 30000, 1e12, 100003)):
        check(off, adj, n, seed, s, c, chunk)
    r = check(off, adj, n, 6, 200000, 3.0, 65536, pinned=True)
    t = oracle.run(e, n, 1.0, 1)["estimate"]
    assert abs(r["estimate"] - t) <= 0.2 * t


def test_stream_degenerate_inputs():
    tc = _tc()
    for e, n in ((np.zeros((0, 2), np.uint32), 5), (gen.star(30), 31), (gen.complete(40), 40),
                 (gen.disjoint_union(*[gen.complete(4)] * 30)[0], 120)):
        off, adj = gen.adjacency_stream(e, n)
        for chunk in (0, 3):
            check(off, adj, n, 2, 500, 3.0, chunk)
    # not a sorted symmetric simple adjacency: rejected
    e = gen.er(100, 400, 1)
    off, adj = gen.adjacency_stream(e, 100)
    bad = adj.copy()
    bad[[0, 1]] = bad[[1, 0]]  # a list out of order
    with pytest.raises(tc.TCError) as ei:
        tc.tc_stream_count(off, bad, 100, 1, 10)
    assert ei.value.status == tc.TC_EINVAL
    bad = adj.copy()
    bad[off[3]] = 3  # a self-loop
    with pytest.raises(tc.TCError):
        tc.tc_stream_count(off, bad, 100, 1, 10)
    one_way = np.concatenate([[0], np.cumsum(np.bincount(e[:, 0], minlength=100))]).astype(np.uint64)
    with pytest.raises(tc.TCError):  # each edge in one list only
        tc.tc_stream_count(one_way, e[:, 1].copy(), 100, 1, 10)
