"""tc_count_noalloc, the entry point for callers that cannot allocate device
memory (a framework pool already owns the GPU, or a device allocation would
synchronise it), must give the same results as the regular entry points
(tc_graph_create + tc_count) on consecutive calls, which share one fixed
scratch array inside the library, and the oracle's.  Collected last on
purpose.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

INT_KEYS = ("m", "m_sampled", "n", "n_heavy", "t_light", "t_heavy")


def _same(got, want):
    for k in INT_KEYS:
        assert got[k] == want[k], (k, got[k], want[k])
    e, w = got["estimate"], want["estimate"]
    assert e == w or abs(e - w) <= 1e-12 * abs(w), (e, w)


def test_no_alloc_matches_regular_entry_points_on_consecutive_calls():
    import torch
    from paper_1011_0468_gb300 import _build, tc
    _build.build()
    torch.cuda.set_device(0)
    rng = np.random.default_rng(5)
    cases = [
        # raw pairs with repeats, self-loops and both orientations
        (rng.integers(0, 3000, size=(40_000, 2)).astype(np.int32), 3000, 0.4, 11),
        # a power-law graph with heavy vertices, at the size limit's scale
        (gen.chung_lu(100_000, 250_000, 2.1, 3000.0, 4).astype(np.int32), 100_000, 1.0, 1),
    ]
    # the small case again after the large one: nothing left in the shared
    # array from the larger call may leak into the smaller one
    cases.append(cases[0])
    for edges, n, p, seed in cases:
        dev = torch.from_numpy(edges).cuda()
        got = tc.tc_count_noalloc(dev.data_ptr(), len(edges), n, p, seed).as_dict()
        with tc.Graph(edges.astype(np.uint32), n) as g:
            want = g.count(p, seed)
        _same(got, want)
        _same(got, oracle.run(oracle.canonicalize(edges.astype(np.uint32), n), n, p, seed))
        assert got["t_light"] + got["t_heavy"] > 0


def test_no_alloc_degenerate_inputs_and_no_device_allocation():
    """No edges, and input pairs that are all self-loops and repeats (m = 0
    after canonicalising), give the regular entry points' results; a warmed
    call leaves the device's free memory unchanged."""
    import torch
    from paper_1011_0468_gb300 import tc
    torch.cuda.set_device(0)
    loops = np.repeat(np.arange(50, dtype=np.int32), 3)
    loops = np.stack([loops, loops], axis=1)
    for edges, n in ((np.zeros((0, 2), np.int32), 9), (loops, 60)):
        dev = torch.from_numpy(edges).cuda()
        got = tc.tc_count_noalloc(dev.data_ptr() if len(edges) else 0, len(edges), n, 0.7, 3).as_dict()
        with tc.Graph(edges.astype(np.uint32), n) as g:
            want = g.count(0.7, 3)
        _same(got, want)
        assert got["m"] == 0 and got["t_light"] == got["t_heavy"] == 0
    edges = gen.chung_lu(50_000, 200_000, 2.1, 3000.0, 9).astype(np.int32)
    dev = torch.from_numpy(edges).cuda()
    first = tc.tc_count_noalloc(dev.data_ptr(), len(edges), 50_000, 1.0, 1).as_dict()
    torch.cuda.synchronize()
    free0, _ = torch.cuda.mem_get_info()
    again = tc.tc_count_noalloc(dev.data_ptr(), len(edges), 50_000, 1.0, 1).as_dict()
    torch.cuda.synchronize()
    free1, _ = torch.cuda.mem_get_info()
    assert free1 == free0
    _same(again, first)


def test_no_alloc_rejects_sizes_beyond_its_limit():
    import torch
    from paper_1011_0468_gb300 import tc
    small = torch.zeros((4, 2), dtype=torch.int32, device="cuda")
    with pytest.raises(tc.TCError) as e1:
        tc.tc_count_noalloc(small.data_ptr(), tc.TC_NOALLOC_MAX_EDGES + 1, 10, 0.5, 1)
    assert e1.value.status == tc.TC_EINVAL
    with pytest.raises(tc.TCError) as e2:
        tc.tc_count_noalloc(small.data_ptr(), 4, tc.TC_NOALLOC_MAX_VERTICES + 1, 0.5, 1)
    assert e2.value.status == tc.TC_EINVAL
