"""C-ABI entry points around the single count: a count on the caller's
stream (tc_count_async), one batched count over graphs that are already
resident (tc_count_batch), and allocation failure (tc_set_allocator ->
TC_ENOMEM, nothing left allocated).  Results are compared with tc_count and
with the oracle."""
import ctypes

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

KEYS = ("m", "m_sampled", "n_heavy", "t_light", "t_heavy", "estimate")


def _tc():
    from paper_1011_0468_gb300 import tc
    return tc


def test_count_async_on_a_callers_stream():
    import torch
    tc = _tc()
    e = gen.chung_lu(30000, 300000, 2.1, 3000.0, 12)
    own = torch.cuda.Stream()
    other = torch.cuda.Stream()
    ps = [(1.0, 1), (0.3, 5), (0.05, 9)]
    buf = torch.zeros((len(ps), ctypes.sizeof(tc.tc_result)), dtype=torch.uint8, pin_memory=True)
    with tc.Graph(e, 30000, stream=own) as g:
        for j, (p, seed) in enumerate(ps):
            g.count_async(p, seed, buf[j].data_ptr(), stream=other if j % 2 == 0 else None)
        g.sync()  # covers the counts enqueued on the other stream
        got = [tc.tc_result.from_address(buf[j].data_ptr()).as_dict() for j in range(len(ps))]
        for (p, seed), r in zip(ps, got):
            want = oracle.run(e, 30000, p, seed)
            assert all(r[k] == want[k] for k in KEYS), (p, seed)
            assert g.count(p, seed)["estimate"] == r["estimate"]
        # a count on a stream the caller synchronises itself
        out = torch.zeros(ctypes.sizeof(tc.tc_result), dtype=torch.uint8, pin_memory=True)
        g.count_async(0.5, 3, out.data_ptr(), stream=other)
        other.synchronize()
        r = tc.tc_result.from_address(out.data_ptr()).as_dict()
        want = oracle.run(e, 30000, 0.5, 3)
        assert all(r[k] == want[k] for k in KEYS)


def test_count_batch_over_resident_graphs():
    tc = _tc()
    graphs = [(gen.chung_lu(20000, 160000, 2.1, 2500.0, 3), 20000),
              (gen.er(5000, 40000, 4), 5000),
              (gen.complete(60), 60),
              (gen.wheel(9), 10),
              (gen.planted_core(60000, 1400, 0.85, 250000, 5), 60000),  # m >= 2^20: alone it uses the tensor cores
              (np.zeros((0, 2), np.uint32), 7)]
    objs = [tc.Graph(e, n) for e, n in graphs]
    try:
        # every graph once, the first two again with other (p, seed)
        sel = list(range(len(objs))) + [0, 1, 4]
        p = [1.0, 0.3, 1.0, 0.5, 1.0, 0.2, 0.1, 1.0, 0.6]
        seed = [1, 2, 3, 4, 5, 6, 7, 8, 9]
        res = tc.tc_count_batch([objs[i] for i in sel], p, seed)
        for j, i in enumerate(sel):
            single = objs[i].count(p[j], seed[j])
            for k in KEYS:
                assert res[k][j] == single[k], (j, i, k)
            # the graph with a heavy block of its own counts on its own path
            # (its work counters filled in; at p = 1 its heavy class runs on
            # the tensor cores); the union reports no work
            assert (res["partners"][j] > 0) == (i == 4), (j, i)
            if i == 4 and p[j] == 1.0:
                assert res["heavy_mma_flops"][j] > 0
            if i != 4:  # the planted core's oracle run takes a while; its single count is exact already
                want = oracle.run(graphs[i][0], graphs[i][1], p[j], seed[j])
                for k in KEYS:
                    assert res[k][j] == want[k], (j, i, k)
        # only graphs with a heavy block of their own: no union at all
        res = tc.tc_count_batch([objs[4], objs[4]], [1.0, 0.45], [11, 12])
        for j, (p1, s1) in enumerate(((1.0, 11), (0.45, 12))):
            single = objs[4].count(p1, s1)
            assert all(res[k][j] == single[k] for k in KEYS), j
        with pytest.raises(tc.TCError) as ei:
            tc.tc_count_batch([objs[0]], [1.5], [1])
        assert ei.value.status == tc.TC_EINVAL
    finally:
        for o in objs:
            o.close()


def test_allocation_failure_returns_enomem_and_leaks_nothing():
    """A caller's allocator that fails at its k-th call: graph creation
    returns TC_ENOMEM and has given back every block it got, for every k."""
    import torch
    tc = _tc()
    L = tc.lib()
    live = {}
    state = {"calls": 0, "fail_at": 0}

    def _alloc(nbytes, stream, ctx):
        state["calls"] += 1
        if state["calls"] == state["fail_at"]:
            return None
        p = torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                               int(stream) if stream else None)
        live[int(p)] = int(nbytes)
        return p

    def _free(ptr, stream, ctx):
        live.pop(int(ptr))
        torch.cuda.caching_allocator_delete(int(ptr))

    hooks = (tc._ALLOC_T(_alloc), tc._FREE_T(_free))
    e = gen.planted_core(60000, 1400, 0.85, 250000, 5)  # above 2^20 edges: heavy block buffers too
    L.tc_set_allocator(ctypes.cast(hooks[0], ctypes.c_void_p), ctypes.cast(hooks[1], ctypes.c_void_p), None)
    try:
        with tc.Graph(e, 60000) as g:  # count the allocations of a successful creation
            total = state["calls"]
            want = g.count(1.0, 1)
        assert total >= 10 and not live
        failed = 0
        for k in range(1, total + 1):
            state["calls"], state["fail_at"] = 0, k
            try:
                g = tc.Graph(e, 60000)
            except tc.TCError as ex:
                assert ex.status == tc.TC_ENOMEM, k
                failed += 1
            else:  # the optional dense blocks are dropped when their memory is refused
                got = g.count(1.0, 1)
                g.close()
                assert all(got[q] == want[q] for q in KEYS), k
            assert not live, (k, live)
        assert failed >= total // 2
        state["fail_at"] = 0
        with tc.Graph(e, 60000) as g:  # and the library still works
            got = g.count(1.0, 1)
        assert all(got[k] == want[k] for k in KEYS)
        assert not live
    finally:
        L.tc_set_allocator(None, None, None)


def test_partition_on_the_original_degrees():
    """tc_graph_set_partition(TC_PARTITION_ORIGINAL) splits the whole
    graph's vertices (deg^2 > m) and classifies the sampled triangles by
    those flags, as the oracle's partition="original" does; the estimate is
    the same as with the sampled partition."""
    tc = _tc()
    L = tc.lib()
    cases = [(gen.chung_lu(20000, 200000, 2.1, 3000.0, 3), 20000),
             (gen.planted_core(60000, 1400, 0.85, 250000, 5), 60000),  # dense heavy block on the tensor cores
             (gen.wheel(4), 5), (gen.wheel(7), 8)]
    for e, n in cases:
        with tc.Graph(e, n) as g:
            for p, seed in ((1.0, 1), (0.5, 2), (0.2, 3)):
                assert L.tc_graph_set_partition(g.handle, 1) == tc.TC_OK
                got = g.count(p, seed)
                want = oracle.run(e, n, p, seed, partition="original")
                assert all(got[k] == want[k] for k in KEYS), (n, p, seed)
                kept, heavy, _ = g.export_sample(p, seed, pairs=False)
                ref = oracle.run(e, n, p, seed, want_sample=True, partition="original")
                assert np.array_equal(heavy, ref["heavy"])
                assert L.tc_graph_set_partition(g.handle, 0) == tc.TC_OK
                plain = g.count(p, seed)
                assert plain["estimate"] == got["estimate"]
                assert plain["t_light"] + plain["t_heavy"] == got["t_light"] + got["t_heavy"]
            assert L.tc_graph_set_partition(g.handle, 2) == tc.TC_EINVAL


def test_sweep_adaptive_and_auto_counts():
    """tc_count_sweep gives each (p, seed) the oracle's result; the adaptive
    count picks the first p of the ladder p0 growth^i whose estimate is
    within tol of the previous one; the auto count runs the pilot and then
    the count at Section 3.3's p."""
    tc = _tc()
    e, n = gen.chung_lu(40000, 400000, 2.1, 4000.0, 8), 40000
    with tc.Graph(e, n) as g:
        ps = [0.02, 0.05, 0.1, 0.3, 1.0]
        res = g.count_sweep(ps, [3, 4, 5, 6, 7])
        for j, (p, seed) in enumerate(zip(ps, [3, 4, 5, 6, 7])):
            want = oracle.run(e, n, p, seed)
            assert all(res[k][j] == want[k] for k in KEYS), p
        for p0, growth, tol in ((0.01, 2.0, 0.05), (0.05, 1.5, 0.01), (0.2, 3.0, 0.0)):
            got, p_used, runs = g.count_adaptive(p0, growth, tol, 9)
            ladder, q = [], p0
            while True:
                ladder.append(min(q, 1.0))
                if q >= 1.0 or len(ladder) == 16:
                    break
                q *= growth
            ests = [oracle.run(e, n, q, 9)["estimate"] for q in ladder]
            pick = next((i for i in range(1, len(ladder)) if abs(ests[i] - ests[i - 1]) <= tol * abs(ests[i])),
                        len(ladder) - 1)
            assert runs == len(ladder) and p_used == ladder[pick]
            assert got["estimate"] == ests[pick]
        # equal to the single counts, also on a graph with a heavy block
        one = [g.count(p, s) for p, s in zip(ps, [3, 4, 5, 6, 7])]
        assert all(res[k][j] == one[j][k] for j in range(len(ps)) for k in KEYS)
        big = gen.planted_core(60000, 1400, 0.85, 250000, 5)
        with tc.Graph(big, 60000) as g2:
            res2 = g2.count_sweep([0.3, 1.0], [1, 2])
            for j, (p, s) in enumerate(((0.3, 1), (1.0, 2))):
                single = g2.count(p, s)
                assert all(res2[k][j] == single[k] for k in KEYS), (p, s)
        got, p_used = g.count_auto(0.1, 0.05, 12)
        pilot = oracle.run(e, n, 0.05, 12)
        assert p_used == oracle.suggest_p(len(e), n, pilot["estimate"], 0.1)
        want = oracle.run(e, n, p_used, 12)
        assert all(got[k] == want[k] for k in KEYS)


def test_schedules_and_strategies_give_identical_counts():
    """Every owner-bucket strategy (hash set, rank-window bitmap or binary
    search of the sorted row, per block kernel), both mid / large splits and
    the item sizes give the oracle's counts; tc_graph_autotune keeps a
    schedule that does too."""
    tc = _tc()
    e, n = gen.planted_core(40000, 2500, 0.9, 300000, 2), 40000  # owners above 1024 and below
    with tc.Graph(e, n) as g:
        want = {p: oracle.run(e, n, p, 5) for p in (1.0, 0.4)}
        for sched in (dict(lookup=1), dict(lookup=2), dict(lookup=3), dict(lookup=4), dict(lookup=8),
                      dict(lookup=12), dict(lookup=13), dict(lookup=14), dict(mid_max=512),
                      dict(mid_max=512, lookup=12, warp_max=32), dict(mid_max=512, lookup=3, warp_max=64),
                      dict(seg_l=1024, seg_b=256, seg_w=256)):
            g.set_schedule()
            g.set_schedule(**sched)
            for p in (1.0, 0.4):
                got = g.count(p, 5)
                assert all(got[k] == want[p][k] for k in KEYS), (sched, p)
        # no large owner's window can exceed its table here (2500 vertices of
        # degree > 512): the default takes the bitmaps for those owners
        g.set_schedule()
        assert g.schedule()["lookup"] == 8
        desc = g.autotune(1.0, 5)
        assert "warp per owner" in desc and any(w in desc for w in ("hash set", "bitmap", "binary search"))
        got = g.count(0.4, 5)
        assert all(got[k] == want[0.4][k] for k in KEYS)
        s = g.schedule()
        assert 512 <= s["mid_max"] <= 1024 and s["lookup"] <= 15
        with pytest.raises(tc.TCError):
            g.set_schedule(mid_max=256)
        with pytest.raises(tc.TCError):
            g.set_schedule(lookup=16)


def test_bitmap_window_too_wide_falls_back_to_the_hash_set():
    """Owners whose rank window (owner to largest out-neighbour) exceeds the
    mid-owner table's 131072 bits take the hash set, the others the bitmap.
    140,000 filler vertices on a circulant graph (i ~ i + 1 .. i + 21, degree
    42 and up), 50 hubs joined to 20,000 fillers each, and 200 owners of
    degree 40 (38 fillers and 2 hubs): every owner's neighbours rank above
    it, so with warp_max = 32 it is a mid owner whose window reaches a hub
    about 140,000 ranks up.  Counts equal the oracle's under the hash sets
    and under the bitmaps."""
    tc = _tc()
    rng = np.random.default_rng(21)
    nf, nh, no = 140000, 50, 200
    f0, h0 = no, no + nf  # ids: owners, fillers, hubs
    i = np.arange(nf)
    circ = np.stack([np.repeat(i, 21), (np.repeat(i, 21) + np.tile(np.arange(1, 22), nf)) % nf], axis=1) + f0
    hub = np.stack([np.repeat(np.arange(nh), 20000) + h0, rng.integers(0, nf, nh * 20000) + f0], axis=1)
    own = np.stack([np.repeat(np.arange(no), 40),
                    np.concatenate([np.concatenate([rng.choice(nf, 38, replace=False) + f0,
                                                    rng.choice(nh, 2, replace=False) + h0]) for _ in range(no)])],
                   axis=1)
    e, n = gen.canonical(np.concatenate([circ, hub, own])), no + nf + nh
    with tc.Graph(e, n) as g:
        for p in (1.0, 0.7):
            want = oracle.run(e, n, p, 3)
            assert want["t_light"] > 0
            for lookup in (0, 12):
                g.set_schedule(warp_max=32, mid_max=1024, lookup=lookup)
                got = g.count(p, 3)
                assert all(got[k] == want[k] for k in KEYS), (p, lookup)
