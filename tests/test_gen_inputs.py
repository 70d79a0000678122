"""The input generators that both the oracle and the CUDA library consume.

The largest graph reaches the library as raw R-MAT draws (gen.rmat_draws,
filled by several threads) while the oracle's expected values are computed
on gen.rmat's host-deduplicated graph; the two must describe the same graph,
whatever the thread count.
"""
import numpy as np
import pytest

import gen


def _canonical(draws: np.ndarray) -> np.ndarray:
    u = np.minimum(draws[:, 0], draws[:, 1]).astype(np.uint64)
    v = np.maximum(draws[:, 0], draws[:, 1]).astype(np.uint64)
    keys = np.unique((u << np.uint64(32) | v)[u != v])
    return np.stack([(keys >> np.uint64(32)).astype(np.uint32), (keys & np.uint64(0xFFFFFFFF)).astype(np.uint32)], 1)


@pytest.mark.parametrize("scale,edge_factor,seed", [(8, 16, 1), (12, 8, 5), (14, 16, 3)])
def test_rmat_draws_canonicalise_to_rmat(scale, edge_factor, seed):
    draws = gen.rmat_draws(scale, edge_factor, seed=seed)
    assert draws.shape == (edge_factor << scale, 2) and draws.dtype == np.uint32
    assert int(draws.max()) < (1 << scale)
    assert np.array_equal(_canonical(draws), gen.rmat(scale, edge_factor, seed=seed))


def test_rmat_draws_do_not_depend_on_threads():
    one = gen.rmat_draws(13, 16, seed=2, threads=1)
    many = gen.rmat_draws(13, 16, seed=2, threads=7)
    assert np.array_equal(one, many)


def test_rmat_draws_fill_a_given_buffer():
    out = np.zeros((8 << 10, 2), dtype=np.uint32)
    got = gen.rmat_draws(10, 8, seed=4, out=out)
    assert got is out and np.array_equal(out, gen.rmat_draws(10, 8, seed=4))


def test_rmat_is_canonical():
    e = gen.rmat(12, 16, seed=9)
    assert (e[:, 0] < e[:, 1]).all()
    k = e[:, 0].astype(np.uint64) << np.uint64(32) | e[:, 1]
    assert (np.diff(k.astype(np.int64)) > 0).all()  # sorted, no repeats
