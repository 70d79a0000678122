"""CPU oracle for the edge-sampled, degree-partitioned triangle counter.

TEST INFRASTRUCTURE ONLY.  This package is the plain, slow, single-threaded
statement of what the method computes (``oracle.c``, one thread, no
blocking, fusion or reordering).  Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it.  The CUDA library
(``paper_1011_0468_gb300``) never imports, links or calls anything here, and
the two share no code; they meet only at the seeded input generators in
``gen/``.

Functions and the paper passages they follow:

* ``splitmix64`` / ``keep`` / ``sample`` -- Section 3.1, edge sparsification
  (keep each edge independently with probability p), with a counter-based
  hash as the random draw so that any implementation draws the same set.
* ``canonicalize`` -- Section 4.1, simple graphs: no self-loops, no repeats.
* ``degrees`` / ``partition`` -- Section 3.2, low degree deg <= m^(1/2),
  high degree deg > m^(1/2), on the sampled graph, in integers (deg^2 > m).
* ``count_classes`` -- Section 3.2, triangles with at least one low-degree
  vertex (T_L) and with three high-degree vertices (T_H), by plain sorted
  neighbour-list merging over vertex ids.
* ``estimate`` -- Section 3.1, T_L / p^3 + T_H / p^3 in float64.

Parity is pinned in ``tests/test_oracle_*.py`` (brute force, closed forms,
published splitmix64 outputs, the exact variance of the estimator).
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)


class OracleResult(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("m_sampled", ctypes.c_uint64), ("n", ctypes.c_uint32),
                ("n_heavy", ctypes.c_uint32), ("t_light", ctypes.c_uint64),
                ("t_heavy", ctypes.c_uint64), ("estimate", ctypes.c_double)]


class StreamResult(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("n", ctypes.c_uint32), ("n_heavy", ctypes.c_uint32),
                ("candidates", ctypes.c_uint64), ("sampled_entries", ctypes.c_uint64), ("universe", ctypes.c_uint64),
                ("samples", ctypes.c_uint64), ("closed_wedge", ctypes.c_uint64), ("closed_pair", ctypes.c_uint64),
                ("estimate", ctypes.c_double)]


class TripleResult(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("m_sampled", ctypes.c_uint64), ("n", ctypes.c_uint32),
                ("n_heavy", ctypes.c_uint32), ("universe", ctypes.c_uint64), ("samples", ctypes.c_uint64),
                ("closed_wedge", ctypes.c_uint64), ("closed_path", ctypes.c_uint64), ("estimate", ctypes.c_double)]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (plain C, one thread)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=gnu11", _SRC, "-o", tmp,
                               "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        lib.oracle_splitmix64.argtypes = [ctypes.c_uint64]
        lib.oracle_splitmix64.restype = ctypes.c_uint64
        lib.oracle_threshold.argtypes = [ctypes.c_double]
        lib.oracle_threshold.restype = ctypes.c_uint64
        lib.oracle_keep.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64]
        lib.oracle_keep.restype = ctypes.c_int
        lib.oracle_canonicalize.argtypes = [_u32p, ctypes.c_uint64, ctypes.c_uint32, _u32p]
        lib.oracle_canonicalize.restype = ctypes.c_int64
        lib.oracle_sample.argtypes = [_u32p, ctypes.c_uint64, ctypes.c_double, ctypes.c_uint64, _u32p]
        lib.oracle_sample.restype = ctypes.c_uint64
        lib.oracle_degrees.argtypes = [_u32p, ctypes.c_uint64, ctypes.c_uint32, _u32p]
        lib.oracle_degrees.restype = None
        lib.oracle_partition.argtypes = [_u32p, ctypes.c_uint32, ctypes.c_uint64, _u8p]
        lib.oracle_partition.restype = ctypes.c_uint32
        lib.oracle_count_classes.argtypes = [_u32p, ctypes.c_uint64, ctypes.c_uint32, _u8p, _u64p, _u64p]
        lib.oracle_count_classes.restype = ctypes.c_int
        lib.oracle_adjacency.argtypes = [_u32p, ctypes.c_uint64, ctypes.c_uint32, _u64p, _u32p]
        lib.oracle_adjacency.restype = ctypes.c_int
        lib.oracle_count_range.argtypes = [_u64p, _u32p, _u8p, ctypes.c_uint32, ctypes.c_uint32, _u64p, _u64p]
        lib.oracle_count_range.restype = None
        lib.oracle_estimate.argtypes = [ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double]
        lib.oracle_estimate.restype = ctypes.c_double
        lib.oracle_run.argtypes = [_u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                   ctypes.c_uint64, _u32p, _u8p, ctypes.POINTER(OracleResult)]
        lib.oracle_run.restype = ctypes.c_int
        lib.oracle_run_partition.argtypes = [_u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double,
                                             ctypes.c_uint64, ctypes.c_int, _u32p, _u8p, ctypes.POINTER(OracleResult)]
        lib.oracle_run_partition.restype = ctypes.c_int
        lib.oracle_suggest_p.argtypes = [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_double]
        lib.oracle_suggest_p.restype = ctypes.c_double
        lib.oracle_triples.argtypes = [_u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64,
                                       ctypes.c_uint64, ctypes.c_int, ctypes.POINTER(TripleResult)]
        lib.oracle_triples.restype = ctypes.c_int
        lib.oracle_triple_enumerate.argtypes = [_u32p, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int,
                                                ctypes.c_uint64, _u32p, _u32p, _u32p, _u8p]
        lib.oracle_triple_enumerate.restype = ctypes.c_int64
        lib.oracle_stream_triples.argtypes = [_u64p, _u32p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64,
                                              ctypes.c_double, ctypes.POINTER(StreamResult)]
        lib.oracle_stream_triples.restype = ctypes.c_int
        _lib = lib
    return _lib


def _pairs(edges) -> np.ndarray:
    a = np.ascontiguousarray(np.asarray(edges, dtype=np.uint32).reshape(-1, 2))
    return a


def splitmix64(x: int) -> int:
    """splitmix64 (Steele, Lea, Flood; Vigna's published form) of a 64-bit word."""
    return int(_load().oracle_splitmix64(x & 0xFFFFFFFFFFFFFFFF))


def threshold(p: float) -> int:
    """floor(p * 2^53), the acceptance threshold of the keep test."""
    return int(_load().oracle_threshold(p))


def keep(u: int, v: int, seed: int, p: float) -> bool:
    """Section 3.1 keep decision for the canonical edge (u, v), u < v."""
    return bool(_load().oracle_keep(u, v, seed & 0xFFFFFFFFFFFFFFFF, threshold(p)))


def canonicalize(edges, n: int) -> np.ndarray:
    """Simple-graph form: (min, max) pairs, no self-loops, sorted, unique."""
    a = _pairs(edges)
    out = np.empty((max(len(a), 1), 2), dtype=np.uint32)
    r = _load().oracle_canonicalize(a.ctypes.data_as(_u32p), len(a), n, out.ctypes.data_as(_u32p))
    if r == -1:
        raise ValueError("endpoint >= n")
    if r < 0:
        raise MemoryError("oracle_canonicalize")
    return out[:r]


def sample(canon, p: float, seed: int) -> np.ndarray:
    """Section 3.1: the kept edges, in input order."""
    a = _pairs(canon)
    out = np.empty((max(len(a), 1), 2), dtype=np.uint32)
    r = _load().oracle_sample(a.ctypes.data_as(_u32p), len(a), p, seed & 0xFFFFFFFFFFFFFFFF,
                              out.ctypes.data_as(_u32p))
    return out[:r]


def degrees(edges, n: int) -> np.ndarray:
    a = _pairs(edges)
    deg = np.zeros(max(n, 1), dtype=np.uint32)
    _load().oracle_degrees(a.ctypes.data_as(_u32p), len(a), n, deg.ctypes.data_as(_u32p))
    return deg[:n]


def partition_flags(deg: np.ndarray, m: int) -> np.ndarray:
    """Section 3.2: heavy flags, deg^2 > m, as uint8."""
    d = np.ascontiguousarray(deg, dtype=np.uint32)
    heavy = np.zeros(max(len(d), 1), dtype=np.uint8)
    _load().oracle_partition(d.ctypes.data_as(_u32p), len(d), m, heavy.ctypes.data_as(_u8p))
    return heavy[:len(d)]


partition = partition_flags  # Section 3.2 partition (name kept for existing callers)


def count_classes(edges, n: int, heavy: np.ndarray, threads: int = 1) -> tuple[int, int]:
    """Section 3.2: (T_L, T_H) of the given simple graph under the given flags.

    With threads > 1 the same enumeration runs over disjoint ranges of the
    smallest vertex u on several host threads (ctypes releases the GIL during
    each call), and the per-range counts are summed: every triangle is seen
    once, at its smallest vertex, so the result does not depend on the split.
    Only the golden-value script uses this, for graphs whose single-threaded
    count takes hours."""
    a = _pairs(edges)
    h = np.ascontiguousarray(heavy, dtype=np.uint8)
    if len(h) < max(n, 1):
        h = np.concatenate([h, np.zeros(max(n, 1) - len(h), dtype=np.uint8)])
    tl, th = ctypes.c_uint64(0), ctypes.c_uint64(0)
    if threads <= 1:
        rc = _load().oracle_count_classes(a.ctypes.data_as(_u32p), len(a), n, h.ctypes.data_as(_u8p),
                                          ctypes.byref(tl), ctypes.byref(th))
        if rc:
            raise MemoryError("oracle_count_classes")
        return int(tl.value), int(th.value)
    from concurrent.futures import ThreadPoolExecutor
    start = np.empty(n + 1, dtype=np.uint64)
    adj = np.empty(max(2 * len(a), 1), dtype=np.uint32)
    lib = _load()
    if lib.oracle_adjacency(a.ctypes.data_as(_u32p), len(a), n, start.ctypes.data_as(_u64p),
                            adj.ctypes.data_as(_u32p)):
        raise MemoryError("oracle_adjacency")
    step = max(1, min(1024, n // (64 * threads) or 1))
    ranges = [(lo, min(n, lo + step)) for lo in range(0, n, step)]

    def one(r):
        x, y = ctypes.c_uint64(0), ctypes.c_uint64(0)
        lib.oracle_count_range(start.ctypes.data_as(_u64p), adj.ctypes.data_as(_u32p), h.ctypes.data_as(_u8p),
                               r[0], r[1], ctypes.byref(x), ctypes.byref(y))
        return int(x.value), int(y.value)

    with ThreadPoolExecutor(threads) as ex:
        parts = list(ex.map(one, ranges))
    return sum(p[0] for p in parts), sum(p[1] for p in parts)


def estimate(t_light: int, t_heavy: int, p: float) -> float:
    """Section 3.1: T_L / p^3 + T_H / p^3 in float64."""
    return float(_load().oracle_estimate(t_light, t_heavy, p))


def run(canon, n: int, p: float, seed: int, want_sample: bool = False, threads: int = 1,
        partition: str = "sampled") -> dict:
    """The whole method on a canonical edge list.  Returns m, m_sampled, n,
    n_heavy, t_light, t_heavy, estimate, and with want_sample the kept edges
    and heavy flags.  threads > 1 runs the same steps with the triangle
    enumeration split over host threads (``count_classes``).  partition:
    "sampled" (deg_p^2 > m_p, the default) or "original" (deg^2 > m of the
    whole graph) for the degree partition of Section 3.2."""
    if partition not in ("sampled", "original"):
        raise ValueError("partition must be 'sampled' or 'original'")
    orig = partition == "original"
    a = _pairs(canon)
    if threads > 1:
        if not (p > 0.0 and p <= 1.0):
            raise ValueError("p must lie in (0, 1]")
        kept = sample(a, p, seed)
        if orig:
            heavy = partition_flags(degrees(a, n), len(a))
        else:
            heavy = partition_flags(degrees(kept, n), len(kept))
        tl, th = count_classes(kept, n, heavy, threads=threads)
        out = {"m": len(a), "m_sampled": len(kept), "n": n, "n_heavy": int(heavy.sum()),
               "t_light": tl, "t_heavy": th, "estimate": estimate(tl, th, p)}
        if want_sample:
            out["kept"], out["heavy"] = kept, heavy
        return out
    res = OracleResult()
    kept = np.empty((max(len(a), 1), 2), dtype=np.uint32) if want_sample else None
    heavy = np.empty(max(n, 1), dtype=np.uint8) if want_sample else None
    rc = _load().oracle_run_partition(a.ctypes.data_as(_u32p), len(a), n, p, seed & 0xFFFFFFFFFFFFFFFF, int(orig),
                                      kept.ctypes.data_as(_u32p) if want_sample else None,
                                      heavy.ctypes.data_as(_u8p) if want_sample else None, ctypes.byref(res))
    if rc == -1:
        raise ValueError("p must lie in (0, 1]")
    if rc:
        raise MemoryError("oracle_run")
    out = {k: getattr(res, k) for k, _ in OracleResult._fields_}
    if want_sample:
        out["kept"] = kept[:res.m_sampled]
        out["heavy"] = heavy[:n]
    return out


def suggest_p(m: int, n: int, t: float, eps: float) -> float:
    """Section 3.3: p = (m^(1/2) ln n / (t eps^2))^(2/5), at most 1; 1 when
    t <= 0; raises for eps <= 0, m == 0 or n < 2."""
    r = float(_load().oracle_suggest_p(m, n, t, eps))
    if r < 0:
        raise ValueError("suggest_p: eps must be > 0, m > 0 and n >= 2")
    return r


def triples(canon, n: int, p: float, seed: int, samples: int = 0, mode: str = "hybrid") -> dict:
    """Triple sampling (Section 3.2) on the sample of Section 3.1 (the
    hybrid of Section 3.3 when p < 1): m, m_sampled, n, n_heavy, universe
    (|U|), samples, closed_wedge, closed_path, estimate.  mode "simple"
    (every vertex contributes its wedges) or "hybrid" (heavy vertices
    contribute 2-paths); samples = 0 draws m_p samples."""
    if mode not in ("simple", "hybrid"):
        raise ValueError("mode must be 'simple' or 'hybrid'")
    a = _pairs(canon)
    res = TripleResult()
    rc = _load().oracle_triples(a.ctypes.data_as(_u32p), len(a), n, p, seed & 0xFFFFFFFFFFFFFFFF, int(samples),
                                int(mode == "hybrid"), ctypes.byref(res))
    if rc == -1:
        raise ValueError("p must lie in (0, 1]")
    if rc:
        raise MemoryError("oracle_triples")
    return {k: getattr(res, k) for k, _ in TripleResult._fields_}


def triple_enumerate(canon, n: int, mode: str = "hybrid"):
    """Every triple of U of the whole graph in index order: arrays u, v, w,
    closed (tests on small graphs)."""
    a = _pairs(canon)
    lib = _load()
    hyb = int(mode == "hybrid")
    size = lib.oracle_triple_enumerate(a.ctypes.data_as(_u32p), len(a), n, hyb, 0, None, None, None, None)
    if size < 0:
        raise MemoryError("oracle_triple_enumerate")
    u, v, w = (np.zeros(max(size, 1), dtype=np.uint32) for _ in range(3))
    c = np.zeros(max(size, 1), dtype=np.uint8)
    if size:
        r = lib.oracle_triple_enumerate(a.ctypes.data_as(_u32p), len(a), n, hyb, size, u.ctypes.data_as(_u32p),
                                        v.ctypes.data_as(_u32p), w.ctypes.data_as(_u32p), c.ctypes.data_as(_u8p))
        if r != size:
            raise MemoryError("oracle_triple_enumerate")
    return u[:size], v[:size], w[:size], c[:size]


def stream_triples(off, adj, n: int, seed: int, samples: int = 0, c: float = 3.0) -> dict:
    """Section 5.2, three passes over a symmetric adjacency stream (off[n+1]
    uint64, adj[2m] uint32, lists sorted): heavy candidates from sampled
    entries, then s uniform triples of U (wedges of the other vertices,
    pairs of an edge and a heavy vertex), then the check of their third
    edges.  Returns m, n, n_heavy, candidates, sampled_entries, universe,
    samples, closed_wedge, closed_pair, estimate."""
    o = np.ascontiguousarray(off, dtype=np.uint64)
    a = np.ascontiguousarray(adj, dtype=np.uint32)
    if len(o) != n + 1 or (len(a) and int(o[-1]) != len(a)):
        raise ValueError("off must hold n + 1 offsets ending at len(adj)")
    if len(a) == 0:
        a = np.zeros(1, dtype=np.uint32)
    res = StreamResult()
    rc = _load().oracle_stream_triples(o.ctypes.data_as(_u64p), a.ctypes.data_as(_u32p), n,
                                       seed & 0xFFFFFFFFFFFFFFFF, int(samples), float(c), ctypes.byref(res))
    if rc:
        raise MemoryError("oracle_stream_triples")
    return {k: getattr(res, k) for k, _ in StreamResult._fields_}
