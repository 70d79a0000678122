"""Seeded synthetic graph generators (input data only).

The paper evaluates on twelve real social and web graphs (Table 1), which are
not available here.  These generators produce seeded stand-ins of the same
shape: Erdos-Renyi G(n, m), Chung-Lu power-law graphs and R-MAT graphs (in C,
``gen.c``), plus small closed-form graphs whose triangle counts are known
(complete graphs, wheels, stars, trees, cycles, complete bipartite graphs).

Every function returns a canonical edge list: a ``(m, 2)`` uint32 numpy array
of pairs ``(u, v)`` with ``u < v``, sorted, without duplicates or self-loops;
the one exception, ``rmat_draws``, returns the raw draws of an R-MAT graph
(whose canonical form is ``rmat``'s output) for inputs too large to
deduplicate quickly on the host.
Nothing here counts triangles or samples edges for the method; the outputs
are inputs to both the CPU oracle and the CUDA library.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "gen.c")
_LIB = os.path.join(_HERE, "libgen.so")
_lib = None


def build(force: bool = False) -> str:
    """Compile gen.c into libgen.so next to it (plain C, no GPU)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-ffp-contract=off", "-fPIC", "-shared", "-std=c11", _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        u32p = ctypes.POINTER(ctypes.c_uint32)
        lib.gen_er.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, u32p]
        lib.gen_er.restype = ctypes.c_int64
        lib.gen_chung_lu.argtypes = [ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double,
                                     ctypes.c_double, ctypes.c_uint64, u32p]
        lib.gen_chung_lu.restype = ctypes.c_int64
        lib.gen_rmat.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                 ctypes.c_double, ctypes.c_uint64, u32p]
        lib.gen_rmat.restype = ctypes.c_int64
        lib.gen_rmat_perm.argtypes = [ctypes.c_uint32, ctypes.c_uint64, u32p]
        lib.gen_rmat_perm.restype = ctypes.c_int
        lib.gen_rmat_draws.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                       ctypes.c_uint64, u32p, ctypes.c_uint64, ctypes.c_uint64, u32p]
        lib.gen_rmat_draws.restype = ctypes.c_int
        lib.gen_planted_core.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint64, u32p]
        lib.gen_planted_core.restype = ctypes.c_int64
        _lib = lib
    return _lib


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def er(n: int, m: int, seed: int) -> np.ndarray:
    """Erdos-Renyi G(n, m): m distinct uniform edges among n vertices."""
    out = np.empty((max(m, 1), 2), dtype=np.uint32)
    r = _load().gen_er(n, m, seed, _ptr(out))
    if r < 0:
        raise ValueError("gen_er failed (%d) for n=%d m=%d" % (r, n, m))
    return out[:r]


def chung_lu(n: int, m: int, gamma: float, wmax: float, seed: int) -> np.ndarray:
    """Chung-Lu power-law graph with exactly m distinct edges, degree exponent
    gamma and maximum expected degree wmax, vertex ids seeded-permuted."""
    out = np.empty((max(m, 1), 2), dtype=np.uint32)
    r = _load().gen_chung_lu(n, m, gamma, wmax, seed, _ptr(out))
    if r < 0:
        raise ValueError("gen_chung_lu failed (%d)" % r)
    return out[:r]


def rmat(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1) -> np.ndarray:
    """R-MAT graph on 2**scale vertices from edge_factor * 2**scale draws,
    symmetrised and deduplicated (the returned m is smaller than the draws)."""
    draws = edge_factor << scale
    out = np.empty((max(draws, 1), 2), dtype=np.uint32)
    r = _load().gen_rmat(scale, edge_factor, a, b, c, seed, _ptr(out))
    if r < 0:
        raise ValueError("gen_rmat failed (%d)" % r)
    return np.ascontiguousarray(out[:r])


def rmat_draws(scale: int, edge_factor: int, a: float = 0.57, b: float = 0.19, c: float = 0.19,
               seed: int = 1, out: np.ndarray | None = None, threads: int | None = None,
               count: int | None = None) -> np.ndarray:
    """The edge_factor * 2**scale raw draws of rmat(scale, edge_factor, a, b,
    c, seed) as (u, v) pairs in draw order, ids permuted, self-loops and
    repeats included: symmetrising and deduplicating them gives rmat's graph.
    Filled by several threads (each draw depends only on its index); out, if
    given, is a (draws, 2) uint32 array (e.g. in pinned memory).  count, if
    given, stops after the first `count` draws (the same draws as the first
    rows of the full output)."""
    from concurrent.futures import ThreadPoolExecutor
    draws = edge_factor << scale
    if count is not None:
        draws = min(draws, int(count))
    if out is None:
        out = np.empty((draws, 2), dtype=np.uint32)
    assert out.shape == (draws, 2) and out.dtype == np.uint32 and out.flags.c_contiguous
    lib = _load()
    perm = np.empty(1 << scale, dtype=np.uint32)
    if lib.gen_rmat_perm(scale, seed, _ptr(perm)) != 0:
        raise ValueError("gen_rmat_perm failed")
    threads = threads or max(1, min(64, os.cpu_count() or 1))
    step = -(-draws // (4 * threads))

    def fill(e0):
        e1 = min(draws, e0 + step)
        sub = out[e0:e1]
        return lib.gen_rmat_draws(scale, a, b, c, seed, _ptr(perm), e0, e1, _ptr(sub))

    with ThreadPoolExecutor(threads) as ex:
        if any(r != 0 for r in ex.map(fill, range(0, draws, step))):
            raise ValueError("gen_rmat_draws failed")
    return out


def planted_core(n: int, core: int, q: float, m_rest: int, seed: int) -> np.ndarray:
    """A dense core (core vertices, pair density q) inside a sparse uniform
    graph of m_rest edges on n vertices, ids scrambled.  Core vertices are
    heavy (degree above m^(1/2)) when q is well above 1/2."""
    cap = core * (core - 1) // 2 + m_rest
    out = np.empty((max(cap, 1), 2), dtype=np.uint32)
    r = _load().gen_planted_core(n, core, q, m_rest, seed, _ptr(out))
    if r < 0:
        raise ValueError("gen_planted_core failed (%d)" % r)
    return np.ascontiguousarray(out[:r])


def cached(kind: str, fn, *args) -> np.ndarray:
    """fn(*args), memoised as an .npy file under $TC_GEN_CACHE (default
    /tmp/tc_gen_cache) keyed by the generator and its arguments."""
    d = os.environ.get("TC_GEN_CACHE", "/tmp/tc_gen_cache")
    import hashlib
    with open(_SRC, "rb") as f:
        src_hash = hashlib.sha1(f.read()).hexdigest()[:12]
    key = "%s_%s_%s" % (kind, "_".join(repr(a) for a in args), src_hash)
    path = os.path.join(d, "".join(c if c.isalnum() or c in "._-" else "_" for c in key) + ".npy")
    if os.path.exists(path):
        try:
            return np.load(path)
        except Exception:
            pass
    out = fn(*args)
    try:
        os.makedirs(d, exist_ok=True)
        tmp = path + ".tmp%d.npy" % os.getpid()
        np.save(tmp, out)
        os.replace(tmp, path)
    except OSError:
        pass
    return out


def adjacency_stream(edges, n: int):
    """The symmetric adjacency of a canonical edge list in the stream layout
    of Section 5.2 (the edges of each vertex given together, in order):
    (off, adj) with off[n + 1] uint64 offsets and adj[2 m] uint32
    neighbours, every list sorted by id."""
    e = np.asarray(edges, dtype=np.uint32).reshape(-1, 2)
    src = np.concatenate([e[:, 0], e[:, 1]]).astype(np.uint64)
    dst = np.concatenate([e[:, 1], e[:, 0]]).astype(np.uint64)
    order = np.argsort((src << np.uint64(32)) | dst, kind="stable")
    adj = dst[order].astype(np.uint32)
    counts = np.bincount(src.astype(np.int64), minlength=n)[:n] if len(src) else np.zeros(n, dtype=np.int64)
    off = np.zeros(n + 1, dtype=np.uint64)
    off[1:] = np.cumsum(counts, dtype=np.uint64)
    return off, adj


# ---------------------------------------------------------------- closed forms

def canonical(pairs) -> np.ndarray:
    """Canonical form of an arbitrary pair list: (min, max), no self-loops,
    sorted, unique.  Input-side helper for the closed-form builders."""
    a = np.asarray(pairs, dtype=np.int64).reshape(-1, 2)
    a = a[a[:, 0] != a[:, 1]]
    a = np.stack([a.min(axis=1), a.max(axis=1)], axis=1)
    if len(a) == 0:
        return np.zeros((0, 2), dtype=np.uint32)
    a = np.unique(a, axis=0)
    return a.astype(np.uint32)


def complete(k: int, offset: int = 0) -> np.ndarray:
    """K_k on vertices offset..offset+k-1 (C(k, 3) triangles)."""
    return canonical([(offset + i, offset + j) for i in range(k) for j in range(i + 1, k)])


def wheel(k: int) -> np.ndarray:
    """Wheel W_k: hub 0 joined to a k-cycle 1..k (k triangles for k >= 4)."""
    rim = [(1 + i, 1 + (i + 1) % k) for i in range(k)]
    return canonical([(0, 1 + i) for i in range(k)] + rim)


def star(k: int) -> np.ndarray:
    """Star with k leaves (no triangles)."""
    return canonical([(0, 1 + i) for i in range(k)])


def cycle(k: int) -> np.ndarray:
    """Cycle C_k (one triangle when k == 3, none otherwise)."""
    return canonical([(i, (i + 1) % k) for i in range(k)])


def random_tree(n: int, seed: int) -> np.ndarray:
    """Random recursive tree on n vertices (no triangles)."""
    rng = np.random.default_rng(seed)
    return canonical([(i, int(rng.integers(0, i))) for i in range(1, n)])


def complete_bipartite(a: int, b: int) -> np.ndarray:
    """K_{a,b} (no triangles)."""
    return canonical([(i, a + j) for i in range(a) for j in range(b)])


def disjoint_union(*graphs) -> tuple[np.ndarray, int]:
    """Disjoint union of canonical edge lists; returns (edges, n)."""
    parts, off = [], 0
    for g in graphs:
        g = np.asarray(g, dtype=np.int64).reshape(-1, 2)
        nv = int(g.max()) + 1 if len(g) else 0
        parts.append(g + off)
        off += nv
    return canonical(np.concatenate(parts) if parts else np.zeros((0, 2))), off


def num_vertices(edges: np.ndarray) -> int:
    return int(edges.max()) + 1 if len(edges) else 0


# ---------------------------------------------------------------- batch mix

def batch_specs(count: int, seed: int = 1):
    """Descriptions of `count` small uneven graphs: n log-uniform in
    [100, 50000], average degree uniform in [4, 64] (below n - 1), alternating
    Erdos-Renyi and Chung-Lu (exponent 2.3), p drawn from {0.1, 0.5, 1.0},
    sampling seed = index + 1."""
    rng = np.random.default_rng(seed)
    specs = []
    for i in range(count):
        n = int(math.floor(math.exp(rng.uniform(math.log(100), math.log(50000)))))
        avg = min(float(rng.uniform(4, 64)), n - 1.0)
        m = int(n * avg / 2)
        kind = "er" if i % 2 == 0 else "chung_lu"
        if kind == "chung_lu":
            m = min(m, n * (n - 1) // 4)
        p = float(rng.choice([0.1, 0.5, 1.0]))
        specs.append({"kind": kind, "n": n, "m": m, "p": p, "seed": i + 1, "gseed": seed * 1000003 + i})
    return specs


def batch_graph(spec) -> np.ndarray:
    """Edges of one graph described by batch_specs."""
    if spec["kind"] == "er":
        return er(spec["n"], spec["m"], spec["gseed"])
    avg = 2.0 * spec["m"] / spec["n"]
    wmax = max(2.0, min(spec["n"] / 4.0, 10.0 * avg))
    return chung_lu(spec["n"], spec["m"], 2.3, wmax, spec["gseed"])
