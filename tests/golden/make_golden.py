"""Writes the stored oracle results used by the full-size parity tests.

Calls only gen/ (seeded inputs) and oracle/ (the CPU oracle); nothing here
touches the CUDA library.  Run from the repository root:

    python tests/golden/make_golden.py [chung_lu_4m] [rmat_s26]

chung_lu_4m: Chung-Lu power-law graph, n = 2^22 vertices, exactly 2^26
undirected edges, degree exponent 2.1, maximum expected degree 1e5, seed 1
(the multi-million-edge social-network shape of the paper's Table 1).  The
oracle result is stored for p = 1 (exact count), p in {0.1, 0.01} with
seeds 1..3, and p = 0.7 and 0.55 (samples that still keep more than 2^25
edges), with a checksum of the generated edge list so that a changed
generator is detected instead of compared against stale numbers.  Runs
already stored for the same checksum are kept, not recomputed.

rmat_s26: R-MAT, scale 26, edge factor 16, (a, b, c, d) = (0.57, 0.19, 0.19,
0.05), seed 1, symmetrised and deduplicated (about 10^9 edges, the largest
graph).  Stored: checksums of the exact degrees and heavy flags of the
whole graph, and the oracle at p = 0.05 (seeds 1 and 2), 0.25 and 0.5, each
with checksums of its kept edges and heavy flags.  The oracle's time grows
with p^2 times the sum of squared degrees: about 80 s at p = 0.05, half an
hour at p = 0.25, two hours at p = 0.5; p = 1 would take about eight hours
of one CPU thread and is not stored (the full-size test checks p = 1 by
properties that hold at any size).  The graph itself is generated
once, here, in about five minutes and 17 GB of host memory.
"""
import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import numpy as np  # noqa: E402

import gen  # noqa: E402
import oracle  # noqa: E402

WORKLOADS = {
    "chung_lu_4m": dict(kind="chung_lu", n=1 << 22, m=1 << 26, gamma=2.1, wmax=1e5, seed=1,
                        runs=[(1.0, 1)] + [(p, s) for p in (0.1, 0.01) for s in (1, 2, 3)] + [(0.7, 1), (0.55, 2)]),
    "rmat_s26": dict(kind="rmat", n=1 << 26, scale=26, edge_factor=16, a=0.57, b=0.19, c=0.19, seed=1,
                     runs=[(0.05, 1), (0.05, 2), (0.25, 1), (0.5, 1), (1.0, 1)], sample_checksums=True,
                     threads={1.0: os.cpu_count() or 1}),
}


def make_graph(spec):
    if spec["kind"] == "chung_lu":
        return gen.chung_lu(spec["n"], spec["m"], spec["gamma"], spec["wmax"], spec["seed"])
    if spec["kind"] == "rmat":
        return gen.rmat(spec["scale"], spec["edge_factor"], spec["a"], spec["b"], spec["c"], spec["seed"])
    raise ValueError(spec["kind"])


def heavy_checksum(heavy: np.ndarray) -> str:
    """sha1 (first 16 hex digits) of the heavy flags, one byte per vertex."""
    import hashlib
    return hashlib.sha1(np.ascontiguousarray(heavy, dtype=np.uint8).tobytes()).hexdigest()[:16]


def deg_checksum(deg: np.ndarray) -> str:
    """sha1 (first 16 hex digits) of the degrees as little-endian uint32."""
    import hashlib
    return hashlib.sha1(np.ascontiguousarray(deg, dtype="<u4").tobytes()).hexdigest()[:16]


def checksum(edges: np.ndarray) -> str:
    """Order-sensitive 64-bit checksum of the canonical edge list."""
    e = edges.astype(np.uint64)
    k = (e[:, 0] << np.uint64(32)) | e[:, 1]
    w = np.arange(1, len(k) + 1, dtype=np.uint64) * np.uint64(0x9E3779B97F4A7C15)
    with np.errstate(over="ignore"):
        return "%016x" % int(np.bitwise_xor.reduce(k * w) if len(k) else 0)


def main(names):
    for name in names:
        spec = WORKLOADS[name]
        t0 = time.time()
        edges = make_graph(spec)
        rec = {"workload": name, "spec": {k: v for k, v in spec.items() if k not in ("runs", "sample_checksums", "threads")},
               "m": int(len(edges)), "checksum": checksum(edges), "runs": []}
        print(name, "generated", len(edges), "edges in %.1fs" % (time.time() - t0), flush=True)
        if spec.get("sample_checksums"):  # the whole graph's degrees and partition (p = 1)
            deg = oracle.degrees(edges, spec["n"])
            rec["deg_checksum"] = deg_checksum(deg)
            heavy = oracle.partition(deg, len(edges))
            rec["heavy_checksum"] = heavy_checksum(heavy)
            rec["n_heavy"] = int(heavy.sum())
            rec["max_degree"] = int(deg.max())
        path = os.path.join(HERE, name + ".json")
        old = json.load(open(path)) if os.path.exists(path) else {}
        stored = {(r["p"], r["seed"]): r for r in old.get("runs", [])} if old.get("checksum") == rec["checksum"] else {}
        for p, seed in spec["runs"]:
            if (p, seed) in stored:
                rec["runs"].append(stored[(p, seed)])
                continue
            t0 = time.time()
            want = bool(spec.get("sample_checksums"))
            threads = spec.get("threads", {}).get(p, 1)
            r = oracle.run(edges, spec["n"], p, seed, want_sample=want, threads=threads)
            if want:
                r["kept_checksum"] = checksum(r.pop("kept"))
                r["heavy_checksum"] = heavy_checksum(r.pop("heavy"))
            r["p"], r["seed"] = p, seed
            r["estimate_hex"] = float(r["estimate"]).hex()
            r["oracle_seconds"] = round(time.time() - t0, 2)
            if threads > 1:
                r["oracle_threads"] = threads
            rec["runs"].append(r)
            print(name, p, seed, r, flush=True)
            with open(path, "w") as f:  # after every run: the long ones come last
                json.dump(rec, f, indent=1)
        with open(path, "w") as f:
            json.dump(rec, f, indent=1)


if __name__ == "__main__":
    main(sys.argv[1:] or list(WORKLOADS))
