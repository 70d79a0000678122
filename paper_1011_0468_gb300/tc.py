"""ctypes binding of libtc.so (the C ABI declared in include/tc.h).

Argument marshalling only: every step of the computation runs in the CUDA
kernels of libtc.so.  The functions carry the C names (``tc_graph_create``,
``tc_count``, ...); ``Graph`` wraps them for convenience.  PyTorch is used,
when present, only for device memory (edge lists already on the GPU) and
streams.  If libtc.so is missing this module raises instead of falling back
to any CPU path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libtc.so")

TC_OK, TC_EINVAL, TC_ENOMEM, TC_ECUDA, TC_ETIMEOUT, TC_EBUSY = range(6)
_STATUS = {0: "TC_OK", 1: "TC_EINVAL", 2: "TC_ENOMEM", 3: "TC_ECUDA", 4: "TC_ETIMEOUT", 5: "TC_EBUSY"}
PHASES = ("sample", "csr", "light", "heavy", "total")


class TCError(RuntimeError):
    def __init__(self, status: int, what: str):
        super().__init__("%s failed: %s" % (what, _STATUS.get(status, status)))
        self.status = status


class tc_result(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("m_sampled", ctypes.c_uint64), ("n", ctypes.c_uint32),
                ("n_heavy", ctypes.c_uint32), ("t_light", ctypes.c_uint64), ("t_heavy", ctypes.c_uint64),
                ("estimate", ctypes.c_double), ("src_elems", ctypes.c_uint64), ("nbr_elems", ctypes.c_uint64),
                ("partners", ctypes.c_uint64), ("heavy_mma_flops", ctypes.c_uint64), ("ms", ctypes.c_float * 8)]

    def as_dict(self) -> dict:
        d = {k: getattr(self, k) for k, _ in self._fields_ if k != "ms"}
        d["ms"] = {name: float(self.ms[i]) for i, name in enumerate(PHASES)}
        return d


_lib = None
_u32p = ctypes.POINTER(ctypes.c_uint32)
_u8p = ctypes.POINTER(ctypes.c_uint8)
_u64p = ctypes.POINTER(ctypes.c_uint64)
_vp = ctypes.c_void_p


class tc_triple_result(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("m_sampled", ctypes.c_uint64), ("n", ctypes.c_uint32),
                ("n_heavy", ctypes.c_uint32), ("universe", ctypes.c_uint64), ("samples", ctypes.c_uint64),
                ("closed_wedge", ctypes.c_uint64), ("closed_path", ctypes.c_uint64), ("estimate", ctypes.c_double),
                ("mode", ctypes.c_uint32), ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


TC_TRIPLES_SIMPLE, TC_TRIPLES_HYBRID = 0, 1
_TRIPLE_MODES = {"simple": TC_TRIPLES_SIMPLE, "hybrid": TC_TRIPLES_HYBRID}


class tc_schedule(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint32) for k in ("warp_max", "seg_w", "seg_b", "seg_l", "work_w", "work_b", "work_l",
                                               "run_b", "mid_max", "lookup")]


class tc_stream_result(ctypes.Structure):
    _fields_ = [("m", ctypes.c_uint64), ("n", ctypes.c_uint32), ("n_heavy", ctypes.c_uint32),
                ("candidates", ctypes.c_uint64), ("sampled_entries", ctypes.c_uint64), ("universe", ctypes.c_uint64),
                ("samples", ctypes.c_uint64), ("closed_wedge", ctypes.c_uint64), ("closed_pair", ctypes.c_uint64),
                ("estimate", ctypes.c_double), ("bytes_streamed", ctypes.c_uint64), ("passes", ctypes.c_uint32),
                ("ms", ctypes.c_float)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class tc_request_info(ctypes.Structure):
    _fields_ = [("res", tc_result), ("status", ctypes.c_int32), ("wave_size", ctypes.c_uint32),
                ("t_submit_us", ctypes.c_double), ("t_admit_us", ctypes.c_double), ("t_done_us", ctypes.c_double)]


class tc_server_stats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "queued", "waves", "max_wave",
                                                "resident_graphs", "resident_bytes", "graphs", "slot_bytes",
                                                "budget_bytes", "uploads", "evictions")]


# (name, restype, argtypes) of every exported entry point of include/tc.h
SIGNATURES = [
    ("tc_set_allocator", None, [_vp, _vp, _vp]),
    ("tc_graph_create", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, _vp,
                                       ctypes.POINTER(_vp)]),
    ("tc_graph_destroy", None, [_vp]),
    ("tc_graph_num_edges", ctypes.c_uint64, [_vp]),
    ("tc_graph_num_vertices", ctypes.c_uint32, [_vp]),
    ("tc_graph_device_bytes", ctypes.c_uint64, [_vp]),
    ("tc_graph_set_timing", ctypes.c_int, [_vp, ctypes.c_int]),
    ("tc_graph_set_sample_floor", ctypes.c_int, [_vp, ctypes.c_int64]),
    ("tc_graph_set_core_ranks", ctypes.c_int, [_vp, ctypes.c_int64]),
    ("tc_graph_set_partition", ctypes.c_int, [_vp, ctypes.c_int]),
    ("tc_graph_set_schedule", ctypes.c_int, [_vp, ctypes.POINTER(tc_schedule)]),
    ("tc_graph_get_schedule", ctypes.c_int, [_vp, ctypes.POINTER(tc_schedule)]),
    ("tc_graph_autotune", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_uint64, ctypes.c_char_p, ctypes.c_uint32]),
    ("tc_graph_get_core_model", ctypes.c_int, [_vp, ctypes.c_double, ctypes.POINTER(ctypes.c_double),
                                               ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_uint32)]),
    ("tc_graph_timing_drain", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_float), ctypes.c_uint32]),
    ("tc_count", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_uint64, ctypes.POINTER(tc_result)]),
    ("tc_count_async", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_uint64, _vp, _vp]),
    ("tc_count_batch", ctypes.c_int, [ctypes.POINTER(_vp), ctypes.POINTER(ctypes.c_double), _u64p, ctypes.c_uint32,
                                      _vp]),
    ("tc_graph_sync", ctypes.c_int, [_vp]),
    ("tc_graph_export_sample", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_uint64, _u32p, _u8p, _u32p, _u64p]),
    ("tc_graph_export_csr", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_uint64, _u32p, _u32p, _u64p]),
    ("tc_graph_export_edges", ctypes.c_int, [_vp, _u32p]),
    ("tc_count_triples", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_int,
                                        ctypes.POINTER(tc_triple_result)]),
    ("tc_suggest_p", ctypes.c_double, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_double]),
    ("tc_count_sweep", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), _u64p, ctypes.c_uint32, _vp]),
    ("tc_count_adaptive", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                         ctypes.c_uint32, ctypes.POINTER(tc_result), ctypes.POINTER(ctypes.c_double),
                                         ctypes.POINTER(ctypes.c_uint32)]),
    ("tc_count_auto", ctypes.c_int, [_vp, ctypes.c_double, ctypes.c_double, ctypes.c_uint64,
                                     ctypes.POINTER(tc_result), ctypes.POINTER(ctypes.c_double)]),
    ("tc_stream_count", ctypes.c_int, [_vp, _vp, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint64, ctypes.c_double,
                                       ctypes.c_uint64, _vp, ctypes.POINTER(tc_stream_result)]),
    ("tc_status_str", ctypes.c_char_p, [ctypes.c_int]),
    ("tc_version", ctypes.c_int, []),
    ("tc_release_cached_memory", ctypes.c_int, []),
    ("tc_check_bounded_wait", ctypes.c_int, [ctypes.c_uint32]),
    ("tc_launch_count", ctypes.c_uint64, []),
    ("tc_count_noalloc", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64,
                                        ctypes.POINTER(tc_result), _vp]),
    ("tc_batch_create", ctypes.c_int, [_vp, _u64p, _u32p, ctypes.c_uint32, ctypes.c_int, _vp, ctypes.POINTER(_vp)]),
    ("tc_batch_count", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), _u64p, _vp]),
    ("tc_batch_autotune", ctypes.c_int, [_vp, ctypes.POINTER(ctypes.c_double), _u64p, ctypes.c_char_p,
                                         ctypes.c_uint32]),
    ("tc_batch_destroy", None, [_vp]),
    ("tc_batch_size", ctypes.c_uint32, [_vp]),
    ("tc_batch_num_edges", ctypes.c_uint64, [_vp]),
    ("tc_batch_device_bytes", ctypes.c_uint64, [_vp]),
    ("tc_server_create", ctypes.c_int, [ctypes.c_uint64, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_uint32,
                                        ctypes.c_uint32, ctypes.POINTER(_vp)]),
    ("tc_server_add_graph", ctypes.c_int, [_vp, _vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.c_int, _u32p]),
    ("tc_server_submit", ctypes.c_int, [_vp, ctypes.c_uint32, ctypes.c_double, ctypes.c_uint64, _u64p]),
    ("tc_server_poll", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.POINTER(tc_request_info)]),
    ("tc_server_wait", ctypes.c_int, [_vp, ctypes.c_uint64, ctypes.c_uint32, ctypes.POINTER(tc_request_info)]),
    ("tc_server_get_stats", ctypes.c_int, [_vp, ctypes.POINTER(tc_server_stats)]),
    ("tc_server_destroy", None, [_vp]),
]

# numpy view of tc_result (same layout as the C struct)
RESULT_DTYPE = np.dtype([("m", "<u8"), ("m_sampled", "<u8"), ("n", "<u4"), ("n_heavy", "<u4"), ("t_light", "<u8"),
                         ("t_heavy", "<u8"), ("estimate", "<f8"), ("src_elems", "<u8"), ("nbr_elems", "<u8"),
                         ("partners", "<u8"), ("heavy_mma_flops", "<u8"), ("ms", "<f4", (8,))])

# limits of tc_count_noalloc (include/tc.h)
TC_NOALLOC_MAX_EDGES = 1 << 18
TC_NOALLOC_MAX_VERTICES = 1 << 18


def lib():
    """The loaded libtc.so (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise RuntimeError("libtc.so is not built (%s); run __graft_entry__.build() or "
                               "python paper_1011_0468_gb300/_build.py" % LIB_PATH)
        L = ctypes.CDLL(LIB_PATH)
        for name, res, args in SIGNATURES:
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(status: int, what: str):
    if status != TC_OK:
        raise TCError(status, what)


def _stream_handle(stream) -> int:
    if stream is None:
        return 0
    if isinstance(stream, int):
        return stream
    return int(stream.cuda_stream)  # torch.cuda.Stream


# ---------------------------------------------------------------- C names

def tc_graph_create(edges, m_in: int, n: int, edges_on_device: bool, stream=None) -> int:
    """edges: address (int) of m_in uint32 pairs in host or device memory."""
    g = _vp()
    _check(lib().tc_graph_create(edges, m_in, n, 1 if edges_on_device else 0, _stream_handle(stream),
                                 ctypes.byref(g)), "tc_graph_create")
    return g.value


def tc_graph_destroy(g: int) -> None:
    lib().tc_graph_destroy(g)


def tc_count(g: int, p: float, seed: int) -> tc_result:
    r = tc_result()
    _check(lib().tc_count(g, p, seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(r)), "tc_count")
    return r


def tc_count_async(g: int, p: float, seed: int, out_addr: int, stream=None) -> None:
    """Enqueue a count; out_addr: address of a tc_result (pinned host memory).
    stream: None for the graph's stream, else a torch.cuda.Stream or a raw
    cudaStream_t to run the count on."""
    _check(lib().tc_count_async(g, p, seed & 0xFFFFFFFFFFFFFFFF, out_addr, _stream_handle(stream)),
           "tc_count_async")


def tc_suggest_p(m: int, n: int, t: float, eps: float) -> float:
    """Section 3.3's p = (m^(1/2) ln n / (t eps^2))^(2/5), at most 1; 1 when
    t <= 0; -1 for bad arguments (host arithmetic in libtc)."""
    return float(lib().tc_suggest_p(m, n, t, eps))


def tc_stream_count(offsets, adj, n: int, seed: int, samples: int = 0, heavy_factor: float = 3.0,
                    chunk_entries: int = 0, stream=None) -> dict:
    """Semi-streaming count (Section 5.2) over a host-resident symmetric
    adjacency: offsets (n + 1 uint64) and adj (uint32), numpy arrays or
    pinned CPU tensors (read in place by the device)."""
    def addr(a, dtype):
        try:
            import torch
            if isinstance(a, torch.Tensor):
                return a.data_ptr(), a
        except ImportError:
            pass
        arr = np.ascontiguousarray(a, dtype=dtype)
        return arr.ctypes.data, arr
    oa, ok = addr(offsets, np.uint64)
    aa, ak = addr(adj, np.uint32)
    r = tc_stream_result()
    _check(lib().tc_stream_count(oa, aa if len(ak) else None, n, seed & 0xFFFFFFFFFFFFFFFF, int(samples),
                                 float(heavy_factor), int(chunk_entries), _stream_handle(stream), ctypes.byref(r)),
           "tc_stream_count")
    del ok, ak
    return r.as_dict()


def tc_count_batch(graphs, p, seed) -> np.ndarray:
    """One batched count over resident graphs (Graph objects or handles),
    each with its own p and seed: a numpy array of RESULT_DTYPE."""
    k = len(graphs)
    hs = (_vp * max(k, 1))(*[g.handle if isinstance(g, Graph) else g for g in graphs])
    pa = np.ascontiguousarray(np.broadcast_to(np.asarray(p, dtype=np.float64), (k,)))
    sa = np.ascontiguousarray(np.broadcast_to(np.asarray(seed, dtype=np.uint64), (k,)))
    out = np.zeros(max(k, 1), dtype=RESULT_DTYPE)
    _check(lib().tc_count_batch(hs, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), sa.ctypes.data_as(_u64p),
                                k, out.ctypes.data), "tc_count_batch")
    return out[:k]


def tc_graph_sync(g: int) -> None:
    _check(lib().tc_graph_sync(g), "tc_graph_sync")


def tc_graph_set_timing(g: int, on: bool) -> None:
    _check(lib().tc_graph_set_timing(g, 1 if on else 0), "tc_graph_set_timing")


def tc_status_str(s: int) -> str:
    return lib().tc_status_str(s).decode()


_ALLOC_T = ctypes.CFUNCTYPE(ctypes.c_void_p, ctypes.c_uint64, ctypes.c_void_p, ctypes.c_void_p)
_FREE_T = ctypes.CFUNCTYPE(None, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p)
_torch_hooks = None


def release_cached_memory() -> None:
    """Return to the system the device memory that the library's default pool
    keeps from destroyed graphs (tc_release_cached_memory)."""
    _check(lib().tc_release_cached_memory(), "tc_release_cached_memory")


def use_torch_allocator(on: bool = True) -> None:
    """Route every device allocation of libtc through PyTorch's caching
    allocator (tc_set_allocator), so graphs share torch's memory pool."""
    global _torch_hooks
    if not on:
        lib().tc_set_allocator(None, None, None)
        _torch_hooks = None
        return
    import torch

    def _alloc(nbytes, stream, ctx):
        try:
            return torch.cuda.caching_allocator_alloc(int(nbytes), torch.cuda.current_device(),
                                                      int(stream) if stream else None)
        except Exception:
            return None

    def _free(ptr, stream, ctx):
        torch.cuda.caching_allocator_delete(int(ptr))

    _torch_hooks = (_ALLOC_T(_alloc), _FREE_T(_free))
    lib().tc_set_allocator(ctypes.cast(_torch_hooks[0], _vp), ctypes.cast(_torch_hooks[1], _vp), None)


def tc_launch_count() -> int:
    return int(lib().tc_launch_count())


def tc_count_noalloc(edges_addr: int, m_in: int, n: int, p: float, seed: int, stream=None) -> tc_result:
    """Count without any device allocation, for callers that cannot allocate
    device memory (their framework's pool owns the GPU, or allocating would
    synchronise the device).  edges_addr: device address of m_in uint32
    pairs.  Inputs above TC_NOALLOC_MAX_EDGES / TC_NOALLOC_MAX_VERTICES raise
    TCError(TC_EINVAL).  Uses one fixed scratch array inside the library, so
    concurrent calls must be serialised by the caller."""
    r = tc_result()
    _check(lib().tc_count_noalloc(edges_addr if m_in else None, m_in, n, p, seed & 0xFFFFFFFFFFFFFFFF,
                                  ctypes.byref(r), _stream_handle(stream)), "tc_count_noalloc")
    return r


# ---------------------------------------------------------------- wrapper

def _as_pairs(edges):
    """Host uint32 (m, 2) array, or a CUDA tensor; returns (addr, m, on_device, keepalive)."""
    try:
        import torch
        if isinstance(edges, torch.Tensor):
            if edges.dtype not in (torch.int32, torch.uint32) and str(edges.dtype) != "torch.uint32":
                raise TypeError("edge tensor must be int32/uint32")
            t = edges.contiguous().view(-1, 2) if edges.numel() else edges.reshape(0, 2)
            return t.data_ptr(), t.shape[0], bool(t.is_cuda), t
    except ImportError:
        pass
    a = np.ascontiguousarray(np.asarray(edges, dtype=np.uint32).reshape(-1, 2))
    return a.ctypes.data, a.shape[0], False, a


class Graph:
    """A graph resident on the GPU (tc_graph_create ... tc_graph_destroy)."""

    def __init__(self, edges, n: int, stream=None):
        addr, m_in, on_dev, keep = _as_pairs(edges)
        self._h = tc_graph_create(addr if m_in else None, m_in, n, on_dev, stream)
        del keep

    @classmethod
    def from_address(cls, addr: int, m_in: int, n: int, on_device: bool, stream=None) -> "Graph":
        """Graph from m_in uint32 pairs at a raw host or device address."""
        self = cls.__new__(cls)
        self._h = tc_graph_create(addr if m_in else None, m_in, n, on_device, stream)
        return self

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("graph is closed")
        return self._h

    @property
    def m(self) -> int:
        return int(lib().tc_graph_num_edges(self.handle))

    @property
    def n(self) -> int:
        return int(lib().tc_graph_num_vertices(self.handle))

    @property
    def device_bytes(self) -> int:
        return int(lib().tc_graph_device_bytes(self.handle))

    def set_timing(self, on: bool = True):
        tc_graph_set_timing(self.handle, on)

    def set_sample_floor(self, m_lo: int):
        """Lower bound on m_p that picks the vertices whose sampled in-degrees are
        counted (tc_graph_set_sample_floor); m_lo < 0 restores the default."""
        _check(lib().tc_graph_set_sample_floor(self.handle, int(m_lo)), "tc_graph_set_sample_floor")

    def set_partition(self, mode: str):
        """Graph split by the degree partition of the later counts
        (tc_graph_set_partition): "sampled" (default) or "original"."""
        _check(lib().tc_graph_set_partition(self.handle, {"sampled": 0, "original": 1}[mode]),
               "tc_graph_set_partition")

    def schedule(self) -> dict:
        """The intersection schedule of the later counts (tc_graph_get_schedule)."""
        s = tc_schedule()
        _check(lib().tc_graph_get_schedule(self.handle, ctypes.byref(s)), "tc_graph_get_schedule")
        return {k: getattr(s, k) for k, _ in s._fields_}

    def set_schedule(self, **kw):
        """Change fields of the intersection schedule (tc_graph_set_schedule);
        no arguments restores the default.  Counts never depend on it."""
        if not kw:
            _check(lib().tc_graph_set_schedule(self.handle, None), "tc_graph_set_schedule")
            return
        cur = self.schedule()
        cur.update(kw)
        s = tc_schedule(**cur)
        _check(lib().tc_graph_set_schedule(self.handle, ctypes.byref(s)), "tc_graph_set_schedule")

    def autotune(self, p: float, seed: int) -> str:
        """tc_graph_autotune: time schedules at (p, seed), keep the fastest."""
        desc = ctypes.create_string_buffer(512)
        _check(lib().tc_graph_autotune(self.handle, p, seed & 0xFFFFFFFFFFFFFFFF, desc, 512), "tc_graph_autotune")
        return desc.value.decode()

    def core_model(self, p: float) -> dict:
        """tc_graph_get_core_model: the rates of the dense-core cost model and
        the core size a count at p uses by default (0: none)."""
        pr, tr, k = ctypes.c_double(), ctypes.c_double(), ctypes.c_uint32()
        _check(lib().tc_graph_get_core_model(self.handle, p, ctypes.byref(pr), ctypes.byref(tr), ctypes.byref(k)),
               "tc_graph_get_core_model")
        return {"probe_entries_per_s": pr.value, "contraction_flops_per_s": tr.value, "core_ranks": k.value}

    def set_core_ranks(self, ranks: int):
        """Dense core of the later counts (tc_graph_set_core_ranks): < 0 chosen
        per count (the default), 0 none, else 8192 .. 65536 top ranks."""
        _check(lib().tc_graph_set_core_ranks(self.handle, int(ranks)), "tc_graph_set_core_ranks")

    def timing_drain(self, max_counts: int = 256) -> np.ndarray:
        """Phase times (counts x 8, ms) of the timed counts since the last drain."""
        buf = np.zeros((max_counts, 8), dtype=np.float32)
        k = lib().tc_graph_timing_drain(self.handle, buf.ctypes.data_as(ctypes.POINTER(ctypes.c_float)), max_counts)
        if k < 0:
            raise TCError(TC_ECUDA, "tc_graph_timing_drain")
        return buf[:k]

    def count(self, p: float, seed: int) -> dict:
        return tc_count(self.handle, p, seed).as_dict()

    def count_async(self, p: float, seed: int, out_addr: int, stream=None) -> None:
        tc_count_async(self.handle, p, seed, out_addr, stream)

    def sync(self):
        tc_graph_sync(self.handle)

    def count_sweep(self, p, seed) -> np.ndarray:
        """Counts at several (p, seed) in one call (tc_count_sweep)."""
        pa = np.ascontiguousarray(np.atleast_1d(np.asarray(p, dtype=np.float64)))
        sa = np.ascontiguousarray(np.broadcast_to(np.asarray(seed, dtype=np.uint64), pa.shape))
        out = np.zeros(len(pa), dtype=RESULT_DTYPE)
        _check(lib().tc_count_sweep(self.handle, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    sa.ctypes.data_as(_u64p), len(pa), out.ctypes.data), "tc_count_sweep")
        return out

    def count_adaptive(self, p0: float, growth: float, tol: float, seed: int, max_counts: int = 16):
        """(result, p used, counts run) of tc_count_adaptive."""
        r, pu, cu = tc_result(), ctypes.c_double(0), ctypes.c_uint32(0)
        _check(lib().tc_count_adaptive(self.handle, p0, growth, tol, seed & 0xFFFFFFFFFFFFFFFF, max_counts,
                                       ctypes.byref(r), ctypes.byref(pu), ctypes.byref(cu)), "tc_count_adaptive")
        return r.as_dict(), pu.value, cu.value

    def count_auto(self, eps: float, pilot_p: float, seed: int):
        """(result, p used) of tc_count_auto: pilot count, suggested p, count."""
        r, pu = tc_result(), ctypes.c_double(0)
        _check(lib().tc_count_auto(self.handle, eps, pilot_p, seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(r),
                                   ctypes.byref(pu)), "tc_count_auto")
        return r.as_dict(), pu.value

    def count_triples(self, p: float, seed: int, samples: int = 0, mode: str = "hybrid") -> dict:
        """Triple sampling (tc_count_triples): mode "simple" or "hybrid";
        samples = 0 draws m_p samples."""
        r = tc_triple_result()
        _check(lib().tc_count_triples(self.handle, p, seed & 0xFFFFFFFFFFFFFFFF, int(samples), _TRIPLE_MODES[mode],
                                      ctypes.byref(r)), "tc_count_triples")
        return r.as_dict()

    def export_sample(self, p: float, seed: int, pairs: bool = True):
        """(kept pairs in canonical order, heavy flags, sampled degrees); with
        pairs=False the first item is None and the kept pairs are not copied."""
        m, n = self.m, self.n
        kept = np.empty((max(m, 1), 2), dtype=np.uint32) if pairs else None
        heavy = np.empty(max(n, 1), dtype=np.uint8)
        deg = np.empty(max(n, 1), dtype=np.uint32)
        mp = ctypes.c_uint64(0)
        _check(lib().tc_graph_export_sample(self.handle, p, seed & 0xFFFFFFFFFFFFFFFF,
                                            kept.ctypes.data_as(_u32p) if pairs else None,
                                            heavy.ctypes.data_as(_u8p), deg.ctypes.data_as(_u32p),
                                            ctypes.byref(mp)), "tc_graph_export_sample")
        return (kept[:mp.value] if pairs else None), heavy[:n], deg[:n]

    def export_csr(self, p: float, seed: int):
        """(rowptr[n+1], col[m_p]) of the degree-oriented sampled graph."""
        m, n = self.m, self.n
        rowptr = np.empty(n + 1, dtype=np.uint32)
        col = np.empty(max(m, 1), dtype=np.uint32)
        mp = ctypes.c_uint64(0)
        _check(lib().tc_graph_export_csr(self.handle, p, seed & 0xFFFFFFFFFFFFFFFF, rowptr.ctypes.data_as(_u32p),
                                         col.ctypes.data_as(_u32p), ctypes.byref(mp)), "tc_graph_export_csr")
        return rowptr, col[:mp.value]

    def export_edges(self):
        out = np.empty((max(self.m, 1), 2), dtype=np.uint32)
        _check(lib().tc_graph_export_edges(self.handle, out.ctypes.data_as(_u32p)), "tc_graph_export_edges")
        return out[:self.m]

    def close(self):
        if self._h:
            tc_graph_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Batch:
    """k independent graphs resident together and counted by one launch
    (tc_batch_create / tc_batch_count / tc_batch_destroy).  graphs: list of
    (edges, n) with edges an (m_g, 2) uint32 array in the graph's own ids."""

    def __init__(self, graphs, stream=None):
        k = len(graphs)
        m_per = np.array([len(np.asarray(e).reshape(-1, 2)) for e, _ in graphs], dtype=np.uint64)
        n_per = np.array([n for _, n in graphs], dtype=np.uint32)
        parts = [np.asarray(e, dtype=np.uint32).reshape(-1, 2) for e, _ in graphs]
        edges = np.ascontiguousarray(np.concatenate(parts) if parts else np.zeros((0, 2), np.uint32))
        h = _vp()
        _check(lib().tc_batch_create(edges.ctypes.data if len(edges) else None, m_per.ctypes.data_as(_u64p),
                                     n_per.ctypes.data_as(_u32p), k, 0, _stream_handle(stream), ctypes.byref(h)),
               "tc_batch_create")
        self._h = h.value
        self.k = k

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("batch is closed")
        return self._h

    @property
    def m(self) -> int:
        return int(lib().tc_batch_num_edges(self.handle))

    @property
    def device_bytes(self) -> int:
        return int(lib().tc_batch_device_bytes(self.handle))

    def autotune(self, p, seed) -> str:
        """tc_batch_autotune: pick the fastest intersection schedule."""
        pa = np.ascontiguousarray(np.broadcast_to(np.asarray(p, dtype=np.float64), (self.k,)))
        sa = np.ascontiguousarray(np.broadcast_to(np.asarray(seed, dtype=np.uint64), (self.k,)))
        desc = ctypes.create_string_buffer(256)
        _check(lib().tc_batch_autotune(self.handle, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                       sa.ctypes.data_as(_u64p), desc, 256), "tc_batch_autotune")
        return desc.value.decode()

    def count(self, p, seed) -> np.ndarray:
        """Results of all graphs as a numpy array of RESULT_DTYPE."""
        pa = np.ascontiguousarray(np.broadcast_to(np.asarray(p, dtype=np.float64), (self.k,)))
        sa = np.ascontiguousarray(np.broadcast_to(np.asarray(seed, dtype=np.uint64), (self.k,)))
        out = np.zeros(self.k, dtype=RESULT_DTYPE)
        _check(lib().tc_batch_count(self.handle, pa.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                    sa.ctypes.data_as(_u64p), out.ctypes.data), "tc_batch_count")
        return out

    def close(self):
        if self._h:
            lib().tc_batch_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Server:
    """Continuous-batching request server (tc_server_*): graphs registered
    once and kept resident within an HBM budget; requests (graph, p, seed)
    are counted in batched slot launches as they arrive."""

    def __init__(self, budget_bytes: int, slots: int = 2, slot_edges: int = 1 << 24,
                 slot_vertices: int = 1 << 22, slot_requests: int = 4096):
        h = _vp()
        _check(lib().tc_server_create(budget_bytes, slots, slot_edges, slot_vertices, slot_requests,
                                      ctypes.byref(h)), "tc_server_create")
        self._h = h.value

    @property
    def handle(self) -> int:
        if not self._h:
            raise ValueError("server is closed")
        return self._h

    def add_graph(self, edges, n: int) -> int:
        addr, m_in, on_dev, keep = _as_pairs(edges)
        gid = ctypes.c_uint32(0)
        _check(lib().tc_server_add_graph(self.handle, addr if m_in else None, m_in, n, 1 if on_dev else 0,
                                         ctypes.byref(gid)), "tc_server_add_graph")
        del keep
        return gid.value

    def submit(self, gid: int, p: float, seed: int) -> int:
        t = ctypes.c_uint64(0)
        _check(lib().tc_server_submit(self.handle, gid, p, seed & 0xFFFFFFFFFFFFFFFF, ctypes.byref(t)),
               "tc_server_submit")
        return t.value

    @staticmethod
    def _info(info: tc_request_info) -> dict:
        d = info.res.as_dict()
        d.pop("ms")
        d.update(status=info.status, wave_size=info.wave_size, t_submit_us=info.t_submit_us,
                 t_admit_us=info.t_admit_us, t_done_us=info.t_done_us)
        return d

    def poll(self, ticket: int):
        """The request's result dict once done (the ticket is then released), else None."""
        info = tc_request_info()
        st = lib().tc_server_poll(self.handle, ticket, ctypes.byref(info))
        if st == TC_EBUSY:
            return None
        _check(st, "tc_server_poll")
        return self._info(info)

    def wait(self, ticket: int, timeout_ms: int = 60000) -> dict:
        info = tc_request_info()
        _check(lib().tc_server_wait(self.handle, ticket, timeout_ms, ctypes.byref(info)), "tc_server_wait")
        return self._info(info)

    def stats(self) -> dict:
        st = tc_server_stats()
        _check(lib().tc_server_get_stats(self.handle, ctypes.byref(st)), "tc_server_get_stats")
        return {k: int(getattr(st, k)) for k, _ in st._fields_}

    def close(self):
        if self._h:
            lib().tc_server_destroy(self._h)
            self._h = None

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
