"""The C ABI library builds, loads without a GPU and exports every entry
point that include/tc.h declares; argument checks that need no device."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "tc.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    names = re.findall(r"^\s*(?:const\s+)?[\w\s\*]*?\b(tc_\w+)\s*\(", src, flags=re.M)
    return sorted(set(n for n in names if not n.endswith("_fn")))


@pytest.fixture(scope="module")
def lib():
    from paper_1011_0468_gb300 import _build, tc
    _build.build()
    return tc.lib()


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tc_graph_create", "tc_count", "tc_graph_destroy", "tc_count_async",
                     "tc_graph_export_sample", "tc_graph_export_csr", "tc_status_str"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_1011_0468_gb300 import tc
    bound = {s[0] for s in tc.SIGNATURES}
    assert set(declared_functions()) <= bound


def test_status_strings(lib):
    from paper_1011_0468_gb300 import tc
    assert tc.tc_status_str(0) == "ok"
    assert tc.tc_status_str(1) == "invalid argument"
    assert lib.tc_version() >= 100


def test_argument_errors_without_device(lib):
    # checked before any device work
    from paper_1011_0468_gb300 import tc
    out = ctypes.c_void_p()
    assert lib.tc_graph_create(None, 0, 10, 0, None, None) == tc.TC_EINVAL
    assert lib.tc_graph_create(None, 5, 10, 0, None, ctypes.byref(out)) == tc.TC_EINVAL
    assert lib.tc_graph_create(None, 0, 0, 0, None, ctypes.byref(out)) == tc.TC_EINVAL
    assert out.value is None
    r = tc.tc_result()
    assert lib.tc_count(None, 0.5, 1, ctypes.byref(r)) == tc.TC_EINVAL
    assert lib.tc_graph_sync(None) == tc.TC_EINVAL
    lib.tc_graph_destroy(None)  # NULL-safe
    assert lib.tc_graph_num_edges(None) == 0
    assert lib.tc_graph_set_sample_floor(None, 0) == tc.TC_EINVAL
    assert lib.tc_graph_set_core_ranks(None, 8192) == tc.TC_EINVAL
    for limit in (0, 1000001):  # bounded-wait check: limits out of range
        assert lib.tc_check_bounded_wait(limit) == tc.TC_EINVAL


def test_result_struct_layout():
    from paper_1011_0468_gb300 import tc
    # uint64 m, m_sampled; uint32 n, n_heavy; uint64 t_light, t_heavy; double;
    # uint64 src_elems, nbr_elems, partners, heavy_mma_flops; float[8]
    assert ctypes.sizeof(tc.tc_result) == 8 + 8 + 4 + 4 + 8 + 8 + 8 + 8 + 8 + 8 + 8 + 32


def test_server_struct_layout():
    from paper_1011_0468_gb300 import tc
    # tc_result; int32 status; uint32 wave_size; double t_submit, t_admit, t_done
    assert ctypes.sizeof(tc.tc_request_info) == ctypes.sizeof(tc.tc_result) + 4 + 4 + 3 * 8
    assert tc.tc_request_info.t_submit_us.offset == ctypes.sizeof(tc.tc_result) + 8
    assert ctypes.sizeof(tc.tc_server_stats) == 12 * 8


def test_server_argument_errors_without_device(lib):
    from paper_1011_0468_gb300 import tc
    out = ctypes.c_void_p()
    assert lib.tc_server_create(1 << 30, 2, 1 << 20, 1 << 20, 64, None) == tc.TC_EINVAL
    assert lib.tc_server_create(1 << 30, 0, 1 << 20, 1 << 20, 64, ctypes.byref(out)) == tc.TC_EINVAL
    assert lib.tc_server_create(1 << 30, 9, 1 << 20, 1 << 20, 64, ctypes.byref(out)) == tc.TC_EINVAL
    assert lib.tc_server_create(1 << 30, 2, 0, 1 << 20, 64, ctypes.byref(out)) == tc.TC_EINVAL
    assert lib.tc_server_create(1 << 30, 2, 1 << 20, 1 << 20, 1 << 16, ctypes.byref(out)) == tc.TC_EINVAL
    assert out.value is None
    t = ctypes.c_uint64()
    assert lib.tc_server_submit(None, 0, 0.5, 1, ctypes.byref(t)) == tc.TC_EINVAL
    info = tc.tc_request_info()
    assert lib.tc_server_poll(None, 1, ctypes.byref(info)) == tc.TC_EINVAL
    assert lib.tc_server_wait(None, 1, 0, ctypes.byref(info)) == tc.TC_EINVAL
    lib.tc_server_destroy(None)  # NULL-safe


def test_suggest_p_host_arithmetic_matches_the_oracle(lib):
    """tc_suggest_p (host code of libtc, no device) against the oracle's
    statement of Section 3.3's p, which the oracle tests pin to the balance
    equation."""
    import oracle
    from paper_1011_0468_gb300 import tc
    for m, n, t, eps in [(10 ** 6, 10 ** 5, 1e7, 0.1), (48709772, 5284457, 3.1e8, 0.05),
                         (1051928416, 1 << 26, 4.9e10, 0.01), (20000, 2000, 1300.0, 0.2),
                         (1000, 100, 1e-3, 0.1), (1000, 100, 0.0, 0.1)]:
        assert tc.tc_suggest_p(m, n, t, eps) == oracle.suggest_p(m, n, t, eps)
    for bad in ((0, 100, 10.0, 0.1), (1000, 1, 10.0, 0.1), (1000, 100, 10.0, 0.0), (1000, 100, 10.0, float("nan"))):
        assert tc.tc_suggest_p(*bad) == -1.0
