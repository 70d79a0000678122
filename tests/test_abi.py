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


def test_result_struct_layout():
    from paper_1011_0468_gb300 import tc
    # uint64 m, m_sampled; uint32 n, n_heavy; uint64 t_light, t_heavy; double;
    # uint64 src_elems, nbr_elems, partners, heavy_mma_flops; float[8]
    assert ctypes.sizeof(tc.tc_result) == 8 + 8 + 4 + 4 + 8 + 8 + 8 + 8 + 8 + 8 + 8 + 32
