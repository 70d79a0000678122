"""GPU (GB300, sm_103a) edge-sampled, degree-partitioned triangle counting.

Kolountzakis, Miller, Peng, Tsourakakis, "Efficient Triangle Counting in
Large Graphs via Degree-based Vertex Partitioning": sample every edge with
probability p (Section 3.1), split vertices at the m^(1/2) degree threshold
(Section 3.2), count the sampled triangles of the light and heavy classes
exactly and rescale by 1/p^3.

The computation lives in libtc.so (hand-written CUDA, C ABI in
include/tc.h); ``tc`` is its ctypes binding.
"""
from .tc import Graph, TCError, tc_count, tc_count_async, tc_graph_create, tc_graph_destroy, tc_result  # noqa: F401

__all__ = ["Graph", "TCError", "tc_graph_create", "tc_count", "tc_count_async", "tc_graph_destroy", "tc_result"]
