"""GB300-native k-hop neighbourhood count.

The library computes the k-hop neighbourhood count benchmarked in
"RedisGraph: GraphBLAS Enabled Graph Database" (Sec. III): for a seed s of a
directed graph held as a sparse Boolean adjacency matrix, the number of
distinct vertices other than s reachable in 1..k hops, computed as k rounds of
a masked (OR, AND) frontier product (Sec. II: traversals as sparse linear
algebra).  The compute path is libkhop.so (hand-written CUDA for sm_103a,
C ABI in include/khop.h); this package is its ctypes binding.
"""
from .khop import *  # noqa: F401,F403
from .khop import Graph, Server, KhopError, lib, as_u64, stats_records  # noqa: F401


def build_library(force: bool = False) -> str:
    """Compile libkhop.so in-tree (nvcc, sm_103a)."""
    import importlib
    return importlib.import_module(__name__ + ".build").build(force=force)
