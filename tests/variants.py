"""Inputs for the reverse and either-direction neighbourhoods, built on the
host from the CSR alone: the oracle counts them on these graphs unchanged.

- reverse (in-neighbourhood, q_r = A q_{r-1}): the transpose, every edge
  u -> w turned into w -> u;
- undirected (q_r = (A OR A^T) q_{r-1}): every edge in both directions.
"""
import numpy as np

import gen


def edges(g):
    """(tails, heads) of every stored edge of a CSR graph, in row order."""
    rp = g.row_ptr.astype(np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.uint64), np.diff(rp))
    return src, g.col_idx[: int(rp[-1])].astype(np.uint32)


def transpose(g):
    src, dst = edges(g)
    return gen.csr_raw(g.n, dst, src)


def either_direction(g):
    src, dst = edges(g)
    return gen.csr_raw(g.n, np.concatenate([src, dst.astype(np.uint64)]),
                       np.concatenate([dst, src.astype(np.uint32)]))
