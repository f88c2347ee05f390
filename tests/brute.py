"""Independent checks used to pin the oracle (and, through it, the library).

Nothing here runs a breadth-first search.  The k-hop set of s is computed as
the Boolean sum of matrix powers

    R_k = A OR A^2 OR ... OR A^k,     count(s, k) = |{u != s : R_k[s, u]}|

which is the definition of "reachable in 1..k hops" written out with dense
Boolean matrix products (the traversal-as-linear-algebra view of Sec. II).
"""
from __future__ import annotations

import numpy as np

import gen


def reach_powers(A: np.ndarray, kmax: int):
    """R_1..R_kmax for a stack of Boolean adjacency matrices (..., n, n)."""
    Ai = A.astype(np.int64)
    P = Ai.copy()
    R = P > 0
    out = [R.copy()]
    for _ in range(kmax - 1):
        P = (np.matmul(P, Ai) > 0).astype(np.int64)
        R = R | (P > 0)
        out.append(R.copy())
    return out


def counts_from_reach(R: np.ndarray) -> np.ndarray:
    """count[..., s] = |{u != s : R[..., s, u]}|."""
    n = R.shape[-1]
    diag = R[..., np.arange(n), np.arange(n)]
    return R.sum(axis=-1) - diag


def per_hop_from_reach(R, k: int) -> np.ndarray:
    """per_hop[..., s, r] = |{u != s : R_r[s, u] and not R_{r-1}[s, u]}| for
    r = 1..k (the vertices first reached in r hops, i.e. at distance exactly
    r), and 1 for r = 0 (the seed itself).  R is the list R_1..R_kmax."""
    n = R[0].shape[-1]
    eye = np.eye(n, dtype=bool)
    out = np.zeros(R[0].shape[:-1] + (k + 1,), dtype=np.int64)
    out[..., 0] = 1
    prev = np.broadcast_to(eye, R[0].shape)          # R_0 = {s}
    for r in range(1, k + 1):
        cur = R[r - 1] | eye
        out[..., r] = (cur & ~prev).sum(axis=-1)
        prev = cur
    return out


def te_from_reach(R_prev, A: np.ndarray, outdeg: np.ndarray) -> np.ndarray:
    """TE(s, k) = sum of outdeg(u) over u = s or R_{k-1}[s, u] (dist < k)."""
    n = A.shape[-1]
    within = np.zeros(A.shape, dtype=bool) if R_prev is None else R_prev.copy()
    within[..., np.arange(n), np.arange(n)] = True
    return (within * outdeg[..., None, :]).sum(axis=-1)


def dense_from_csr(g) -> np.ndarray:
    A = np.zeros((g.n, g.n), dtype=bool)
    deg = np.diff(g.row_ptr).astype(np.int64)
    rows = np.repeat(np.arange(g.n), deg)
    A[rows, g.col_idx.astype(np.int64)] = True
    return A


def union_csr_from_dense_stack(A: np.ndarray) -> gen.CSRGraph:
    """Disjoint union of a stack of graphs (G, n, n): vertex g*n + i."""
    G, n, _ = A.shape
    g_, i_, j_ = np.nonzero(A)
    src = (g_ * n + i_).astype(np.int64)
    dst = (g_ * n + j_).astype(np.uint32)
    N = G * n
    row_ptr = np.zeros(N + 1, dtype=np.uint64)
    row_ptr[1:] = np.cumsum(np.bincount(src, minlength=N))
    return gen.CSRGraph(N, row_ptr, dst, False, "union", {})


def all_digraphs(n: int, self_loops: bool) -> np.ndarray:
    """Every digraph on n labelled vertices: (2^slots, n, n) Boolean."""
    slots = [(i, j) for i in range(n) for j in range(n) if self_loops or i != j]
    G = 1 << len(slots)
    bits = np.arange(G, dtype=np.int64)
    A = np.zeros((G, n, n), dtype=bool)
    for b, (i, j) in enumerate(slots):
        A[:, i, j] = ((bits >> b) & 1).astype(bool)
    return A
