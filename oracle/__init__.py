"""CPU oracle for the k-hop neighbourhood count -- TEST INFRASTRUCTURE ONLY.

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import this package.  The CUDA library never calls it, and it
shares no code with the library.

``khop_oracle.c`` is a plain first-in first-out breadth-first search with a hop
limit (the definition of the count; see its header).  It is pinned in the
tests against brute-force Boolean matrix powers, closed forms and invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "khop_oracle.c")
_SO = os.path.join(_HERE, "libkhop_oracle.so")
_lock = threading.Lock()
_lib = None

UNSET = -1


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (portable flags)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-pthread", _SRC,
                        "-o", tmp], check=True)
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            vp, u64 = ctypes.c_void_p, ctypes.c_uint64
            lib.oracle_khop_many.restype = ctypes.c_int
            lib.oracle_khop_many.argtypes = [u64, vp, vp, vp, vp, u64, vp, vp, vp, u64, ctypes.c_int]
            lib.oracle_khop_dist.restype = ctypes.c_int
            lib.oracle_khop_dist.argtypes = [u64, vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp]
            _lib = lib
    return _lib


def _p(a):
    return ctypes.c_void_p(a.ctypes.data)


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint64)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.uint32)
    if ci.size == 0:
        ci = np.zeros(1, np.uint32)
    return rp, ci


def khop_counts(g, seeds, ks, nthreads: int = 0, with_te: bool = True, per_hop: bool = False):
    """Counts (uint64) for queries (seeds[i], ks[i]); ks may be a scalar.

    Returns (counts, te) or (counts, te, per_hop[nq, max_k+1]).  An out-of-range
    seed gives UINT64_MAX for both."""
    seeds = np.ascontiguousarray(np.atleast_1d(seeds), dtype=np.uint32)
    ks = np.ascontiguousarray(np.broadcast_to(np.asarray(ks, dtype=np.uint32), seeds.shape))
    nq = seeds.size
    counts = np.zeros(nq, dtype=np.uint64)
    te = np.zeros(nq, dtype=np.uint64)
    stride = int(ks.max()) + 1 if (per_hop and nq) else 0
    ph = np.zeros((nq, max(stride, 1)), dtype=np.uint64) if per_hop else None
    rp, ci = _csr(g)
    rc = _L().oracle_khop_many(g.n, _p(rp), _p(ci), _p(seeds), _p(ks), nq, _p(counts),
                               _p(te) if with_te else None, _p(ph) if per_hop else None,
                               stride, nthreads)
    if rc != 0:
        raise MemoryError("oracle out of memory")
    if per_hop:
        return counts, te, ph
    return counts, te


def khop_count(g, s: int, k: int) -> int:
    c, _ = khop_counts(g, [s], [k], nthreads=1)
    return int(c[0])


def khop_dist(g, s: int, k: int) -> np.ndarray:
    """int32 distances from s, UNSET (-1) beyond k hops."""
    out = np.empty(g.n, dtype=np.int32)
    rp, ci = _csr(g)
    rc = _L().oracle_khop_dist(g.n, _p(rp), _p(ci), s, k, _p(out))
    if rc != 0:
        raise ValueError("seed out of range" if rc == -1 else "oracle out of memory")
    return out


def bfs_parents(g, s: int, k: int) -> np.ndarray:
    """uint32 BFS parents over the (MIN, SECOND) semiring, from the hop
    distances (Sec. II's semiring view of a traversal; parent = the smallest
    predecessor one hop closer): parent[v] = min{u : u -> v, dist(u) =
    dist(v) - 1} for 1 <= dist(v) <= k, parent[s] = s, UINT32_MAX elsewhere.
    The definition written out over every edge."""
    d = khop_dist(g, s, k)
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    dst = np.asarray(g.col_idx[: int(rp[-1])], dtype=np.int64)
    ok = (d[src] >= 0) & (d[dst] == d[src] + 1)
    par = np.full(g.n, np.iinfo(np.uint32).max, dtype=np.uint64)
    np.minimum.at(par, dst[ok], src[ok].astype(np.uint64))
    par[s] = s
    return par.astype(np.uint32)


# ---- masked matrix-vector products over semirings ----------------------------

SR_OR_AND, SR_PLUS_TIMES, SR_MIN_SECOND, SR_MAX_SECOND = 0, 1, 2, 3
U64MAX = np.uint64(2**64 - 1)


def mxv(g, semiring: int, x, mask=None, complement: bool = False) -> np.ndarray:
    """y = A^T x over a semiring, edge by edge (Sec. II: a traversal step is a
    sparse matrix-vector product): for every stored edge u -> v the term
    x[u] (x) 1 is folded into y[v] with the semiring's (+); vertices the mask
    does not select, and vertices with no in-edge, keep the (+)-identity.
      OR_AND: y[v] = 1 if some u -> v has x[u] != 0;  PLUS_TIMES: sum of x[u]
      mod 2^64;  MIN_SECOND / MAX_SECOND: min / max of x[u].
    mask: uint32 bitmap (bit v of word v // 32) or None; complement selects
    the clear bits.  A plain loop over the edge list (numpy ufunc.at)."""
    x = np.ascontiguousarray(x, dtype=np.uint64)
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.int64), np.diff(rp))
    dst = np.asarray(g.col_idx[: int(rp[-1])], dtype=np.int64)
    if semiring == SR_OR_AND:
        y = np.zeros(g.n, dtype=np.uint64)
        np.bitwise_or.at(y, dst, (x[src] != 0).astype(np.uint64))
    elif semiring == SR_PLUS_TIMES:
        y = np.zeros(g.n, dtype=np.uint64)
        np.add.at(y, dst, x[src])          # uint64: wraps mod 2^64
    elif semiring == SR_MIN_SECOND:
        y = np.full(g.n, U64MAX, dtype=np.uint64)
        np.minimum.at(y, dst, x[src])
    elif semiring == SR_MAX_SECOND:
        y = np.zeros(g.n, dtype=np.uint64)
        np.maximum.at(y, dst, x[src])
    else:
        raise ValueError("unknown semiring")
    if mask is not None:
        m = np.asarray(mask, dtype=np.uint32)
        bits = ((m[np.arange(g.n) >> 5] >> (np.arange(g.n) & 31).astype(np.uint32)) & 1).astype(bool)
        sel = ~bits if complement else bits
        ident = U64MAX if semiring == SR_MIN_SECOND else np.uint64(0)
        y[~sel] = ident
    return y
