"""Seeded synthetic inputs for the k-hop neighbourhood count.

This module makes graphs, seed lists and request streams and nothing else: it
holds none of the counting method.  The CPU oracle and the CUDA library both
consume its output, so the two sides always see the same inputs.

Workload shapes follow the paper's benchmark (Sec. III): Graph500-style
Kronecker (R-MAT) graphs and a Twitter-like power-law graph, 300 seeds for the
1- and 2-hop queries and 10 seeds for the 3- and 6-hop queries.

The heavy lifting is in ``khopgen.c`` (counter-based splitmix64, R-MAT,
Fisher-Yates relabelling, CSR build with dedup, Walker alias tables), compiled
on first use with gcc into ``libkhopgen.so`` next to this file.
"""
from __future__ import annotations

import ctypes
import hashlib
import json
import os
import shutil
import subprocess
import threading
from dataclasses import dataclass, field

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "khopgen.c")
_SO = os.path.join(_HERE, "libkhopgen.so")
_lock = threading.Lock()
_lib = None

# Stream sub-keys derived from a user seed: draw j of stream `seed`.
_SUB_EDGES, _SUB_PERM, _SUB_SRC, _SUB_DST, _SUB_WPERM_OUT, _SUB_WPERM_IN = range(6)


def build(force: bool = False) -> str:
    """Compile khopgen.c into libkhopgen.so (portable flags, no -march)."""
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.run(["gcc", "-O3", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                        _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _SO)
    return _SO


def _L():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_SO)
            u64, i64, u32p, u64p = ctypes.c_uint64, ctypes.c_int64, ctypes.c_void_p, ctypes.c_void_p
            lib.khopgen_rand.restype = u64
            lib.khopgen_rand.argtypes = [u64, u64]
            lib.khopgen_unif.restype = ctypes.c_double
            lib.khopgen_unif.argtypes = [u64, u64]
            lib.khopgen_rand_fill.argtypes = [u64, u64, u64, u64p]
            lib.khopgen_rmat_edges.restype = ctypes.c_int
            lib.khopgen_rmat_edges.argtypes = [ctypes.c_int, u64, ctypes.c_double, ctypes.c_double,
                                               ctypes.c_double, u64, u32p, u32p, ctypes.c_int]
            lib.khopgen_permutation.argtypes = [u64, u64, u32p]
            lib.khopgen_relabel.argtypes = [u32p, u32p, u64, ctypes.c_int]
            lib.khopgen_csr_begin.restype = i64
            lib.khopgen_csr_begin.argtypes = [u64, u64, u32p, u32p, ctypes.c_int, ctypes.c_int,
                                              ctypes.POINTER(ctypes.c_void_p)]
            lib.khopgen_csr_finish.argtypes = [ctypes.c_void_p, u64p, u32p]
            lib.khopgen_seeds.restype = i64
            lib.khopgen_seeds.argtypes = [u64, u64p, u64, u64, u32p]
            lib.khopgen_alias_build.restype = ctypes.c_int
            lib.khopgen_alias_build.argtypes = [u64, ctypes.c_void_p, ctypes.c_void_p, u32p]
            lib.khopgen_chunglu_edges.argtypes = [u64, ctypes.c_void_p, u32p, ctypes.c_void_p, u32p,
                                                  u64, u64, u64, u64, u32p, u32p, ctypes.c_int]
            lib.khopgen_poisson.argtypes = [u64, ctypes.c_double, u64, ctypes.c_void_p, u32p,
                                            ctypes.c_int, u64, u32p, ctypes.c_void_p, u32p, u32p]
            lib.khopgen_checksum.restype = u64
            lib.khopgen_checksum.argtypes = [ctypes.c_void_p, u64, ctypes.c_int]
            lib.khopgen_powerlaw_weights.restype = ctypes.c_double
            lib.khopgen_powerlaw_weights.argtypes = [u64, ctypes.c_double, ctypes.c_double,
                                                     ctypes.c_void_p]
            lib.khopgen_chunglu_begin.restype = i64
            lib.khopgen_chunglu_begin.argtypes = [u64, ctypes.c_void_p, u32p, ctypes.c_void_p,
                                                  u32p, u64, u64, u64, u64, ctypes.c_int,
                                                  ctypes.POINTER(ctypes.c_uint64),
                                                  ctypes.POINTER(ctypes.c_void_p)]
            lib.khopgen_chunglu_finish.argtypes = [ctypes.c_void_p, u64p, u32p]
            _lib = lib
    return _lib


def _p(a: np.ndarray):
    return ctypes.c_void_p(a.ctypes.data)


def rand(key: int, i: int) -> int:
    """Draw i of the counter-based splitmix64 stream `key` (uint64)."""
    return int(_L().khopgen_rand(key & (2**64 - 1), i))


def rand_array(key: int, start: int, count: int) -> np.ndarray:
    out = np.empty(count, dtype=np.uint64)
    _L().khopgen_rand_fill(key & (2**64 - 1), start, count, _p(out))
    return out


def subkey(seed: int, j: int) -> int:
    return rand(seed, j)


@dataclass
class CSRGraph:
    """A directed graph as CSR: row u lists the heads of the edges u -> w.

    row_ptr is uint64[n+1], col_idx is uint32[nnz].  `symmetric` records that
    every edge has its reverse (so CSC equals CSR)."""
    n: int
    row_ptr: np.ndarray
    col_idx: np.ndarray
    symmetric: bool = False
    name: str = ""
    params: dict = field(default_factory=dict)

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1])

    def out_degree(self) -> np.ndarray:
        return np.diff(self.row_ptr).astype(np.int64)

    def row_ptr_as(self, width: int) -> np.ndarray:
        if width == 8:
            return self.row_ptr
        if self.nnz >= 2**32:
            raise ValueError("nnz does not fit 32-bit row_ptr")
        return self.row_ptr.astype(np.uint32)


def csr_from_edges(n: int, src, dst, symmetrize: bool = False, nthreads: int = 0,
                   name: str = "", params: dict | None = None) -> CSRGraph:
    """Edge list -> CSR with self-loops removed, optional symmetrisation and
    duplicate edges collapsed; each row sorted ascending."""
    src = np.ascontiguousarray(src, dtype=np.uint32)
    dst = np.ascontiguousarray(dst, dtype=np.uint32)
    if src.shape != dst.shape:
        raise ValueError("src/dst length mismatch")
    if src.size and (int(src.max()) >= n or int(dst.max()) >= n):
        raise ValueError("vertex id out of range")
    h = ctypes.c_void_p()
    nnz = _L().khopgen_csr_begin(n, src.size, _p(src), _p(dst), int(symmetrize), nthreads,
                                 ctypes.byref(h))
    if nnz < 0:
        raise MemoryError("csr build failed")
    row_ptr = np.empty(n + 1, dtype=np.uint64)
    col = np.empty(max(nnz, 1), dtype=np.uint32)
    _L().khopgen_csr_finish(h, _p(row_ptr), _p(col))
    return CSRGraph(n, row_ptr, col[:nnz], symmetrize, name, dict(params or {}))


def csr_raw(n: int, src, dst) -> CSRGraph:
    """Edge list -> CSR keeping duplicates and self-loops, edges of a row in
    input order (a stable sort by tail)."""
    src = np.asarray(src, dtype=np.uint64)
    dst = np.asarray(dst, dtype=np.uint32)
    order = np.argsort(src, kind="stable")
    counts = np.bincount(src.astype(np.int64), minlength=n)[:n] if src.size else np.zeros(n, np.int64)
    row_ptr = np.zeros(n + 1, dtype=np.uint64)
    row_ptr[1:] = np.cumsum(counts)
    return CSRGraph(n, row_ptr, dst[order].astype(np.uint32), False, "raw", {})


def rmat(scale: int, edge_factor: int = 16, A: float = 0.57, B: float = 0.19, C: float = 0.19,
         seed: int = 1, symmetrize: bool = False, permute: bool = True,
         nthreads: int = 0) -> CSRGraph:
    """Graph500-shaped Kronecker (R-MAT) graph on 2^scale vertices.

    edge_factor * 2^scale candidate edges; edge e, level l draws
    u = draw(e*scale + l) of stream subkey(seed, 0) and picks quadrant
    (0,0) if u < A, (0,1) if u < A+B, (1,0) if u < A+B+C, else (1,1), most
    significant bit first.  With `permute`, vertex ids are relabelled by a
    seeded Fisher-Yates permutation (stream subkey(seed, 1)), as Graph500 does.
    Self-loops are dropped and duplicates collapsed; `symmetrize` adds every
    reverse edge first."""
    n = 1 << scale
    m = edge_factor * n
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    rc = _L().khopgen_rmat_edges(scale, m, A, B, C, subkey(seed, _SUB_EDGES), _p(src), _p(dst),
                                 nthreads)
    if rc != 0:
        raise ValueError("bad R-MAT parameters")
    if permute:
        perm = np.empty(n, dtype=np.uint32)
        _L().khopgen_permutation(n, subkey(seed, _SUB_PERM), _p(perm))
        _L().khopgen_relabel(_p(perm), _p(src), m, nthreads)
        _L().khopgen_relabel(_p(perm), _p(dst), m, nthreads)
    params = dict(kind="rmat", scale=scale, edge_factor=edge_factor, A=A, B=B, C=C, seed=seed,
                  symmetrize=symmetrize, permute=permute, candidates=m)
    name = f"rmat-s{scale}-ef{edge_factor}-seed{seed}{'-sym' if symmetrize else ''}"
    return csr_from_edges(n, src, dst, symmetrize, nthreads, name, params)


def rmat_edges_unpermuted(scale: int, m: int, A=0.57, B=0.19, C=0.19, seed: int = 1):
    """Raw R-MAT candidate edges before relabelling (for generator checks)."""
    src = np.empty(m, dtype=np.uint32)
    dst = np.empty(m, dtype=np.uint32)
    rc = _L().khopgen_rmat_edges(scale, m, A, B, C, subkey(seed, _SUB_EDGES), _p(src), _p(dst), 0)
    if rc != 0:
        raise ValueError("bad R-MAT parameters")
    return src, dst


def powerlaw_weights(n: int, w_max: float, total: float) -> tuple[np.ndarray, float]:
    """Quantile weights of the density p(w) ~ w^-2 on [w_min, w_max]:
    w(i) = w_min / (1 - u_i (1 - w_min / w_max)), u_i = (i + 1/2) / n, with
    w_min chosen (bisection) so that the weights sum to `total`."""
    w = np.empty(n, dtype=np.float64)
    w_min = _L().khopgen_powerlaw_weights(n, float(w_max), float(total), _p(w))
    if w_min < 0:
        raise ValueError("no w_min gives that total")
    return w, w_min


def alias_table(w: np.ndarray):
    """Walker alias table (prob, alias) for weights w."""
    w = np.ascontiguousarray(w, dtype=np.float64)
    prob = np.empty(w.size, dtype=np.float64)
    alias = np.empty(w.size, dtype=np.uint32)
    if _L().khopgen_alias_build(w.size, _p(w), _p(prob), _p(alias)) != 0:
        raise ValueError("bad weights")
    return prob, alias


def chunglu(n: int, edges: int, w_max: float, seed: int = 4, nthreads: int = 0,
            overdraw: float = 1.25) -> CSRGraph:
    """Directed Chung-Lu graph shaped like a social follow graph.

    Out- and in-weights are the power-law quantile weights of powerlaw_weights
    (summing to `edges`), each assigned to the vertices by its own seeded
    permutation.  Candidate edge i has tail ~ w_out and head ~ w_in (alias
    tables, draw i of two counter-based streams); self-loops are dropped and
    duplicates collapsed.  The graph keeps the distinct edges whose first
    occurrence lies in the shortest prefix of candidates -- a multiple of 2^20
    -- that yields at least `edges` distinct edges.  Rows are sorted."""
    w, w_min = powerlaw_weights(n, w_max, edges)
    w_out = np.empty(n, np.float64)
    w_in = np.empty(n, np.float64)
    w_out[permutation(n, subkey(seed, _SUB_WPERM_OUT))] = w
    w_in[permutation(n, subkey(seed, _SUB_WPERM_IN))] = w
    del w
    po, ao = alias_table(w_out)
    pi, ai = alias_table(w_in)
    del w_out, w_in
    m = -(-int(edges * overdraw) // (1 << 20)) << 20
    while True:
        h = ctypes.c_void_p()
        mstar = ctypes.c_uint64()
        kept = _L().khopgen_chunglu_begin(n, _p(po), _p(ao), _p(pi), _p(ai),
                                          subkey(seed, _SUB_SRC), subkey(seed, _SUB_DST), m,
                                          edges, nthreads, ctypes.byref(mstar), ctypes.byref(h))
        if kept == -2:
            m = -(-int(m * 1.1) // (1 << 20)) << 20
            continue
        if kept < 0:
            raise MemoryError("Chung-Lu build failed")
        break
    row_ptr = np.empty(n + 1, dtype=np.uint64)
    col = np.empty(max(kept, 1), dtype=np.uint32)
    _L().khopgen_chunglu_finish(h, _p(row_ptr), _p(col))
    params = dict(kind="chunglu", n=n, edges_target=edges, w_max=w_max, w_min=w_min, seed=seed,
                  candidates_drawn=m, prefix_kept=int(mstar.value), edges=int(kept))
    return CSRGraph(n, row_ptr, col[:kept], False, f"chunglu-n{n}-m{edges}-seed{seed}", params)


# --------------------------------------------------------------------------
# On-disk graph cache.  A cached graph is one file:
#   bytes 0..7     magic b"KHOPCSR1"
#   bytes 8..15    header length H (uint64, little-endian)
#   bytes 16..     H bytes of JSON: n, nnz, row_ptr_bytes (8), col_idx_bytes
#                  (4), symmetric, name, params, the generator's source hash,
#                  and checksum() of each array
#   offset 4096*ceil((16 + H) / 4096): row_ptr (uint64[n+1]), then col_idx
#                  (uint32[nnz])
# The file name carries a hash of the builder's name, its parameters and the
# generator sources, so a change to any of them misses the cache.  Loading
# re-verifies n, nnz, row_ptr[n] = nnz and both checksums; a file that fails
# is ignored (and rebuilt).

_MAGIC = b"KHOPCSR1"
_ALIGN = 4096


def checksum(a: np.ndarray, nthreads: int = 0) -> int:
    """64-bit checksum of an array's bytes (khopgen_checksum)."""
    a = np.ascontiguousarray(a)
    return int(_L().khopgen_checksum(ctypes.c_void_p(a.ctypes.data), a.nbytes, nthreads))


def _generator_hash() -> str:
    h = hashlib.sha256()
    for f in (_SRC, os.path.abspath(__file__)):
        with open(f, "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def cache_dir() -> str:
    """$KHOP_GRAPH_CACHE, else ~/.cache/khop_graphs."""
    return os.environ.get("KHOP_GRAPH_CACHE") or os.path.join(os.path.expanduser("~"), ".cache",
                                                             "khop_graphs")


def _cache_path(builder: str, params: dict, directory: str | None) -> str:
    key = json.dumps({"builder": builder, "params": params, "gen": _generator_hash()},
                     sort_keys=True)
    tag = hashlib.sha256(key.encode()).hexdigest()[:20]
    return os.path.join(directory or cache_dir(), f"{builder}-{tag}.csr")


def save_graph(g: CSRGraph, path: str) -> bool:
    """Write g to `path` (atomically: a temporary file, then a rename).
    Returns False (writing nothing) when the disk lacks room for it."""
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint64)
    ci = np.ascontiguousarray(g.col_idx, dtype=np.uint32)
    hdr = json.dumps({"n": int(g.n), "nnz": int(g.nnz), "row_ptr_bytes": 8, "col_idx_bytes": 4,
                      "symmetric": bool(g.symmetric), "name": g.name, "params": g.params,
                      "generator": _generator_hash(), "checksum_row_ptr": checksum(rp),
                      "checksum_col_idx": checksum(ci)}, sort_keys=True).encode()
    off = -(-(16 + len(hdr)) // _ALIGN) * _ALIGN
    total = off + rp.nbytes + ci.nbytes
    d = os.path.dirname(path) or "."
    os.makedirs(d, exist_ok=True)
    if shutil.disk_usage(d).free < total + (1 << 30):
        return False
    tmp = f"{path}.tmp{os.getpid()}"
    try:
        with open(tmp, "wb") as f:
            f.write(_MAGIC)
            f.write(np.uint64(len(hdr)).tobytes())
            f.write(hdr)
            f.write(b"\0" * (off - 16 - len(hdr)))
            rp.tofile(f)
            ci.tofile(f)
        os.replace(tmp, path)
    except OSError:
        if os.path.exists(tmp):
            os.remove(tmp)
        return False
    return True


def load_graph(path: str) -> CSRGraph | None:
    """The graph stored at `path`, or None if the file is missing, truncated
    or fails a check (magic, sizes, row_ptr[n] = nnz, checksums)."""
    try:
        with open(path, "rb") as f:
            if f.read(8) != _MAGIC:
                return None
            hlen = int(np.frombuffer(f.read(8), dtype=np.uint64)[0])
            if hlen > (1 << 20):
                return None
            h = json.loads(f.read(hlen))
            n, nnz = int(h["n"]), int(h["nnz"])
            if h.get("row_ptr_bytes") != 8 or h.get("col_idx_bytes") != 4:
                return None
            off = -(-(16 + hlen) // _ALIGN) * _ALIGN
            if os.fstat(f.fileno()).st_size != off + 8 * (n + 1) + 4 * nnz:
                return None
            f.seek(off)
            rp = np.fromfile(f, dtype=np.uint64, count=n + 1)
            ci = np.fromfile(f, dtype=np.uint32, count=nnz)
    except (OSError, ValueError, KeyError, json.JSONDecodeError):
        return None
    if rp.size != n + 1 or ci.size != nnz or int(rp[-1]) != nnz:
        return None
    if checksum(rp) != h["checksum_row_ptr"] or checksum(ci) != h["checksum_col_idx"]:
        return None
    return CSRGraph(n, rp, ci, bool(h["symmetric"]), h["name"], dict(h["params"]))


def cached(builder: str, directory: str | None = None, **params) -> CSRGraph:
    """gen.<builder>(**params), read from the on-disk cache when a verified
    copy is there, else built and (room permitting) written to it."""
    path = _cache_path(builder, params, directory)
    g = load_graph(path)
    if g is not None:
        return g
    g = globals()[builder](**params)
    save_graph(g, path)
    return g


def permutation(n: int, key: int) -> np.ndarray:
    perm = np.empty(n, dtype=np.uint32)
    _L().khopgen_permutation(n, key, _p(perm))
    return perm


def seeds(g: CSRGraph, count: int, seed: int = 2) -> np.ndarray:
    """`count` seeds drawn uniformly with replacement from the vertices with
    out-degree > 0: seed i = eligible[floor(u_i * |eligible|)], u_i = draw i
    of stream `seed` (53-bit uniform)."""
    out = np.zeros(count, dtype=np.uint32)
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.uint64)
    ne = _L().khopgen_seeds(g.n, _p(rp), count, seed, _p(out))
    if ne < 0:
        raise MemoryError
    if ne == 0 and count:
        raise ValueError("graph has no vertex with out-degree > 0")
    return out


def mixed_ks(count: int, choices=(1, 2, 3, 6), seed: int = 2, stream: int = 7) -> np.ndarray:
    """k values drawn uniformly from `choices` (stream subkey(seed, stream))."""
    r = rand_array(subkey(seed, stream), 0, count)
    idx = ((r >> np.uint64(11)).astype(np.float64) * 2.0**-53 * len(choices)).astype(np.int64)
    idx = np.minimum(idx, len(choices) - 1)
    return np.asarray(choices, dtype=np.uint32)[idx]


def poisson_stream(g: CSRGraph, count: int, rate_qps: float, seed: int = 3,
                   k_probs=((1, 0.4), (2, 0.3), (3, 0.2), (6, 0.1))):
    """Open-loop request stream: arrival times (s) with exponential gaps of
    mean 1/rate, k drawn from k_probs, seeds uniform over out-degree > 0."""
    rp = g.row_ptr
    eligible = np.nonzero(rp[1:] > rp[:-1])[0].astype(np.uint32)
    vals = np.asarray([k for k, _ in k_probs], dtype=np.uint32)
    cdf = np.cumsum([p for _, p in k_probs]).astype(np.float64)
    t = np.empty(count, dtype=np.float64)
    ks = np.empty(count, dtype=np.uint32)
    sd = np.empty(count, dtype=np.uint32)
    _L().khopgen_poisson(count, float(rate_qps), seed, _p(cdf), _p(vals), len(vals),
                         eligible.size, _p(eligible), _p(t), _p(ks), _p(sd))
    return t, ks, sd


# --------------------------------------------------------------------------
# Small named graphs (test fixtures with closed-form answers).

def path_graph(n: int) -> CSRGraph:
    s = np.arange(max(n - 1, 0), dtype=np.uint32)
    return csr_from_edges(n, s, s + 1, name=f"path{n}")


def cycle_graph(n: int) -> CSRGraph:
    s = np.arange(n, dtype=np.uint32)
    return csr_from_edges(n, s, (s + 1) % n, name=f"cycle{n}")


def out_star(leaves: int) -> CSRGraph:
    d = np.arange(1, leaves + 1, dtype=np.uint32)
    return csr_from_edges(leaves + 1, np.zeros(leaves, np.uint32), d, name=f"ostar{leaves}")


def sym_star(leaves: int) -> CSRGraph:
    d = np.arange(1, leaves + 1, dtype=np.uint32)
    return csr_from_edges(leaves + 1, np.zeros(leaves, np.uint32), d, symmetrize=True,
                          name=f"sstar{leaves}")


def complete_graph(n: int) -> CSRGraph:
    a, b = np.meshgrid(np.arange(n, dtype=np.uint32), np.arange(n, dtype=np.uint32), indexing="ij")
    return csr_from_edges(n, a.ravel(), b.ravel(), name=f"complete{n}")


def empty_graph(n: int) -> CSRGraph:
    return CSRGraph(n, np.zeros(n + 1, np.uint64), np.zeros(0, np.uint32), True, f"empty{n}", {})


def disjoint_union(graphs) -> CSRGraph:
    """Vertex-disjoint union; graph i's vertices are offset by the sizes before it."""
    rps, cols, off_v, off_e = [np.zeros(1, np.uint64)], [], 0, 0
    for g in graphs:
        rps.append(g.row_ptr[1:] + np.uint64(off_e))
        cols.append(g.col_idx + np.uint32(off_v))
        off_v += g.n
        off_e += g.nnz
    col = np.concatenate(cols) if cols else np.zeros(0, np.uint32)
    return CSRGraph(off_v, np.concatenate(rps), col.astype(np.uint32),
                    all(g.symmetric for g in graphs), "union", {})
