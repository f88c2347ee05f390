"""Pins for the CPU oracle: checks against things other than the oracle itself.

* a hand-worked example (tests/golden/handworked8.txt);
* brute force: Boolean matrix powers on every digraph with n <= 4 (self-loops
  included) and n = 5 (no self-loops), and on random multigraphs n <= 64;
* closed forms for path, cycle, stars, complete and empty graphs;
* a library routine: scipy's unweighted shortest paths on the 1024-vertex
  R-MAT graph;
* invariants (monotone in k, <= n-1, 1-hop = distinct out-neighbours,
  stabilisation, components of symmetric graphs, per-hop sums);
* planted mistakes: mutated copies of the oracle source must fail the pins.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import tempfile

import numpy as np
import pytest

import gen
import oracle
from tests import brute

HERE = os.path.dirname(os.path.abspath(__file__))


def load_golden(path):
    edges, queries, n = [], [], None
    with open(path) as f:
        for line in f:
            t = line.split("#", 1)[0].split()
            if not t:
                continue
            if t[0] == "edge":
                edges.append((int(t[1]), int(t[2])))
            elif t[0] == "n":
                n = int(t[1])
            elif t[0] == "q":
                queries.append(tuple(int(x) for x in t[1:5]))
    src = [a for a, _ in edges]
    dst = [b for _, b in edges]
    return gen.csr_raw(n, src, dst), queries


def test_golden_handworked():
    g, queries = load_golden(os.path.join(HERE, "golden", "handworked8.txt"))
    seeds = [q[0] for q in queries]
    ks = [q[1] for q in queries]
    counts, te = oracle.khop_counts(g, seeds, ks)
    for i, (s, k, c, t) in enumerate(queries):
        assert int(counts[i]) == c, (s, k)
        assert int(te[i]) == t, (s, k)


def _check_stack(A, kmax, ks):
    G, n, _ = A.shape
    g = brute.union_csr_from_dense_stack(A)
    R = brute.reach_powers(A, kmax)
    outdeg = A.sum(axis=-1)
    seeds = np.arange(G * n, dtype=np.uint32)
    for k in ks:
        counts, te, ph = oracle.khop_counts(g, seeds, k, per_hop=True)
        want = brute.counts_from_reach(R[k - 1]).reshape(-1)
        np.testing.assert_array_equal(counts.astype(np.int64), want)
        want_te = brute.te_from_reach(R[k - 2] if k >= 2 else None, A, outdeg).reshape(-1)
        np.testing.assert_array_equal(te.astype(np.int64), want_te)
        np.testing.assert_array_equal(ph.astype(np.int64),
                                      brute.per_hop_from_reach(R, k).reshape(G * n, k + 1))
    c0, t0 = oracle.khop_counts(g, seeds[: 4 * n], 0)
    assert not c0.any() and not t0.any()


def test_exhaustive_n4_with_self_loops():
    _check_stack(brute.all_digraphs(4, self_loops=True), 6, [1, 2, 3, 4, 6])


def test_exhaustive_n3_with_self_loops():
    _check_stack(brute.all_digraphs(3, self_loops=True), 4, [1, 2, 3, 4])


def test_exhaustive_n5_no_self_loops():
    _check_stack(brute.all_digraphs(5, self_loops=False), 6, [1, 2, 3, 6])


def test_random_multigraphs_vs_matrix_powers():
    rng = np.random.default_rng(12345)
    for trial in range(60):
        n = int(rng.integers(1, 65))
        m = int(rng.integers(0, 4 * n + 1))
        src = rng.integers(0, n, m)
        dst = rng.integers(0, n, m)
        g = gen.csr_raw(n, src, dst)           # duplicates and self-loops kept
        A = brute.dense_from_csr(g)
        kset = sorted({1, 2, 3, 6, max(n, 1)})
        R = brute.reach_powers(A[None], kset[-1])
        outdeg = np.diff(g.row_ptr).astype(np.int64)[None]
        seeds = np.arange(n, dtype=np.uint32)
        for k in kset:
            counts, te, ph = oracle.khop_counts(g, seeds, k, per_hop=True)
            np.testing.assert_array_equal(counts.astype(np.int64),
                                          brute.counts_from_reach(R[k - 1])[0])
            np.testing.assert_array_equal(ph.astype(np.int64), brute.per_hop_from_reach(R, k)[0])
            np.testing.assert_array_equal(
                te.astype(np.int64),
                brute.te_from_reach(R[k - 2] if k >= 2 else None, A[None], outdeg)[0])


@pytest.mark.parametrize("n", [1, 2, 7, 33])
def test_closed_form_path(n):
    g = gen.path_graph(n)
    for s in range(n):
        for k in (0, 1, 2, 3, 6, n + 2):
            assert oracle.khop_count(g, s, k) == min(k, n - 1 - s)


@pytest.mark.parametrize("n", [2, 5, 32, 100])
def test_closed_form_cycle(n):
    g = gen.cycle_graph(n)
    for s in (0, n // 2, n - 1):
        for k in (0, 1, 2, 6, n - 1, n, n + 5):
            assert oracle.khop_count(g, s, k) == min(k, n - 1)


@pytest.mark.parametrize("L", [1, 5, 40])
def test_closed_form_stars(L):
    og, sg = gen.out_star(L), gen.sym_star(L)
    for k in (1, 2, 3, 6):
        assert oracle.khop_count(og, 0, k) == L
        assert oracle.khop_count(og, 1, k) == 0
        assert oracle.khop_count(sg, 0, k) == L
        assert oracle.khop_count(sg, L, k) == (1 if k == 1 else L)


def test_closed_form_complete_and_empty():
    for n in (1, 2, 6, 40):
        g = gen.complete_graph(n)
        e = gen.empty_graph(n)
        for s in range(n):
            for k in (1, 2, 6):
                assert oracle.khop_count(g, s, k) == n - 1
                assert oracle.khop_count(e, s, k) == 0
            assert oracle.khop_count(g, s, 0) == 0


def test_two_disjoint_cycles():
    g = gen.disjoint_union([gen.cycle_graph(7), gen.cycle_graph(11)])
    for s in range(18):
        size = 7 if s < 7 else 11
        for k in (1, 3, 6, 20):
            assert oracle.khop_count(g, s, k) == min(k, size - 1)


def test_out_of_range_seed():
    g = gen.path_graph(4)
    c, t = oracle.khop_counts(g, [4, 100], 2)
    assert (c == np.iinfo(np.uint64).max).all() and (t == np.iinfo(np.uint64).max).all()


def _scipy_dist(g, s):
    sp = pytest.importorskip("scipy.sparse")
    cg = pytest.importorskip("scipy.sparse.csgraph")
    data = np.ones(g.nnz, dtype=np.float64)
    M = sp.csr_matrix((data, g.col_idx.astype(np.int64), g.row_ptr.astype(np.int64)),
                      shape=(g.n, g.n))
    return cg.shortest_path(M, method="D", directed=True, unweighted=True, indices=int(s))


@pytest.mark.parametrize("symmetrize", [False, True])
def test_rmat_scale10_vs_library_shortest_paths(symmetrize):
    """The 1024-vertex R-MAT graph, 64 seeds, k in {1,2,3,6}, against scipy's
    unweighted shortest paths (a library BFS with no hop limit)."""
    g = gen.rmat(10, 16, seed=1, symmetrize=symmetrize)
    seeds = gen.seeds(g, 64, seed=2)
    outdeg = np.diff(g.row_ptr).astype(np.int64)
    dists = [_scipy_dist(g, s) for s in seeds]
    for k in (1, 2, 3, 6):
        counts, te, ph = oracle.khop_counts(g, seeds, k, per_hop=True)
        for i, s in enumerate(seeds):
            d = dists[i]
            reach = (d <= k) & np.isfinite(d)
            reach[s] = False
            assert int(counts[i]) == int(reach.sum())
            assert int(te[i]) == int(outdeg[np.isfinite(d) & (d < k)].sum())
            # per_hop[r] = vertices at library distance exactly r
            want_ph = [int((d == r).sum()) for r in range(k + 1)]
            assert ph[i].tolist() == want_ph, (int(s), k)


def _components(g):
    parent = np.arange(g.n)

    def find(x):
        while parent[x] != x:
            parent[x] = parent[parent[x]]
            x = parent[x]
        return x

    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr).astype(np.int64))
    for a, b in zip(rows.tolist(), g.col_idx.tolist()):
        ra, rb = find(a), find(b)
        if ra != rb:
            parent[ra] = rb
    roots = np.array([find(x) for x in range(g.n)])
    _, inv, cnt = np.unique(roots, return_inverse=True, return_counts=True)
    return cnt[inv]


def test_invariants_rmat_scale10_all_seeds():
    g = gen.rmat(10, 16, seed=1)
    n = g.n
    seeds = np.arange(n, dtype=np.uint32)
    ks = [0, 1, 2, 3, 4, 5, 6, 7, 8, 12, 40]
    res = {k: oracle.khop_counts(g, seeds, k)[0].astype(np.int64) for k in ks}
    for a, b in zip(ks, ks[1:]):
        assert (res[a] <= res[b]).all()                       # monotone in k
    assert (res[40] <= n - 1).all()
    for s in range(n):                                        # 1-hop = distinct out-nbrs
        row = g.col_idx[g.row_ptr[s]:g.row_ptr[s + 1]]
        assert res[1][s] == np.setdiff1d(np.unique(row), [s]).size
    for a, b in zip(ks[:-2], ks[1:-1]):                       # once flat, flat forever
        if b == a + 1:
            flat = res[a] == res[b]
            assert (res[40][flat] == res[a][flat]).all()
    c, te, ph = oracle.khop_counts(g, seeds, 6, per_hop=True)
    assert (ph[:, 0] == 1).all()
    np.testing.assert_array_equal(ph[:, 1:].sum(axis=1), c)  # sum over rounds of |q_r|


def test_invariants_symmetric_components_and_distance_symmetry():
    g = gen.rmat(10, 16, seed=1, symmetrize=True)
    n = g.n
    comp = _components(g)
    seeds = np.arange(n, dtype=np.uint32)
    c_inf, _ = oracle.khop_counts(g, seeds, n)
    np.testing.assert_array_equal(c_inf.astype(np.int64), comp - 1)
    rng = np.random.default_rng(7)
    for s in rng.choice(n, 12, replace=False):
        for k in (1, 2, 3):
            ds = oracle.khop_dist(g, int(s), k)
            for u in np.nonzero(ds >= 0)[0][:50]:
                du = oracle.khop_dist(g, int(u), k)
                assert du[s] >= 0 and du[s] == ds[u]


MUTANTS = [
    # hop limit off by one: expands vertices at distance k
    ("if ((uint32_t)du >= k) continue;", "if ((uint32_t)du > k) continue;"),
    # the seed is counted again when a cycle returns to it
    ("dist[s] = 0;\n    queue[tail++] = s;\n    if (per_hop)",
     "queue[tail++] = s;\n    if (per_hop)"),
    # out-degree of the wrong end: counts edges of vertices at distance <= k
    ("edges += row_ptr[u + 1] - row_ptr[u];\n        for",
     "for"),
    # per-hop bins shifted: a vertex at distance 2 lands in bin 1
    ("if (per_hop) per_hop[du + 1]++;", "if (per_hop) per_hop[du == 1 ? 1 : du + 1]++;"),
    # row end taken from the wrong index
    ("for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {\n            uint32_t w = col_idx[e];\n            if (dist[w] == UNSET) {\n                dist[w] = du + 1;",
     "for (uint64_t e = row_ptr[u]; e + 1 < row_ptr[u + 1]; ++e) {\n            uint32_t w = col_idx[e];\n            if (dist[w] == UNSET) {\n                dist[w] = du + 1;"),
]


@pytest.mark.parametrize("mi", range(len(MUTANTS)))
def test_planted_mistakes_are_caught(mi, monkeypatch, tmp_path):
    """A plausible mistake planted in a copy of the oracle source fails a pin."""
    src = open(oracle._SRC).read()
    a, b = MUTANTS[mi]
    assert a in src, "mutation site moved"
    mutated = src.replace(a, b, 1)
    if mi == 1:
        # the vertex still needs dist 0 once it is popped; set it after counting
        mutated = mutated.replace("int32_t du = dist[u];",
                                  "int32_t du = dist[u] < 0 ? 0 : dist[u];")
    cfile = tmp_path / "mut.c"
    cfile.write_text(mutated)
    so = tmp_path / "libmut.so"
    subprocess.run(["gcc", "-O1", "-std=gnu11", "-fPIC", "-shared", "-pthread", str(cfile),
                    "-o", str(so)], check=True)
    lib = ctypes.CDLL(str(so))
    vp, u64 = ctypes.c_void_p, ctypes.c_uint64
    lib.oracle_khop_many.restype = ctypes.c_int
    lib.oracle_khop_many.argtypes = [u64, vp, vp, vp, vp, u64, vp, vp, vp, u64, ctypes.c_int]
    lib.oracle_khop_dist.restype = ctypes.c_int
    lib.oracle_khop_dist.argtypes = [u64, vp, vp, ctypes.c_uint32, ctypes.c_uint32, vp]
    monkeypatch.setattr(oracle, "_lib", lib)
    failed = 0
    for check in (test_golden_handworked, test_exhaustive_n3_with_self_loops,
                  lambda: test_closed_form_cycle(5)):
        try:
            check()
        except AssertionError:
            failed += 1
    assert failed > 0


# ---- BFS levels and (MIN, SECOND) parents -----------------------------------

def test_parents_on_path_star_and_diamond():
    p = oracle.bfs_parents(gen.path_graph(8), 2, 3)
    assert p[2] == 2 and list(p[3:6]) == [2, 3, 4]
    assert (p[[0, 1, 6, 7]] == 0xFFFFFFFF).all()       # behind the seed, beyond k
    st = gen.out_star(6)
    assert (oracle.bfs_parents(st, 0, 1)[1:] == 0).all()
    # diamond 0->1, 0->2, 1->3, 2->3, 2->4: vertex 3 has two predecessors -> the smaller
    d = gen.csr_raw(5, [0, 0, 1, 2, 2], [1, 2, 3, 3, 4])
    assert list(oracle.bfs_parents(d, 0, 2)) == [0, 0, 0, 1, 2]
    assert list(oracle.bfs_parents(d, 0, 1)) == [0, 0, 0, 0xFFFFFFFF, 0xFFFFFFFF]


def test_levels_and_parents_against_networkx_bfs():
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(17)
    for _ in range(20):
        n = int(rng.integers(2, 60))
        m = int(rng.integers(0, 4 * n))
        src, dst = rng.integers(0, n, m), rng.integers(0, n, m)
        g = gen.csr_raw(n, src, dst)
        G = nx.DiGraph()
        G.add_nodes_from(range(n))
        G.add_edges_from(zip(src.tolist(), dst.tolist()))
        s, k = int(rng.integers(0, n)), int(rng.integers(0, 6))
        ref = nx.single_source_shortest_path_length(G, s, cutoff=k)
        d = oracle.khop_dist(g, s, k)
        assert {v: int(x) for v, x in enumerate(d) if x >= 0} == ref
        par = oracle.bfs_parents(g, s, k)
        for v in range(n):
            if v == s:
                assert par[v] == s
            elif v in ref:
                preds = [u for u in G.predecessors(v) if ref.get(u, -9) == ref[v] - 1]
                assert par[v] == min(preds)
            else:
                assert par[v] == 0xFFFFFFFF


# ---- masked matrix-vector products over semirings --------------------------

def _mult_matrix(g):
    """Dense edge-multiplicity matrix M[u, v] = number of stored edges u -> v."""
    M = np.zeros((g.n, g.n), dtype=np.int64)
    rp = np.asarray(g.row_ptr, dtype=np.int64)
    src = np.repeat(np.arange(g.n), np.diff(rp))
    np.add.at(M, (src, np.asarray(g.col_idx[: int(rp[-1])], dtype=np.int64)), 1)
    return M


def test_mxv_plus_times_iterated_counts_walks_like_matrix_powers():
    """PLUS_TIMES applied k times to e_s gives the number of walks of length k
    from s to each vertex: row s of M^k (numpy's matrix power of the
    multiplicity matrix; parallel edges are distinct walks)."""
    rng = np.random.default_rng(21)
    for trial in range(12):
        n = int(rng.integers(2, 40))
        m = int(rng.integers(0, 4 * n))
        g = gen.csr_raw(n, rng.integers(0, n, m), rng.integers(0, n, m))   # duplicates, self-loops
        M = _mult_matrix(g)
        for s in rng.choice(n, min(n, 4), replace=False):
            x = np.zeros(n, np.uint64)
            x[s] = 1
            for k in range(1, 6):
                x = oracle.mxv(g, oracle.SR_PLUS_TIMES, x)
                want = np.linalg.matrix_power(M, k)[s]
                np.testing.assert_array_equal(x.astype(np.int64), want)


def test_mxv_plus_times_wraps_mod_2_64():
    g = gen.csr_raw(3, [0, 1], [2, 2])
    x = np.array([2**63, 2**63 + 5, 0], np.uint64)
    y = oracle.mxv(g, oracle.SR_PLUS_TIMES, x)
    assert y.tolist() == [0, 0, 5]


def test_mxv_or_and_with_complemented_visited_mask_is_a_bfs_step():
    """Iterating q <- (A^T q) AND NOT v, v <- v OR q from e_s with OR_AND and the
    visited set as the complemented mask gives the vertices at each hop
    distance exactly (the k-hop count's own iteration), checked against the
    oracle's BFS distances and the matrix-power reach sets."""
    for g in (gen.rmat(8, 8, seed=3), gen.rmat(8, 8, seed=4, symmetrize=True)):
        A = brute.dense_from_csr(g)
        R = brute.reach_powers(A[None], 6)
        for s in (0, 5, 17, 200):
            d = oracle.khop_dist(g, s, 6)
            q = np.zeros(g.n, np.uint64)
            q[s] = 1
            vis = q.copy()
            for r in range(1, 7):
                words = np.zeros((g.n + 31) // 32, np.uint32)
                idx = np.nonzero(vis)[0]
                np.bitwise_or.at(words, idx >> 5, (np.uint32(1) << (idx & 31).astype(np.uint32)))
                q = oracle.mxv(g, oracle.SR_OR_AND, q, mask=words, complement=True)
                np.testing.assert_array_equal(np.nonzero(q)[0], np.nonzero(d == r)[0])
                reach = R[r - 1][0, s] | (np.arange(g.n) == s)
                prev = (R[r - 2][0, s] if r >= 2 else np.zeros(g.n, bool)) | (np.arange(g.n) == s)
                np.testing.assert_array_equal(q.astype(bool), reach & ~prev)
                vis = vis | q


def test_mxv_min_and_max_second_give_extreme_predecessors():
    """With x[u] = u on the frontier {u : dist(u) = r}, MIN_SECOND / MAX_SECOND
    masked to the unvisited vertices give, for every vertex at distance r+1,
    its smallest / largest in-neighbour at distance r (networkx BFS)."""
    nx = pytest.importorskip("networkx")
    rng = np.random.default_rng(23)
    for _ in range(15):
        n = int(rng.integers(2, 50))
        m = int(rng.integers(0, 4 * n))
        src, dst = rng.integers(0, n, m), rng.integers(0, n, m)
        g = gen.csr_raw(n, src, dst)
        G = nx.DiGraph()
        G.add_nodes_from(range(n))
        G.add_edges_from(zip(src.tolist(), dst.tolist()))
        s = int(rng.integers(0, n))
        dist = nx.single_source_shortest_path_length(G, s)
        for r in range(0, 4):
            front = [u for u, d in dist.items() if d == r]
            x_min = np.full(n, 2**64 - 1, np.uint64)
            x_max = np.zeros(n, np.uint64)
            x_min[front] = front
            x_max[front] = front
            words = np.zeros((n + 31) // 32, np.uint32)
            for u, d in dist.items():
                if d <= r:
                    words[u >> 5] |= np.uint32(1) << np.uint32(u & 31)
            y_min = oracle.mxv(g, oracle.SR_MIN_SECOND, x_min, mask=words, complement=True)
            y_max = oracle.mxv(g, oracle.SR_MAX_SECOND, x_max, mask=words, complement=True)
            for v in range(n):
                preds = [u for u in G.predecessors(v) if dist.get(u) == r]
                if dist.get(v, -1) == r + 1:
                    assert y_min[v] == min(preds) and y_max[v] == max(preds)
                elif dist.get(v, 99) <= r:          # masked out: the identity
                    assert y_min[v] == 2**64 - 1 and y_max[v] == 0


def test_mxv_mask_selects_outputs():
    g = gen.rmat(7, 8, seed=5)
    x = np.arange(g.n, dtype=np.uint64) + 1
    words = np.random.default_rng(1).integers(0, 2**32, (g.n + 31) // 32, dtype=np.uint64).astype(np.uint32)
    bits = ((words[np.arange(g.n) >> 5] >> (np.arange(g.n) & 31).astype(np.uint32)) & 1).astype(bool)
    full = oracle.mxv(g, oracle.SR_PLUS_TIMES, x)
    for comp in (False, True):
        y = oracle.mxv(g, oracle.SR_PLUS_TIMES, x, mask=words, complement=comp)
        sel = ~bits if comp else bits
        np.testing.assert_array_equal(y[sel], full[sel])
        assert (y[~sel] == 0).all()
