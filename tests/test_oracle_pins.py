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
