"""GPU parity of khop_mxv (y = A^T x over a semiring, masked): every output
equals the oracle's edge-by-edge fold bit for bit (integers: tolerance 0),
for all four semirings, with no mask, a mask and its complement, on directed
and symmetric R-MAT graphs, random multigraphs with duplicate edges and
self-loops, n not a multiple of 32, an empty graph, hubs whose in-lists take
the warp-wide pass, 32- and 64-bit edge offsets, and reverse and
either-direction graphs; iterated forms (walk counts, a BFS step, parents)
agree too."""
import numpy as np
import pytest

import gen
import oracle
from tests import variants

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
kh = pytest.importorskip("paper_1905_01294_gb300")

SEMIRINGS = [kh.SR_OR_AND, kh.SR_PLUS_TIMES, kh.SR_MIN_SECOND, kh.SR_MAX_SECOND]
U64MAX = 2**64 - 1


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    kh.lib()


def rand_x(n, sr, rng):
    x = rng.integers(0, 2**63, n, dtype=np.uint64) * np.uint64(2) + rng.integers(0, 2, n, dtype=np.uint64)
    ident = np.uint64(U64MAX) if sr == kh.SR_MIN_SECOND else np.uint64(0)
    x[rng.random(n) < 0.3] = ident          # "no entry" for a third of the vertices
    return x


def check(g, seed=0, **kw):
    h = g
    if kw.get("undirected") and not g.symmetric:
        h = variants.either_direction(g)
    elif kw.get("reverse") and not g.symmetric:
        h = variants.transpose(g)
    rng = np.random.default_rng(seed)
    G = kh.Graph.from_csr(g, **kw)
    try:
        words = rng.integers(0, 2**32, max((g.n + 31) // 32, 1), dtype=np.uint64).astype(np.uint32)
        for sr in SEMIRINGS:
            x = rand_x(g.n, sr, rng)
            for mask, comp in ((None, False), (words, False), (words, True)):
                y = kh.as_u64(G.mxv(sr, x, mask=mask, complement=comp))
                want = oracle.mxv(h, sr, x, mask=mask, complement=comp)
                np.testing.assert_array_equal(y, want, err_msg=f"semiring {sr} mask {mask is not None} comp {comp}")
    finally:
        G.close()


@pytest.mark.parametrize("wide", [False, True])
def test_rmat_directed_and_symmetric(wide):
    check(gen.rmat(10, 16, seed=1), wide=wide)
    check(gen.rmat(12, 16, seed=2, symmetrize=True), seed=1, wide=wide)


def test_random_multigraphs_and_small_sizes():
    rng = np.random.default_rng(5)
    for trial in range(20):
        n = int(rng.integers(1, 130))
        m = int(rng.integers(0, 6 * n))
        check(gen.csr_raw(n, rng.integers(0, n, m), rng.integers(0, n, m)), seed=trial)
    for n in (1, 31, 33, 65):
        check(gen.cycle_graph(n), seed=n)
    check(gen.empty_graph(40))


def test_hubs_with_long_in_lists():
    """In-lists of thousands of edges (a symmetric star's centre, a dense
    block) take the warp-wide pass, including the OR_AND early stop."""
    check(gen.sym_star(5000))
    rng = np.random.default_rng(9)
    src = np.concatenate([rng.integers(0, 3000, 20000), np.arange(3000)])
    dst = np.concatenate([rng.integers(0, 8, 20000), np.full(3000, 7)])
    check(gen.csr_raw(3000, src, dst), seed=3)


@pytest.mark.parametrize("kw", [{"reverse": True}, {"undirected": True}])
def test_reverse_and_either_direction_graphs(kw):
    check(gen.rmat(10, 16, seed=3), seed=4, **kw)


def test_iterated_walk_counts_bfs_step_and_parents():
    """Iterated from e_s, PLUS_TIMES counts walks (as the oracle's iterates);
    OR_AND with the complemented visited mask steps the BFS frontier (the
    k-hop count's iteration: the union of the frontiers has the count's size);
    MIN_SECOND on the frontier's ids gives the (MIN, SECOND) BFS parents."""
    g = gen.rmat(11, 16, seed=6)
    G = kh.Graph.from_csr(g)
    s = int(gen.seeds(g, 1, seed=7)[0])
    x = np.zeros(g.n, np.uint64)
    x[s] = 1
    xd = torch.from_numpy(x.view(np.int64)).cuda()
    for _ in range(4):
        xd = G.mxv(kh.SR_PLUS_TIMES, xd)
        x = oracle.mxv(g, oracle.SR_PLUS_TIMES, x)
    np.testing.assert_array_equal(kh.as_u64(xd), x)
    # BFS: q <- (A^T q) AND NOT v for 4 rounds
    q = np.zeros(g.n, np.uint64)
    q[s] = 1
    vis = q.astype(bool)
    for r in range(4):
        words = np.zeros((g.n + 31) // 32, np.uint32)
        idx = np.nonzero(vis)[0]
        np.bitwise_or.at(words, idx >> 5, np.uint32(1) << (idx & 31).astype(np.uint32))
        q = kh.as_u64(G.mxv(kh.SR_OR_AND, q, mask=words, complement=True)).copy()
        vis |= q.astype(bool)
    want, _ = oracle.khop_counts(g, [s], 4)
    assert int(vis.sum()) - 1 == int(want[0])
    # parents of the vertices at distance 2 from the frontier at distance 1
    d = oracle.khop_dist(g, s, 4)
    xm = np.full(g.n, U64MAX, np.uint64)
    xm[d == 1] = np.nonzero(d == 1)[0].astype(np.uint64)
    words = np.zeros((g.n + 31) // 32, np.uint32)
    idx = np.nonzero((d >= 0) & (d <= 1))[0]
    np.bitwise_or.at(words, idx >> 5, np.uint32(1) << (idx & 31).astype(np.uint32))
    par = kh.as_u64(G.mxv(kh.SR_MIN_SECOND, xm, mask=words, complement=True))
    want_par = oracle.bfs_parents(g, s, 4)
    at2 = d == 2
    np.testing.assert_array_equal(par[at2], want_par[at2].astype(np.uint64))
    assert G.error_bits() == 0
    G.close()


def test_invalid_arguments():
    g = gen.rmat(6, 4, seed=1)
    G = kh.Graph.from_csr(g)
    y = torch.empty(g.n, dtype=torch.int64, device="cuda")
    with pytest.raises(kh.KhopError) as e:
        kh.khop_mxv(G.handle, 7, y.data_ptr(), None, 0, y.data_ptr(), 0)
    assert e.value.status == kh.EINVAL
    with pytest.raises(kh.KhopError):
        kh.khop_mxv(G.handle, kh.SR_OR_AND, None, None, 0, y.data_ptr(), 0)
    G.close()
