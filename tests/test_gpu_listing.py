"""GPU parity of the k-hop neighbourhood as a set (khop_neighbourhood bitmap
and khop_neighbourhood_list ids) with the oracle's hop distances: v is in the
set iff dist(s, v) <= k, the seed included; the count equals the plain count;
the id list is ascending and truncates at the capacity.  Directed, symmetric,
reverse and either-direction graphs; seeds below and above the fused-round
degree bound; k = 0 and seeds without out-edges."""
import numpy as np
import pytest

import gen
import oracle
from tests import variants

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
kh = pytest.importorskip("paper_1905_01294_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    kh.lib()


def want_set(h, s, k):
    d = oracle.khop_dist(h, int(s), int(k))
    return np.nonzero(d >= 0)[0].astype(np.uint32)


def bits_to_ids(bits, n):
    b = bits.cpu().numpy().view(np.uint32)
    v = np.unpackbits(b.view(np.uint8), bitorder="little")[:n]
    return np.nonzero(v)[0].astype(np.uint32)


def check_sets(g, seeds, ks, **kw):
    h = g
    if kw.get("undirected") and not g.symmetric:
        h = variants.either_direction(g)
    elif kw.get("reverse") and not g.symmetric:
        h = variants.transpose(g)
    G = kh.Graph.from_csr(g, **kw)
    try:
        for s, k in zip(seeds, ks):
            want = want_set(h, s, k)
            bits, cnt = G.neighbourhood(s, k)
            ids, size = G.neighbourhood_list(s, k)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(bits_to_ids(bits, g.n), want, err_msg=f"bitmap s={s} k={k}")
            assert int(cnt.item()) == want.size - 1
            assert int(size.item()) == want.size
            np.testing.assert_array_equal(ids.cpu().numpy().view(np.uint32), want, err_msg=f"ids s={s} k={k}")
            if want.size > 3:   # truncated listing: the first ids, full size
                ids3, size3 = G.neighbourhood_list(s, k, capacity=3)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(ids3.cpu().numpy().view(np.uint32), want[:3])
                assert int(size3.item()) == want.size
        # the plain counts agree with the sets
        c = kh.as_u64(G.count_mixed(np.asarray(seeds, np.uint32), np.asarray(ks, np.uint32),
                                    mode=kh.MODE_PLAIN))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(c, [want_set(h, s, k).size - 1 for s, k in zip(seeds, ks)])
        assert G.error_bits() == 0
    finally:
        G.close()


def test_directed_and_symmetric_rmat():
    for sym in (False, True):
        g = gen.rmat(10, 16, seed=2, symmetrize=sym)
        rng = np.random.default_rng(3)
        seeds = rng.integers(0, g.n, 24).astype(np.uint32)
        ks = rng.choice([0, 1, 2, 3, 6, 50], 24).astype(np.uint32)
        check_sets(g, seeds, ks)


def test_reverse_and_either_direction():
    g = gen.rmat(10, 8, seed=5)
    seeds = np.arange(0, g.n, 97, dtype=np.uint32)
    ks = np.resize(np.array([1, 2, 3, 6], np.uint32), seeds.size)
    check_sets(g, seeds, ks, reverse=True)
    check_sets(g, seeds, ks, undirected=True)


def test_hub_above_the_fused_bound_self_loops_and_sinks():
    rng = np.random.default_rng(8)
    n = 5000
    src = np.concatenate([np.zeros(3000, np.int64), rng.integers(1, 2500, 8000), [7, 7]])
    dst = np.concatenate([rng.integers(0, n, 3000), rng.integers(0, n, 8000), [7, 7]])
    g = gen.csr_raw(n, src, dst)
    seeds = np.array([0, 0, 0, 7, 1, 4999, 2600], np.uint32)   # 4999, 2600: no out-edges
    ks = np.array([1, 2, 3, 2, 6, 3, 1], np.uint32)
    check_sets(g, seeds, ks)
    check_sets(g, seeds, ks, wide=True)


def test_rejects_bad_seed():
    g = gen.rmat(8, 8, seed=1)
    G = kh.Graph.from_csr(g)
    with pytest.raises(kh.KhopError):
        G.neighbourhood(g.n, 2)
    G.close()


def test_tiny_and_edgeless_graphs():
    for g in (gen.empty_graph(1), gen.empty_graph(33), gen.csr_raw(2, [0, 0], [0, 1]),
              gen.path_graph(2)):
        G = kh.Graph.from_csr(g)
        for s in range(g.n):
            for k in (0, 1, 3):
                want = want_set(g, s, k)
                bits, cnt = G.neighbourhood(s, k)
                ids, size = G.neighbourhood_list(s, k)
                lv, par = G.levels(s, k)
                torch.cuda.synchronize()
                np.testing.assert_array_equal(bits_to_ids(bits, g.n), want)
                np.testing.assert_array_equal(ids.cpu().numpy().view(np.uint32), want)
                assert int(size.item()) == want.size and int(cnt.item()) == want.size - 1
                np.testing.assert_array_equal(lv.cpu().numpy(), oracle.khop_dist(g, s, k))
                np.testing.assert_array_equal(par.cpu().numpy().view(np.uint32),
                                              oracle.bfs_parents(g, s, k))
        G.close()
