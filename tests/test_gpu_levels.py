"""GPU parity of khop_levels: hop levels equal the oracle's distances (-1
beyond k) and the (MIN, SECOND) BFS parents equal the oracle's, bit for bit,
on directed, symmetric, reverse and either-direction graphs, with duplicate
edges, self-loops, sinks and hubs above the fused-round degree bound."""
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


def check_levels(g, seeds, ks, **kw):
    h = g
    if kw.get("undirected") and not g.symmetric:
        h = variants.either_direction(g)
    elif kw.get("reverse") and not g.symmetric:
        h = variants.transpose(g)
    G = kh.Graph.from_csr(g, **kw)
    try:
        for s, k in zip(seeds, ks):
            for d in (kh.DIR_AUTO, kh.DIR_PUSH, kh.DIR_PULL):
                G.set_tuning(direction=d)
                lv, par = G.levels(int(s), int(k))
                torch.cuda.synchronize()
                np.testing.assert_array_equal(lv.cpu().numpy(), oracle.khop_dist(h, int(s), int(k)),
                                              err_msg=f"levels s={s} k={k} dir={d}")
                np.testing.assert_array_equal(par.cpu().numpy().view(np.uint32),
                                              oracle.bfs_parents(h, int(s), int(k)),
                                              err_msg=f"parents s={s} k={k} dir={d}")
        assert G.error_bits() == 0
    finally:
        G.close()


def test_rmat_directed_and_symmetric():
    for sym in (False, True):
        g = gen.rmat(10, 16, seed=4, symmetrize=sym)
        rng = np.random.default_rng(6)
        seeds = rng.integers(0, g.n, 10).astype(np.uint32)
        ks = rng.choice([0, 1, 2, 3, 6], 10).astype(np.uint32)
        check_levels(g, seeds, ks)


def test_reverse_either_direction_and_wide():
    g = gen.rmat(9, 8, seed=2)
    seeds = np.arange(0, g.n, 61, dtype=np.uint32)
    ks = np.resize(np.array([1, 2, 4], np.uint32), seeds.size)
    check_levels(g, seeds, ks, reverse=True)
    check_levels(g, seeds, ks, undirected=True, wide=True)


def test_multigraph_hub_self_loops_sinks():
    rng = np.random.default_rng(12)
    n = 3000
    src = np.concatenate([np.zeros(2500, np.int64), rng.integers(1, 1500, 6000), [5, 5]])
    dst = np.concatenate([rng.integers(0, n, 2500), rng.integers(0, n, 6000), [5, 5]])
    g = gen.csr_raw(n, src, dst)
    check_levels(g, np.array([0, 5, 1, 2999], np.uint32), np.array([3, 2, 6, 2], np.uint32))
