"""GPU parity of the in-neighbourhood (KHOP_REVERSE) and either-direction
(KHOP_UNDIRECTED) counts with the CPU oracle run on the transposed / both-
direction graph built on the host (tests/variants.py): counts, TE and per-hop
counts of the plain path in every direction mode, and the batched path, on
directed graphs with duplicate edges, self-loops and sinks."""
import numpy as np
import pytest

import gen
import oracle
from tests import variants

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
kh = pytest.importorskip("paper_1905_01294_gb300")

MODES = [kh.DIR_AUTO, kh.DIR_PUSH, kh.DIR_PULL]


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    kh.lib()


def check_variant(g, seeds, ks, reverse=False, undirected=False, wide=False):
    h = variants.either_direction(g) if undirected else (variants.transpose(g) if reverse else g)
    seeds = np.asarray(seeds, np.uint32)
    ks = np.broadcast_to(np.asarray(ks, np.uint32), seeds.shape).copy()
    want_c, want_te, want_ph = oracle.khop_counts(h, seeds, ks, per_hop=True)
    G = kh.Graph.from_csr(g, reverse=reverse, undirected=undirected, wide=wide)
    try:
        for d in MODES:
            G.set_tuning(direction=d)
            res = G.count_ex(seeds, ks, hop_stride=want_ph.shape[1])
            torch.cuda.synchronize()
            np.testing.assert_array_equal(kh.as_u64(res["counts"]), want_c, err_msg=f"counts dir {d}")
            np.testing.assert_array_equal(kh.as_u64(res["te"]), want_te, err_msg=f"te dir {d}")
            ph = kh.as_u64(res["per_hop"]).reshape(len(seeds), -1)
            np.testing.assert_array_equal(ph, want_ph, err_msg=f"per-hop dir {d}")
        G.set_tuning(direction=kh.DIR_AUTO)
        got_b = kh.as_u64(G.count_mixed(seeds, ks, mode=kh.MODE_BATCHED64))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got_b, want_c, err_msg="batched")
        assert G.error_bits() == 0
    finally:
        G.close()


@pytest.mark.parametrize("reverse,undirected", [(True, False), (False, True), (True, True)])
def test_directed_rmat_scale11(reverse, undirected):
    g = gen.rmat(11, 16, seed=7)
    seeds = np.arange(0, g.n, 5, dtype=np.uint32)
    ks = gen.mixed_ks(seeds.size, choices=(0, 1, 2, 3, 6), seed=4)
    check_variant(g, seeds, ks, reverse=reverse, undirected=undirected)


@pytest.mark.parametrize("reverse,undirected", [(True, False), (False, True)])
def test_multigraphs_with_duplicates_self_loops_and_sinks(reverse, undirected):
    rng = np.random.default_rng(11)
    for _ in range(8):
        n = int(rng.integers(1, 400))
        m = int(rng.integers(0, 5 * n + 1))
        src = rng.integers(0, max(n // 2, 1), m)          # the upper half has no out-edges
        dst = rng.integers(0, n, m)
        g = gen.csr_raw(n, src, dst)
        seeds = rng.integers(0, n, 40).astype(np.uint32)
        ks = rng.choice([1, 2, 3, 6, 50], 40).astype(np.uint32)
        check_variant(g, seeds, ks, reverse=reverse, undirected=undirected)


def test_stars_paths_and_wide_offsets():
    for g in (gen.out_star(3000), gen.path_graph(700)):
        seeds = np.arange(0, g.n, 7, dtype=np.uint32)
        for k in (1, 2, 6):
            check_variant(g, seeds, k, reverse=True)
            check_variant(g, seeds, k, undirected=True, wide=True)


def test_undirected_of_a_symmetric_graph_is_the_graph():
    g = gen.rmat(10, 8, seed=3, symmetrize=True)
    seeds = np.arange(0, g.n, 3, dtype=np.uint32)
    want, _ = oracle.khop_counts(g, seeds, 3)
    for kw in ({"undirected": True}, {"reverse": True}):
        G = kh.Graph.from_csr(g, **kw)
        got = kh.as_u64(G.count(seeds, 3))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got, want)
        G.close()
