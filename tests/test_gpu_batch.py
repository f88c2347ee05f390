"""GPU parity of the 64-lane bit-sliced batched path.

Each lane's count must equal the oracle's (and the plain path's) exactly,
whatever the lane, the batch and the mix of k around it: the batched counts
are compared with the oracle on the same seeded inputs, and with themselves
under a permutation of the query order.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
kh = pytest.importorskip("paper_1905_01294_gb300")


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    kh.lib()


LANES = [kh.MODE_BATCHED64, kh.MODE_BATCHED128, kh.MODE_BATCHED256]   # 64, 128 or 256 queries per traversal
WIDTH = {kh.MODE_BATCHED64: 64, kh.MODE_BATCHED128: 128, kh.MODE_BATCHED256: 256}


def batched(G, seeds, ks, mode=kh.MODE_BATCHED64):
    out = G.count_mixed(np.asarray(seeds, np.uint32), np.asarray(ks, np.uint32),
                        mode=mode)
    torch.cuda.synchronize()
    return kh.as_u64(out)


def check(g, seeds, ks, wide=False, mode=kh.MODE_BATCHED64, **tune):
    G = kh.Graph.from_csr(g, wide=wide)
    if tune:
        G.set_tuning(**tune)
    seeds = np.asarray(seeds, np.uint32)
    ks = np.broadcast_to(np.asarray(ks, np.uint32), seeds.shape).copy()
    want, _ = oracle.khop_counts(g, seeds, np.minimum(ks, g.n + 1))
    got = batched(G, seeds, ks, mode)
    np.testing.assert_array_equal(got, want)
    # lane/batch invariance: a permuted query order gives the same per-query counts
    perm = np.random.default_rng(len(seeds)).permutation(len(seeds))
    got_p = batched(G, seeds[perm], ks[perm], mode)
    np.testing.assert_array_equal(got_p, want[perm])
    bits = G.error_bits()
    G.close()
    return bits


@pytest.mark.parametrize("mode", LANES)
def test_rmat_scale10_mixed_k(mode):
    g = gen.rmat(10, 16, seed=1)
    seeds = gen.seeds(g, 64, seed=2)
    ks = np.tile(np.array([1, 2, 3, 6], np.uint32), 16)
    assert check(g, seeds, ks, mode=mode) == 0


@pytest.mark.parametrize("mode", LANES)
@pytest.mark.parametrize("k", [1, 2, 3, 6])
def test_rmat_scale10_every_vertex(k, mode):
    g = gen.rmat(10, 16, seed=1)
    assert check(g, np.arange(g.n, dtype=np.uint32), k, mode=mode) == 0


@pytest.mark.parametrize("mode", LANES)
def test_symmetric_scale12_many_batches_wide(mode):
    g = gen.rmat(12, 16, seed=3, symmetrize=True)
    seeds = gen.seeds(g, 700, seed=4)
    ks = gen.mixed_ks(700, seed=5)
    assert check(g, seeds, ks, wide=True, mode=mode) == 0


@pytest.mark.parametrize("mode", LANES)
@pytest.mark.parametrize("alpha,beta,tile", [(1e-6, 1e6, 256), (1e6, 1e-6, 8192), (14, 24, 1024)])
def test_direction_extremes(alpha, beta, tile, mode):
    """alpha tiny: pull from round 2 on; alpha huge: push only."""
    g = gen.rmat(11, 16, seed=6)
    seeds = gen.seeds(g, 200, seed=7)
    ks = gen.mixed_ks(200, choices=(1, 2, 3, 4, 6), seed=8)
    assert check(g, seeds, ks, batch_alpha=alpha, batch_beta=beta, batch_push_tile=tile, mode=mode) == 0


@pytest.mark.parametrize("mode", LANES)
def test_edge_cases_k0_bad_seed_duplicates_and_sinks(mode):
    g = gen.csr_raw(40, [0, 0, 1, 2, 3, 3, 5, 5, 7], [1, 1, 2, 3, 0, 3, 5, 6, 7])
    seeds = np.array([0, 0, 0, 3, 39, 5, 7, 40, 1000, 2, 6, 1], np.uint32)
    ks = np.array([1, 2, 0, 6, 3, 2, 4, 2, 1, 2**31, 3, 5], np.uint32)
    G = kh.Graph.from_csr(g)
    got = batched(G, seeds, ks, mode)
    ok = seeds < g.n
    want, _ = oracle.khop_counts(g, seeds[ok], np.minimum(ks[ok], 100))
    np.testing.assert_array_equal(got[ok], want)
    assert (got[~ok] == np.uint64(2**64 - 1)).all()
    assert G.error_bits() & kh.DEVERR_SEED
    G.close()


@pytest.mark.parametrize("n", [1, 31, 33, 100])
def test_small_named_graphs(n):
    for g in (gen.path_graph(n), gen.cycle_graph(n), gen.complete_graph(min(n, 40)),
              gen.empty_graph(n), gen.sym_star(n)):
        seeds = np.arange(g.n, dtype=np.uint32)
        ks = (np.arange(g.n) % 7).astype(np.uint32)
        assert check(g, seeds, ks) == 0


@pytest.mark.parametrize("mode", LANES)
def test_random_multigraphs(mode):
    rng = np.random.default_rng(77)
    for _ in range(8):
        n = int(rng.integers(1, 400))
        m = int(rng.integers(0, 8 * n + 1))
        g = gen.csr_raw(n, rng.integers(0, n, m), rng.integers(0, n, m))
        nq = int(rng.integers(1, 200))
        seeds = rng.integers(0, n, nq).astype(np.uint32)
        ks = rng.choice([0, 1, 2, 3, 6, 9], nq).astype(np.uint32)
        assert check(g, seeds, ks, mode=mode) == 0


@pytest.fixture(scope="module")
def scale21_mixed():
    """The batched benchmark workload: the scale-21 symmetrized Kronecker
    graph, 4096 seeds (stream 2) with k uniform over {1,2,3,6}, and the
    oracle's count for every one of them (all host cores, one query per
    thread)."""
    g = gen.rmat(21, 16, seed=1, symmetrize=True)
    seeds = gen.seeds(g, 4096, seed=2)
    ks = gen.mixed_ks(4096, seed=2)
    want, _ = oracle.khop_counts(g, seeds, ks, with_te=False)
    G = kh.Graph.from_csr(g)
    yield g, G, seeds, ks, want
    G.close()


@pytest.mark.parametrize("mode", LANES)
def test_scale21_mixed_workload_every_count_equals_the_oracle(scale21_mixed, mode):
    """All 4096 batched counts of the benchmark's batched leg equal the
    oracle's, at every lane width, in the tuning the benchmark times (the
    graph tuned as the benchmark tunes it, bench.tune_graph); the plain path agrees
    on the same queries."""
    g, G, seeds, ks, want = scale21_mixed
    if mode == kh.MODE_BATCHED64:
        import bench
        bench.tune_graph(G, g)
        plain = G.count_mixed(seeds, ks, mode=kh.MODE_PLAIN)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(kh.as_u64(plain), want)
    got = batched(G, seeds, ks, mode)
    np.testing.assert_array_equal(got, want)
    assert G.error_bits() == 0


@pytest.mark.parametrize("mode", LANES)
def test_long_in_lists_deferred_to_chunks(mode):
    """A hub with 10,000 in-edges that the lanes seeded in a separate cycle
    never reach: with pull from round 2 on, every pull round scans the hub's
    whole in-list for those lanes (the chunked path), and counts still match."""
    L = 10000
    hub = 0
    leaves = np.arange(1, L + 1, dtype=np.uint32)
    src = [leaves, np.array([hub, hub], np.uint32), leaves[:-1]]
    dst = [np.full(L, hub, np.uint32), np.array([L + 1, 1], np.uint32), leaves[1:]]
    cyc = np.arange(L + 2, L + 40, dtype=np.uint32)
    src.append(cyc)
    dst.append(np.append(cyc[1:], cyc[0]).astype(np.uint32))
    g = gen.csr_from_edges(L + 40, np.concatenate(src), np.concatenate(dst))
    seeds = np.concatenate([np.array([5, 17, 300, 9999, hub, L + 1], np.uint32),
                            np.arange(L + 2, L + 40, dtype=np.uint32)])
    ks = np.tile(np.array([1, 2, 3, 6, 9], np.uint32), len(seeds))[:len(seeds)]
    for alpha in (1e-6, 14.0):
        assert check(g, seeds, ks, batch_alpha=alpha, batch_beta=1e-6, mode=mode) == 0


def test_captured_cuda_graph_replays_batched_and_plain():
    """Both paths captured in a CUDA graph (after a first direct call) and
    replayed twice give the direct call's counts."""
    g = gen.rmat(12, 16, seed=9, symmetrize=True)
    G = kh.Graph.from_csr(g)
    seeds = gen.seeds(g, 300, seed=1)
    ks = gen.mixed_ks(300, seed=3)
    s = torch.from_numpy(seeds.view(np.int32)).cuda()
    k = torch.from_numpy(ks.view(np.int32)).cuda()
    want, _ = oracle.khop_counts(g, seeds, ks)
    for mode in (kh.MODE_BATCHED64, kh.MODE_BATCHED128, kh.MODE_BATCHED256, kh.MODE_PLAIN):
        out = torch.zeros(300, dtype=torch.int64, device="cuda")
        side = torch.cuda.Stream()
        with torch.cuda.stream(side):
            kh.khop_count_mixed(G.handle, s.data_ptr(), k.data_ptr(), 300, out.data_ptr(), mode,
                                side.cuda_stream)
        torch.cuda.synchronize()
        np.testing.assert_array_equal(kh.as_u64(out), want)
        graph = torch.cuda.CUDAGraph()
        out.zero_()
        with torch.cuda.graph(graph, stream=side):
            kh.khop_count_mixed(G.handle, s.data_ptr(), k.data_ptr(), 300, out.data_ptr(), mode,
                                side.cuda_stream)
        for _ in range(2):
            out.zero_()
            graph.replay()
            torch.cuda.synchronize()
            np.testing.assert_array_equal(kh.as_u64(out), want)
    assert G.error_bits() == 0
    G.close()


def _spread(g, n, seed):
    """g's vertices relabelled to a seeded sorted sample of range(n)."""
    ids = np.sort(np.random.default_rng(seed).choice(n, g.n, replace=False)).astype(np.uint32)
    deg = np.diff(g.row_ptr).astype(np.int64)
    src = np.repeat(np.arange(g.n, dtype=np.uint32), deg)
    return gen.csr_from_edges(n, ids[src], ids[g.col_idx]), ids


@pytest.mark.parametrize("mode", LANES)
def test_sparse_id_space_several_harvest_flushes(mode):
    """A 4096-vertex R-MAT graph spread over 6M vertex ids: the harvest
    sweeps every id (dozens of steps per thread, so its bit-sliced counters
    are summed more than once) and every count still equals the oracle's and
    the plain path's."""
    g, ids = _spread(gen.rmat(12, 16, seed=5, symmetrize=True), 6_000_000, seed=6)
    seeds = gen.seeds(g, 128, seed=7)
    ks = np.tile(np.array([1, 2, 3, 6], np.uint32), 32)
    assert check(g, seeds, ks, mode=mode) == 0
    G = kh.Graph.from_csr(g)
    plain = G.count_mixed(seeds, ks, mode=kh.MODE_PLAIN)
    torch.cuda.synchronize()
    want, _ = oracle.khop_counts(g, seeds, ks)
    np.testing.assert_array_equal(kh.as_u64(plain), want)
    G.close()


@pytest.mark.parametrize("mode", LANES)
def test_strided_star_fills_every_counter_plane(mode):
    """A symmetric star whose leaves are the multiples of 512 in 6M ids: for
    any grid of 512-thread CTAs a harvest thread meets a leaf at every step,
    so each lane's counters run through all their planes between flushes."""
    n = 6_000_000
    hub = 1
    leaves = np.arange(0, n, 512, dtype=np.uint32)
    src = np.concatenate([np.full(leaves.size, hub, np.uint32), leaves])
    dst = np.concatenate([leaves, np.full(leaves.size, hub, np.uint32)])
    g = gen.csr_from_edges(n, src, dst)
    lanes = WIDTH[mode]
    seeds = np.array([hub] * (lanes // 2) + list(leaves[: lanes // 2]), np.uint32)
    ks = np.array([1, 2] * (lanes // 4) + [2] * (lanes // 2), np.uint32)
    want, _ = oracle.khop_counts(g, seeds, ks)
    assert set(want.tolist()) == {leaves.size}   # hub: its leaves; leaf at k=2: hub + other leaves
    G = kh.Graph.from_csr(g)
    np.testing.assert_array_equal(batched(G, seeds, ks, mode), want)
    assert G.error_bits() == 0
    G.close()
