"""GPU parity of the plain single-query path against the CPU oracle.

Every count (and TE, per-hop count) must equal the oracle's bit for bit, in
every direction mode (Beamer switch, push only, pull only), for 32- and 64-bit
edge offsets, several push-tile and CTA sizes (many tiles, ragged tails), and
the degenerate cases (k = 0, huge k, seeds without out-edges, seeds >= n, n
not a multiple of 32, n = 1, empty graphs, duplicate edges and self-loops).
All calls go through the C ABI.
"""
import os

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
kh = pytest.importorskip("paper_1905_01294_gb300")

MODES = [("auto", kh.DIR_AUTO), ("push", kh.DIR_PUSH), ("pull", kh.DIR_PULL)]
U64MAX = np.uint64(2**64 - 1)
HERE = os.path.dirname(os.path.abspath(__file__))


@pytest.fixture(scope="module", autouse=True)
def _device():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    kh.lib()


def gpu_counts(G, seeds, ks, direction=kh.DIR_AUTO, hop_stride=0, **tune):
    G.set_tuning(direction=direction, **tune)
    res = G.count_ex(np.asarray(seeds, np.uint32),
                     np.broadcast_to(np.asarray(ks, np.uint32), np.shape(seeds)),
                     te=True, stats=True, hop_stride=hop_stride)
    torch.cuda.synchronize()
    out = {k: kh.as_u64(v) for k, v in res.items()}
    return out


def check_graph(g, seeds, ks, modes=MODES, wide=False, hop=False, **tune):
    G = kh.Graph.from_csr(g, wide=wide)
    try:
        ks = np.broadcast_to(np.asarray(ks, np.uint32), np.shape(seeds))
        want_c, want_te, want_ph = oracle.khop_counts(g, seeds, ks, per_hop=True)
        for name, d in modes:
            stride = want_ph.shape[1] if hop else 0
            got = gpu_counts(G, seeds, ks, d, hop_stride=stride, **tune)
            np.testing.assert_array_equal(got["counts"], want_c, err_msg=f"counts ({name})")
            np.testing.assert_array_equal(got["te"], want_te, err_msg=f"te ({name})")
            if hop:
                ph = got["per_hop"].reshape(len(seeds), stride)
                np.testing.assert_array_equal(ph, want_ph, err_msg=f"per-hop ({name})")
            # plain khop_count with a uniform k agrees too
            if len(set(ks.tolist())) == 1 and len(seeds):
                c = kh.as_u64(G.count(np.asarray(seeds, np.uint32), int(ks[0])))
                np.testing.assert_array_equal(c, want_c, err_msg=f"khop_count ({name})")
        assert G.error_bits() == 0
    finally:
        G.close()


def test_golden_handworked():
    from tests.test_oracle_pins import load_golden
    g, queries = load_golden(os.path.join(HERE, "golden", "handworked8.txt"))
    seeds = np.array([q[0] for q in queries], np.uint32)
    ks = np.array([q[1] for q in queries], np.uint32)
    G = kh.Graph.from_csr(g)
    for name, d in MODES:
        got = gpu_counts(G, seeds, ks, d)
        assert got["counts"].tolist() == [q[2] for q in queries], name
        assert got["te"].tolist() == [q[3] for q in queries], name
    G.close()


@pytest.mark.parametrize("wide", [False, True])
def test_rmat_scale10_seeds(wide):
    """The 1024-vertex R-MAT graph (edge factor 16, A/B/C/D = .57/.19/.19/.05,
    seed 1, directed), 64 seeds (seed 2) x k in {1, 2, 3, 6}."""
    g = gen.rmat(10, 16, seed=1)
    seeds = gen.seeds(g, 64, seed=2)
    for k in (1, 2, 3, 6):
        check_graph(g, seeds, k, wide=wide, hop=True)


def test_rmat_scale10_every_vertex():
    g = gen.rmat(10, 16, seed=1)
    seeds = np.arange(g.n, dtype=np.uint32)
    for k in (1, 2, 3, 6):
        check_graph(g, seeds, k)


def test_rmat_symmetric_flag_equals_derived_csc():
    g = gen.rmat(11, 16, seed=4, symmetrize=True)
    seeds = gen.seeds(g, 48, seed=2)
    ks = gen.mixed_ks(48, seed=5)
    check_graph(g, seeds, ks)                              # CSC = CSR (KHOP_SYMMETRIC)
    g2 = gen.CSRGraph(g.n, g.row_ptr, g.col_idx, False)   # CSC derived on the device
    check_graph(g2, seeds, ks)


@pytest.mark.parametrize("tile,block,per_sm", [(256, 256, 1), (8192, 1024, 1), (512, 512, 0),
                                               (2048, 256, 4)])
def test_tilings_and_grids(tile, block, per_sm):
    g = gen.rmat(12, 16, seed=3, symmetrize=True)
    seeds = gen.seeds(g, 24, seed=7)
    check_graph(g, seeds, gen.mixed_ks(24, seed=8), push_tile=tile, block_threads=block,
                blocks_per_sm=per_sm)


def test_directed_rmat_wide_offsets_mixed_k():
    g = gen.rmat(13, 8, seed=9)
    seeds = gen.seeds(g, 40, seed=2)
    ks = np.array([1, 2, 3, 4, 5, 6, 8, 30] * 5, np.uint32)
    check_graph(g, seeds, ks, wide=True, hop=True)


@pytest.mark.parametrize("n", [1, 2, 31, 32, 33, 65, 100])
def test_small_named_graphs(n):
    for g in (gen.path_graph(n), gen.cycle_graph(n), gen.complete_graph(min(n, 40)),
              gen.empty_graph(n)):
        seeds = np.arange(g.n, dtype=np.uint32)
        for k in (0, 1, 2, 3, 6, g.n + 1):
            check_graph(g, seeds, k)


def test_stars_and_unions():
    gs = [gen.out_star(70), gen.sym_star(70),
          gen.disjoint_union([gen.cycle_graph(7), gen.cycle_graph(40), gen.path_graph(33)])]
    for g in gs:
        seeds = np.arange(g.n, dtype=np.uint32)
        for k in (1, 2, 3, 6):
            check_graph(g, seeds, k)


def test_random_multigraphs_with_duplicates_and_self_loops():
    rng = np.random.default_rng(2024)
    for _ in range(12):
        n = int(rng.integers(1, 300))
        m = int(rng.integers(0, 6 * n + 1))
        src = rng.integers(0, n, m)
        dst = rng.integers(0, n, m)
        g = gen.csr_raw(n, src, dst)
        seeds = rng.integers(0, n, 32).astype(np.uint32)
        ks = rng.choice([0, 1, 2, 3, 6, 50], 32).astype(np.uint32)
        check_graph(g, seeds, ks)


def test_hub_rows_many_tiles():
    """A hub whose row spans many push tiles, plus many tiny rows."""
    n = 20000
    hub = np.zeros(n - 1, np.uint32)
    leaves = np.arange(1, n, dtype=np.uint32)
    rng = np.random.default_rng(5)
    s2 = rng.integers(1, n, 30000).astype(np.uint32)
    d2 = rng.integers(0, n, 30000).astype(np.uint32)
    g = gen.csr_from_edges(n, np.concatenate([hub, s2]), np.concatenate([leaves, d2]))
    seeds = np.array([0, 1, 2, 5, 19999, 7, 0], np.uint32)
    for k in (1, 2, 3, 6):
        check_graph(g, seeds, k, push_tile=256)


def test_runs_of_small_1hop_queries():
    """Runs of 1-hop queries at small seeds (answered by one CTA, the rest of
    the grid waiting) longer than one run, seed degrees on both sides of
    the one-CTA bound (2048 out-edges) with duplicate heads and self-loops,
    and other queries (k = 0, k > 1, seeds without out-edges) cutting the
    runs."""
    rng = np.random.default_rng(77)
    n = 5000
    src, dst = [], []
    for v, d in ((0, 2048), (1, 2049), (2, 2047), (3, 4000), (4, 1)):
        heads = rng.integers(0, n, d)
        heads[: d // 3] = heads[0]          # duplicate heads
        heads[-1] = v                       # self-loop
        src.append(np.full(d, v))
        dst.append(heads)
    src.append(rng.integers(5, n - 100, 20000))   # the last 100 vertices have no out-edges
    dst.append(rng.integers(0, n, 20000))
    g = gen.csr_raw(n, np.concatenate(src), np.concatenate(dst))
    seeds = rng.integers(0, n, 9000).astype(np.uint32)
    seeds[:6] = [0, 1, 2, 3, 4, n - 1]
    ks = np.ones(9000, np.uint32)
    cut = rng.choice(np.arange(8400, 9000), 60, replace=False)
    ks[cut] = rng.choice([0, 2, 3, 6], 60)
    seeds[rng.choice(np.arange(8400, 9000), 10, replace=False)] = n - 3   # no out-edges
    check_graph(g, seeds, ks, hop=True)


def test_fused_first_rounds_at_the_seed_degree_bound():
    """Multi-hop queries whose first two rounds run as one grid round (seed
    out-degree up to 1024: every CTA lists the seed's distinct out-neighbours
    itself) and the ones just above the bound, with duplicate heads,
    self-loops, sinks among the neighbours, and heads that are also
    neighbours of neighbours; counts, TE and per-hop counts in all three
    direction modes."""
    rng = np.random.default_rng(91)
    n = 6000
    src, dst = [], []
    for v, d in ((0, 2048), (1, 2049), (2, 2047), (3, 5), (4, 1), (5, 1024), (6, 1025), (7, 1023)):
        heads = rng.integers(0, 600, d)     # a dense neighbourhood: many shared heads
        heads[: d // 4] = heads[0]          # duplicate heads
        heads[-1] = v                       # self-loop
        src.append(np.full(d, v))
        dst.append(heads)
    src.append(rng.integers(0, 600, 9000))  # the neighbourhood links back into itself
    dst.append(rng.integers(0, 600, 9000))
    src.append(rng.integers(600, n - 50, 20000))
    dst.append(rng.integers(0, n, 20000))
    g = gen.csr_raw(n, np.concatenate(src), np.concatenate(dst))
    seeds = np.array([0, 1, 2, 3, 4, 0, 1, 2, 3, 4, 7, 500, n - 1, 5999, 42, 5, 6, 5, 6], np.uint32)
    ks = np.array([2, 2, 2, 2, 2, 3, 3, 6, 6, 3, 2, 2, 2, 2, 6, 2, 2, 3, 3], np.uint32)
    check_graph(g, seeds, ks, hop=True)
    check_graph(g, seeds, ks, hop=True, wide=True)


def test_edge_cases_seed_out_of_range_and_k0():
    g = gen.rmat(8, 8, seed=1)
    G = kh.Graph.from_csr(g)
    seeds = np.array([0, g.n, 5, g.n + 100, 3], np.uint32)
    ks = np.array([2, 2, 0, 1, 2**32 - 1], np.uint32)
    got = gpu_counts(G, seeds, ks)
    want, _ = oracle.khop_counts(g, seeds, np.minimum(ks, g.n + 1))
    assert got["counts"][1] == U64MAX and got["counts"][3] == U64MAX
    assert got["counts"][2] == 0
    np.testing.assert_array_equal(got["counts"][[0, 2, 4]], want[[0, 2, 4]])
    assert G.error_bits() & kh.DEVERR_SEED
    assert G.error_bits() == 0   # cleared by the read
    # empty call
    kh.khop_count(G.handle, 0, 0, 3, 0, torch.cuda.current_stream().cuda_stream)
    G.close()


def test_invalid_arguments_and_validation():
    g = gen.path_graph(10)
    G = kh.Graph.from_csr(g)
    with pytest.raises(kh.KhopError) as e:
        kh.khop_count(G.handle, None, 3, 1, None, 0)
    assert e.value.status == kh.EINVAL
    with pytest.raises(kh.KhopError):
        G.set_tuning(push_tile=300)
    G.close()
    bad = g.row_ptr.copy()
    bad[3] = 100
    with pytest.raises(kh.KhopError) as e:
        kh.Graph(10, bad, g.col_idx, validate=True)
    assert e.value.status == kh.EINVAL
    badc = g.col_idx.copy()
    badc[0] = 10
    with pytest.raises(kh.KhopError):
        kh.Graph(10, g.row_ptr, badc, validate=True)
    G2 = kh.Graph(10, g.row_ptr, g.col_idx, validate=True)
    G2.close()


def test_device_pointer_inputs_and_32bit_row_ptr():
    g = gen.rmat(10, 16, seed=1)
    rp = torch.from_numpy(g.row_ptr.astype(np.int64)).cuda()
    ci = torch.from_numpy(g.col_idx.view(np.int32)).cuda()
    G64 = kh.Graph(g.n, rp, ci)
    G32 = kh.Graph(g.n, g.row_ptr.astype(np.uint32), g.col_idx)
    seeds = gen.seeds(g, 64, seed=2)
    want, _ = oracle.khop_counts(g, seeds, 3)
    for G in (G64, G32):
        np.testing.assert_array_equal(kh.as_u64(G.count(seeds, 3)), want)
        G.close()


def test_streams_and_back_to_back_calls():
    g = gen.rmat(11, 16, seed=2, symmetrize=True)
    G = kh.Graph.from_csr(g)
    seeds = gen.seeds(g, 64, seed=3)
    want, _ = oracle.khop_counts(g, seeds, 6)
    s1, s2 = torch.cuda.Stream(), torch.cuda.Stream()
    outs = []
    for i in range(6):
        st = s1 if i % 2 else s2
        with torch.cuda.stream(st):
            outs.append(G.count(seeds, 6, stream=st))
    torch.cuda.synchronize()
    for o in outs:
        np.testing.assert_array_equal(kh.as_u64(o), want)
    G.close()


def test_stats_are_consistent():
    g = gen.rmat(12, 16, seed=1, symmetrize=True)
    seeds = gen.seeds(g, 16, seed=2)
    G = kh.Graph.from_csr(g)
    res = G.count_ex(seeds, np.full(16, 6, np.uint32))
    torch.cuda.synchronize()
    rec = kh.stats_records(res["stats"])
    assert (rec["rounds"] <= 6).all() and (rec["rounds"] >= 1).all()
    assert (rec["t_end_ns"] >= rec["t_start_ns"]).all()
    assert (rec["bytes"] > 0).all()
    np.testing.assert_array_equal(rec["te"], kh.as_u64(res["te"]))
    G.close()


def test_scale21_paper_protocol_in_bench_configuration():
    """The benchmark workload -- Kronecker scale 21, edge factor 16,
    symmetrized -- in the launch configuration the benchmark times: the
    graph tuned as the benchmark tunes it (bench.tune_graph: samples of seed
    stream 9), then all 620 paper-protocol queries (300/300/10/10
    seeds at k = 1/2/3/6) in one khop_count_ex launch.  Every count, TE and
    per-hop count equals the oracle's."""
    import bench
    g = gen.rmat(21, 16, seed=1, symmetrize=True)
    G = kh.Graph.from_csr(g)
    bench.tune_graph(G, g)
    seeds, ks = bench.paper_queries(g)
    assert seeds.size == 620
    want_c, want_te, want_ph = oracle.khop_counts(g, seeds, ks, per_hop=True)
    stride = want_ph.shape[1]
    res = G.count_ex(seeds, ks, te=True, hop_stride=stride)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(kh.as_u64(res["counts"]), want_c)
    np.testing.assert_array_equal(kh.as_u64(res["te"]), want_te)
    ph = kh.as_u64(res["per_hop"]).reshape(seeds.size, stride)
    np.testing.assert_array_equal(ph, want_ph)     # bins beyond a query's k are 0 on both sides
    assert G.error_bits() == 0
    G.close()


def test_autotune_changes_speed_only():
    g = gen.rmat(13, 16, seed=4, symmetrize=True)
    G = kh.Graph.from_csr(g)
    seeds = gen.seeds(g, 32, seed=5)
    before = kh.as_u64(G.count(seeds, 6))
    t = G.autotune(seeds, 6)
    assert t.block_threads in (256, 512, 1024) and t.push_tile in (512, 1024, 2048, 4096)
    assert t.alpha > 0 and t.beta > 0 and t.batch_alpha > 0 and t.batch_beta > 0
    assert t.batch_push_tile in (1024, 2048, 4096)
    want, _ = oracle.khop_counts(g, seeds, 6)
    np.testing.assert_array_equal(before, want)
    np.testing.assert_array_equal(kh.as_u64(G.count(seeds, 6)), want)
    np.testing.assert_array_equal(
        kh.as_u64(G.count_mixed(seeds, np.full(32, 6, np.uint32), mode=kh.MODE_BATCHED64)), want)
    G.close()
