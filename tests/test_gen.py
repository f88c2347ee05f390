"""Input generators: determinism, CSR validity, R-MAT quadrant rates, seeds."""
import numpy as np

import gen

M64 = (1 << 64) - 1


def _splitmix64_stream(state, count):
    """Textbook splitmix64 (Steele, Lea, Flood 2014): state += gamma; mix."""
    out = []
    for _ in range(count):
        state = (state + 0x9E3779B97F4A7C15) & M64
        z = state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & M64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & M64
        out.append(z ^ (z >> 31))
    return out


def test_splitmix64_counter_form_matches_sequential_generator():
    # key 0: mix64(0) = 0, so the stream is splitmix64 started at state 0,
    # whose first output is the published 0xE220A8397B1DCDAF.
    assert gen.rand(0, 0) == 0xE220A8397B1DCDAF
    seq = _splitmix64_stream(0, 5)
    assert [gen.rand(0, i) for i in range(5)] == seq
    start = gen.rand(12345, 0)  # any key: stream = splitmix64 from state mix64(key)
    arr = gen.rand_array(99, 10, 4)
    assert [int(x) for x in arr] == [gen.rand(99, 10 + j) for j in range(4)]
    assert start != gen.rand(12346, 0)


def test_rmat_deterministic_and_thread_independent():
    a = gen.rmat(10, 16, seed=1, nthreads=1)
    b = gen.rmat(10, 16, seed=1, nthreads=7)
    np.testing.assert_array_equal(a.row_ptr, b.row_ptr)
    np.testing.assert_array_equal(a.col_idx, b.col_idx)
    c = gen.rmat(10, 16, seed=2)
    assert a.nnz != c.nnz or not np.array_equal(a.col_idx, c.col_idx)


def _check_csr(g, symmetric):
    assert g.row_ptr[0] == 0 and g.row_ptr[-1] == g.col_idx.size
    assert (np.diff(g.row_ptr.astype(np.int64)) >= 0).all()
    assert (g.col_idx < g.n).all()
    rows = np.repeat(np.arange(g.n), np.diff(g.row_ptr).astype(np.int64))
    assert not (rows == g.col_idx).any()                       # no self-loops
    key = rows.astype(np.int64) * g.n + g.col_idx
    assert (np.diff(key) > 0).all()                            # sorted, no duplicates
    if symmetric:
        rkey = g.col_idx.astype(np.int64) * g.n + rows
        np.testing.assert_array_equal(np.sort(rkey), key)


def test_rmat_csr_valid():
    _check_csr(gen.rmat(10, 16, seed=1), False)
    _check_csr(gen.rmat(11, 8, seed=5, symmetrize=True), True)


def test_rmat_quadrant_rates():
    m = 400_000
    s, d = gen.rmat_edges_unpermuted(1, m, 0.57, 0.19, 0.19, seed=1)
    rates = [np.mean((s == a) & (d == b)) for a, b in ((0, 0), (0, 1), (1, 0), (1, 1))]
    for got, want in zip(rates, (0.57, 0.19, 0.19, 0.05)):
        assert abs(got - want) < 4 * np.sqrt(want * (1 - want) / m)
    # at scale 10 the top bit of the source is 0 with probability A + B
    s, d = gen.rmat_edges_unpermuted(10, m, seed=3)
    p = np.mean((s >> 9) == 0)
    assert abs(p - 0.76) < 4 * np.sqrt(0.76 * 0.24 / m)


def test_permutation_is_bijection():
    p = gen.permutation(1000, 17)
    np.testing.assert_array_equal(np.sort(p), np.arange(1000))
    assert not np.array_equal(p, np.arange(1000))


def test_seeds_have_out_edges_and_are_deterministic():
    g = gen.rmat(10, 16, seed=1)
    s1 = gen.seeds(g, 64, seed=2)
    s2 = gen.seeds(g, 64, seed=2)
    np.testing.assert_array_equal(s1, s2)
    deg = np.diff(g.row_ptr)
    assert (deg[s1] > 0).all()
    assert len(np.unique(gen.seeds(g, 5000, seed=9))) > 300


def test_poisson_stream_shape():
    g = gen.rmat(10, 16, seed=1)
    t, ks, sd = gen.poisson_stream(g, 20000, 1000.0, seed=3)
    assert (np.diff(t) > 0).all()
    assert abs(np.mean(np.diff(t)) - 1e-3) < 5e-5
    for k, p in ((1, .4), (2, .3), (3, .2), (6, .1)):
        assert abs(np.mean(ks == k) - p) < 0.02
    assert (np.diff(g.row_ptr)[sd] > 0).all()


def test_mixed_ks():
    ks = gen.mixed_ks(4096, seed=2)
    assert set(np.unique(ks).tolist()) == {1, 2, 3, 6}


def test_powerlaw_weights_are_the_quantiles_and_sum_to_the_total():
    w, w_min = gen.powerlaw_weights(100000, 5000.0, 1e6)
    assert abs(w.sum() - 1e6) < 1e-3
    assert (np.diff(w) > 0).all() and w[0] > w_min and w[-1] < 5000.0
    # the fraction of weights above x follows the density p(w) ~ w^-2:
    # P(W > x) = (1/x - 1/w_max) / (1/w_min - 1/w_max)
    for x in (2 * w_min, 10 * w_min, 100 * w_min):
        want = (1 / x - 1 / 5000.0) / (1 / w_min - 1 / 5000.0)
        assert abs(np.mean(w > x) - want) < 2e-4


def test_alias_sampler_matches_the_weights():
    n, m = 1000, 2_000_000
    w = np.arange(1, n + 1, dtype=np.float64) ** 1.5
    po, ao = gen.alias_table(w)
    src = np.empty(m, np.uint32)
    dst = np.empty(m, np.uint32)
    gen._L().khopgen_chunglu_edges(n, gen._p(po), gen._p(ao), gen._p(po), gen._p(ao), 5, 6, 0, m,
                                   gen._p(src), gen._p(dst), 0)
    for x in (src, dst):
        c = np.bincount(x, minlength=n)
        e = m * w / w.sum()
        z = (c - e) / np.sqrt(e)
        assert np.abs(z).max() < 5.5 and abs(np.mean(z ** 2) - 1) < 0.15


def test_chunglu_graph_valid_deterministic_and_sized():
    g = gen.chunglu(50000, 600000, 3000.0, seed=4)
    _check_csr(g, False)
    assert 600000 <= g.nnz < 600000 + (1 << 20)
    g2 = gen.chunglu(50000, 600000, 3000.0, seed=4, nthreads=3)
    np.testing.assert_array_equal(g.col_idx, g2.col_idx)
    np.testing.assert_array_equal(g.row_ptr, g2.row_ptr)
    outd = np.diff(g.row_ptr).astype(np.int64)
    ind = np.bincount(g.col_idx, minlength=g.n)
    assert 0.5 * 3000 < outd.max() < 3000 * 1.3 and 0.5 * 3000 < ind.max() < 3000 * 1.3
    assert np.corrcoef(outd, ind)[0, 1] < 0.1      # independent out/in weights


# ---- on-disk graph cache -----------------------------------------------------

def test_checksum_is_order_sensitive_and_thread_independent():
    a = np.arange(1000003, dtype=np.uint32)
    c1 = gen.checksum(a, nthreads=1)
    assert c1 == gen.checksum(a, nthreads=7)
    b = a.copy()
    b[[10, 11]] = b[[11, 10]]                    # swap two entries
    assert gen.checksum(b) != c1
    assert gen.checksum(a[:-1]) != c1            # length matters
    assert gen.checksum(np.zeros(3, np.uint8)) != gen.checksum(np.zeros(4, np.uint8))


def test_graph_cache_round_trip_and_rejects_damage(tmp_path):
    g = gen.cached("rmat", directory=str(tmp_path), scale=9, edge_factor=8, seed=3)
    files = list(tmp_path.glob("rmat-*.csr"))
    assert len(files) == 1
    h = gen.cached("rmat", directory=str(tmp_path), scale=9, edge_factor=8, seed=3)
    assert h.n == g.n and h.params == g.params
    np.testing.assert_array_equal(h.row_ptr, g.row_ptr)
    np.testing.assert_array_equal(h.col_idx, g.col_idx)
    ref = gen.rmat(9, 8, seed=3)
    np.testing.assert_array_equal(h.col_idx, ref.col_idx)
    # other parameters miss the cache
    gen.cached("rmat", directory=str(tmp_path), scale=9, edge_factor=8, seed=4)
    assert len(list(tmp_path.glob("rmat-*.csr"))) == 2
    # one flipped byte in the edge array, or a truncated file, fails the checks
    path = str(files[0])
    raw = bytearray(open(path, "rb").read())
    raw[-3] ^= 0x40
    open(path, "wb").write(bytes(raw))
    assert gen.load_graph(path) is None
    open(path, "wb").write(bytes(raw[:-4]))
    assert gen.load_graph(path) is None
    # and the next cached() call rebuilds a good copy
    k = gen.cached("rmat", directory=str(tmp_path), scale=9, edge_factor=8, seed=3)
    np.testing.assert_array_equal(k.col_idx, ref.col_idx)
    assert gen.load_graph(path) is not None
