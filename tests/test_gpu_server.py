"""GPU tests of the continuous-batching request server (khop_server_*).

Each served result must equal the same query answered alone (the oracle, and
the plain path), whatever mix of graphs, seeds and k it was served in; the
tolerance is zero because counts are integers.
"""
import time

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


def drain(srv, n, timeout_s=60.0):
    got, t0 = {}, time.time()
    while len(got) < n and time.time() - t0 < timeout_s:
        for r in srv.poll(4096, 100000):
            got[r.ticket] = r
    return got


def test_served_results_equal_alone_on_two_resident_graphs():
    ga = gen.rmat(13, 16, seed=1, symmetrize=True)
    gb = gen.rmat(12, 16, seed=5)
    A, B = kh.Graph.from_csr(ga), kh.Graph.from_csr(gb)
    t, ks_a, sd_a = gen.poisson_stream(ga, 600, 200000.0, seed=3)
    _, ks_b, sd_b = gen.poisson_stream(gb, 400, 200000.0, seed=4)
    srv = kh.Server(max_batches=3)
    tickets = {}
    t0 = time.perf_counter()
    ia = ib = 0
    while ia < len(sd_a) or ib < len(sd_b):
        # open loop: submit whatever has "arrived" by now (graph A's clock)
        now = time.perf_counter() - t0
        while ia < len(sd_a) and t[ia] <= now:
            tickets[srv.submit(A, sd_a[ia], ks_a[ia])] = ("a", ia)
            if ib < len(sd_b):
                tickets[srv.submit(B, sd_b[ib], ks_b[ib])] = ("b", ib)
                ib += 1
            ia += 1
        if ia >= len(sd_a):
            while ib < len(sd_b):
                tickets[srv.submit(B, sd_b[ib], ks_b[ib])] = ("b", ib)
                ib += 1
    got = drain(srv, len(tickets))
    assert len(got) == len(tickets)
    want_a, _ = oracle.khop_counts(ga, sd_a, ks_a)
    want_b, _ = oracle.khop_counts(gb, sd_b, ks_b)
    for tk, (which, i) in tickets.items():
        r = got[tk]
        assert r.status == kh.OK
        assert r.count == (want_a[i] if which == "a" else want_b[i])
        assert r.t_done_ns >= r.t_submit_ns
    # alone: the plain path gives the same counts
    np.testing.assert_array_equal(kh.as_u64(A.count_mixed(sd_a, ks_a, mode=kh.MODE_PLAIN)), want_a)
    st = srv.stats()
    assert st["submitted"] == st["completed"] == len(tickets)
    assert 1 <= st["batches"] <= 6
    srv.close()
    A.close()
    B.close()


def test_k0_invalid_seed_and_full_queue():
    g = gen.rmat(10, 16, seed=1)
    G = kh.Graph.from_csr(g)
    srv = kh.Server(max_pending=4)
    t0 = srv.submit(G, 3, 0)
    with pytest.raises(kh.KhopError) as e:
        srv.submit(G, g.n, 2)
    assert e.value.status == kh.EINVAL
    res = drain(srv, 1)
    assert res[t0].count == 0 and res[t0].status == kh.OK
    # fill the queue beyond max_pending: EBUSY (the worker may drain some first)
    busy = 0
    for i in range(64):
        try:
            srv.submit(G, i % 50, 6)
        except kh.KhopError as ex:
            assert ex.status == kh.EBUSY
            busy += 1
    srv.close()
    G.close()


def test_memory_budget_admission():
    g = gen.rmat(11, 16, seed=2)
    G = kh.Graph.from_csr(g)
    srv = kh.Server(mem_budget_bytes=1)          # no slot can be admitted
    tks = [srv.submit(G, s, 3) for s in gen.seeds(g, 10, seed=1)]
    res = drain(srv, len(tks), timeout_s=20)
    assert all(res[t].status == kh.ENOMEM for t in tks)
    srv.close()
    seeds = gen.seeds(g, 200, seed=1)
    srv = kh.Server(max_batches=1)               # one slot: cohorts run one after another
    tks = [srv.submit(G, s, 1 + i % 6) for i, s in enumerate(seeds)]
    res = drain(srv, len(tks))
    want, _ = oracle.khop_counts(g, seeds, [1 + i % 6 for i in range(200)])
    assert [res[t].count for t in tks] == want.tolist()
    assert srv.stats()["batches"] == 1
    srv.close()
    G.close()


def test_shutdown_with_requests_in_flight():
    g = gen.rmat(14, 16, seed=3, symmetrize=True)
    G = kh.Graph.from_csr(g)
    srv = kh.Server(max_batches=1)
    for s in gen.seeds(g, 1000, seed=2):
        srv.submit(G, s, 6)
    srv.close()                                  # drains in-flight work, fails the rest
    G.close()
