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
    srv = kh.Server(max_batches=1)               # one slot: every request joins its rolling batch
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


def test_requests_join_a_running_traversal_and_retire_on_their_own():
    """Continuous batching at round granularity: with one rolling slot that
    admits at every step, heavy requests submitted while a traversal runs are
    admitted into its free lanes at the next round boundary (joined_running),
    each with its own round counter; a 3-hop request that joined is posted
    before the first lane, whose traversal runs forty rounds; lanes
    whose frontier empties before their k retire early; every served count
    equals the oracle's for the query alone."""
    # an R-MAT graph plus a directed 40-vertex path: a lane seeded at the
    # path's start runs 40 rounds
    gr = gen.rmat(16, 16, seed=7, symmetrize=True)
    g = gen.disjoint_union([gr, gen.path_graph(40)])
    G = kh.Graph.from_csr(g)
    seeds = np.concatenate([np.array([gr.n], np.uint32), gen.seeds(gr, 119, seed=9)])
    ks = np.array([50] + [3 + i % 4 for i in range(100)] + [50] * 19, np.uint32)
    want, _ = oracle.khop_counts(g, seeds, ks)
    srv = kh.Server(max_batches=1, admit_rounds=0xFFFFFFFF, plain_heavy=-1)
    first = srv.submit(G, seeds[0], 50)
    t0 = time.time()
    while srv.counters()["steps"] < 1 and time.time() - t0 < 10:
        time.sleep(1e-4)
    rest = [srv.submit(G, s, k) for s, k in zip(seeds[1:], ks[1:])]
    got = drain(srv, len(rest) + 1)
    assert len(got) == len(rest) + 1
    tks = [first] + rest
    assert [got[t].status for t in tks] == [kh.OK] * len(tks)
    assert [got[t].count for t in tks] == want.tolist()
    c = srv.counters()
    assert c["joined_running"] >= 1 and c["max_lanes_busy"] >= 2
    assert c["retired_early"] >= 1           # the k = 50 lanes stop when their frontier empties
    assert c["submitted"] == c["completed"] == len(tks)
    assert c["plain_launches"] == 0          # every request ran in the rolling slot
    # a 3-hop request that joined was posted before the first, deeper lane
    three = [t for t, k in zip(rest, ks[1:]) if k == 3]
    assert min(got[t].t_done_ns for t in three) < got[first].t_done_ns
    srv.close()
    G.close()


def test_light_requests_take_the_single_query_path():
    """Light requests (k <= 2) are answered by plain launches, several per
    launch, and equal the oracle's counts."""
    g = gen.rmat(14, 16, seed=11, symmetrize=True)
    G = kh.Graph.from_csr(g)
    seeds = gen.seeds(g, 300, seed=12)
    ks = np.array([1 + i % 2 for i in range(300)], np.uint32)
    srv = kh.Server()
    tks = srv.submit_many(G, seeds, ks)
    got = drain(srv, len(tks))
    want, _ = oracle.khop_counts(g, seeds, ks)
    assert [got[t].count for t in tks.tolist()] == want.tolist()
    c = srv.counters()
    assert c["plain_launches"] >= 1 and c["steps"] == 0
    srv.close()
    G.close()


def test_step_wait_timeout_then_reused_slot_is_exact():
    """A step that runs past the server's wait bound is given up: its
    requests complete with KHOP_ETIMEDOUT at once.  With the default bound
    restored, the same slot (reset to zeroed state) serves the same requests
    exactly."""
    g = gen.rmat(14, 16, seed=9, symmetrize=True)
    G = kh.Graph.from_csr(g)
    seeds = gen.seeds(g, 40, seed=10)
    ks = np.full(40, 3, np.uint32)
    srv = kh.Server(max_batches=1, wait_timeout_us=1, plain_heavy=-1)
    tks = srv.submit_many(G, seeds, ks)
    got = drain(srv, len(tks))
    assert all(got[t].status == kh.ETIMEDOUT for t in tks.tolist())
    assert srv.counters()["timed_out"] == len(tks)
    srv.set_wait_timeout(0)
    tks = srv.submit_many(G, seeds, ks)
    got = drain(srv, len(tks))
    want, _ = oracle.khop_counts(g, seeds, ks)
    assert [got[t].status for t in tks.tolist()] == [kh.OK] * len(tks)
    assert [got[t].count for t in tks.tolist()] == want.tolist()
    assert srv.stats()["batches"] == 1       # the same slot, reused
    with pytest.raises(kh.KhopError):
        srv.set_wait_timeout(-1)
    srv.close()
    G.close()
