"""Failure detection of the device-side waits, without faulting the GPU.

Every grid barrier of a traversal is bounded (khop_graph_set_wait_limit).
khop_graph_test_absent_cta makes one CTA of the next launch stay away from a
chosen barrier -- the way a lost CTA would -- so the others' wait must run
out: the launch records KHOP_DEVERR_TIMEOUT and returns instead of hanging,
the absent CTA leaves once it sees the timeout, and the graph stays usable:
the next call (default limit) gives the oracle's counts exactly, on the plain
path and on the batched path (whose unfinished launch left its state dirty,
so the next launch re-zeroes it).
"""
import time

import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
kh = pytest.importorskip("paper_1905_01294_gb300")


@pytest.fixture(scope="module")
def graph():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    torch.cuda.set_device(0)
    g = gen.rmat(14, 16, seed=5, symmetrize=True)
    seeds = gen.seeds(g, 200, seed=6)
    ks = gen.mixed_ks(200, seed=6)
    want, _ = oracle.khop_counts(g, seeds, ks)
    G = kh.Graph.from_csr(g)
    yield G, seeds, ks, want
    G.close()


@pytest.mark.parametrize("mode,barrier", [(kh.MODE_PLAIN, 1), (kh.MODE_PLAIN, 3),
                                          (kh.MODE_BATCHED64, 1), (kh.MODE_BATCHED64, 4),
                                          (kh.MODE_BATCHED128, 5)])
def test_absent_cta_times_out_then_next_call_is_exact(graph, mode, barrier):
    G, seeds, ks, want = graph
    assert G.error_bits() == 0
    G.set_wait_limit(5_000_000)              # 5 ms
    G.test_absent_cta(barrier)
    t0 = time.time()
    G.count_mixed(seeds, ks, mode=mode)
    torch.cuda.synchronize()
    assert time.time() - t0 < 5.0            # the launch returned: the wait was bounded
    assert G.error_bits() & kh.DEVERR_TIMEOUT
    G.set_wait_limit(0)                      # back to the default (2 s)
    for m in (mode, kh.MODE_PLAIN):
        got = kh.as_u64(G.count_mixed(seeds, ks, mode=m))
        torch.cuda.synchronize()
        np.testing.assert_array_equal(got, want, err_msg=f"after the timeout, mode {m}")
    assert G.error_bits() == 0


def test_wait_limit_arguments(graph):
    G, _, _, _ = graph
    with pytest.raises(kh.KhopError) as e:
        G.set_wait_limit(61_000_000_000)     # beyond 60 s
    assert e.value.status == kh.EINVAL
    G.set_wait_limit(0)
    G.test_absent_cta(0)                      # off: nothing happens
    G.count(np.array([0], np.uint32), 2)
    torch.cuda.synchronize()
    assert G.error_bits() == 0
