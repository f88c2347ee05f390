"""Host logic of the benchmark (no GPU): how bench.tune_graph merges the two
autotuner passes, and which serving sweep point counts as sustained."""
import numpy as np
import pytest

import bench
import gen


class _Tuning:
    _fields_ = [(f, None) for f in ("direction", "alpha", "beta", "block_threads", "blocks_per_sm",
                                    "push_tile", "batch_alpha", "batch_beta", "batch_push_tile")]

    def __init__(self, **kw):
        for f, _ in self._fields_:
            setattr(self, f, kw.get(f, 0))


class _FakeGraph:
    """Records the autotuner calls and returns a different tuning per sample."""

    def __init__(self):
        self.calls = []
        self.current = _Tuning()

    def autotune(self, seeds, k=None, ks=None, stream=None):
        ks = np.asarray(ks)
        self.calls.append((np.asarray(seeds).copy(), ks.copy()))
        if (ks == 6).mean() > 0.1:   # the mixed-k sample
            t = _Tuning(direction=0, alpha=40.0, beta=8.0, block_threads=1024, blocks_per_sm=1,
                        push_tile=4096, batch_alpha=5.0, batch_beta=100.0, batch_push_tile=1024)
        else:                         # the paper-protocol-shaped sample
            t = _Tuning(direction=0, alpha=14.0, beta=64.0, block_threads=512, blocks_per_sm=2,
                        push_tile=512, batch_alpha=2.0, batch_beta=6.0, batch_push_tile=4096)
        self.current = t
        return t

    def set_tuning(self, **kw):
        self.current = _Tuning(**kw)

    def tuning(self):
        return self.current


def test_tune_graph_takes_plain_fields_from_the_paper_sample_and_batched_from_the_mixed():
    g = gen.rmat(10, 16, seed=1, symmetrize=True)
    G = _FakeGraph()
    t = bench.tune_graph(G, g)
    assert len(G.calls) == 2
    (s1, k1), (s2, k2) = G.calls
    # first pass: 1024 seeds of stream 9, k mixed over {1,2,3,6}
    assert s1.size == 1024 and set(np.unique(k1)) == {1, 2, 3, 6}
    np.testing.assert_array_equal(s1, gen.seeds(g, 1024, seed=9))
    # second pass: the paper protocol's shape (300/300/10/10) from stream 9, not the measured seeds
    assert s2.size == 620 and [int((k2 == k).sum()) for k in (1, 2, 3, 6)] == [300, 300, 10, 10]
    measured, _ = bench.paper_queries(g)
    assert not np.array_equal(s2, measured)
    assert (t.block_threads, t.blocks_per_sm, t.push_tile, t.alpha, t.beta) == (512, 2, 512, 14.0, 64.0)
    assert (t.batch_alpha, t.batch_beta, t.batch_push_tile) == (5.0, 100.0, 1024)


def _pt(offered, achieved):
    return {"offered_qps": offered, "achieved_qps": achieved}


def test_sustained_rate_needs_98_percent_of_the_offered_rate():
    pts = [_pt(25e3, 24.9e3), _pt(100e3, 99.5e3), _pt(150e3, 147.1e3), _pt(200e3, 186e3), _pt(300e3, 185e3)]
    best, top = bench.best_and_sustained(pts)
    assert best["offered_qps"] == 200e3            # the highest achieved rate
    assert top["offered_qps"] == 150e3             # 147.1k of 150k = 98.07%; 186k of 200k = 93% is not
    best, top = bench.best_and_sustained([_pt(5e3, 4.8e3), _pt(10e3, 9.5e3)])
    assert top is None and best["offered_qps"] == 10e3


def test_a_rate_exactly_at_the_bound_counts():
    _, top = bench.best_and_sustained([_pt(100.0, 98.0), _pt(200.0, 195.0)])
    assert top["offered_qps"] == 100.0
