"""Pins of the reverse / either-direction inputs (tests/variants.py) with the
oracle on graphs whose neighbourhoods are known by hand."""
import numpy as np

import gen
import oracle
from tests import variants


def test_transpose_twice_is_the_same_edge_multiset():
    rng = np.random.default_rng(5)
    g = gen.csr_raw(50, rng.integers(0, 50, 400), rng.integers(0, 50, 400))
    t2 = variants.transpose(variants.transpose(g))
    a = sorted(zip(*variants.edges(g)))
    b = sorted(zip(*variants.edges(t2)))
    assert a == b


def test_out_star_in_and_either_direction_counts():
    # 0 -> 1..L
    L = 9
    g = gen.out_star(L)
    leaves = np.arange(1, L + 1, dtype=np.uint32)
    fwd, _ = oracle.khop_counts(g, leaves, 2)
    assert (fwd == 0).all()                      # leaves have no out-edges
    rev, _ = oracle.khop_counts(variants.transpose(g), leaves, 3)
    assert (rev == 1).all()                      # the centre, nothing beyond
    centre_rev, _ = oracle.khop_counts(variants.transpose(g), np.array([0], np.uint32), 2)
    assert centre_rev[0] == 0
    und = variants.either_direction(g)
    c1, _ = oracle.khop_counts(und, leaves, 1)
    c2, _ = oracle.khop_counts(und, leaves, 2)
    assert (c1 == 1).all() and (c2 == L).all()   # centre, then the other leaves


def test_directed_path_reverse_and_either_direction():
    # 0 -> 1 -> 2 -> ... -> 9
    g = gen.path_graph(10)
    s = np.array([5], np.uint32)
    for k in range(0, 8):
        f, _ = oracle.khop_counts(g, s, k)
        r, _ = oracle.khop_counts(variants.transpose(g), s, k)
        u, _ = oracle.khop_counts(variants.either_direction(g), s, k)
        assert f[0] == min(k, 4)       # 6..9
        assert r[0] == min(k, 5)       # 4..0
        assert u[0] == min(k, 4) + min(k, 5)
