"""The allocation-free entry point khop_count_static.

It serves callers that cannot allocate device memory (their memory belongs to
another allocator, or they cannot take an allocation's implicit device
synchronisation), so it keeps its traversal state in a fixed device array and
takes the graph as raw device arrays.  Its counts must equal those of
khop_count on a graph created the usual way and the oracle's, on two calls in
a row (the second call reuses the state the first one left behind), with a
separate CSC, with the CSR passed again as the CSC of a symmetric graph, and
without a CSC (push only).  A seed >= n gives UINT64_MAX.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
kh = pytest.importorskip("paper_1905_01294_gb300")


U64MAX = np.uint64(2**64 - 1)


def _dev_u32(a):
    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.uint32).view(np.int32)).cuda()


def _csc(g):
    rows = np.repeat(np.arange(g.n, dtype=np.uint32), np.diff(g.row_ptr).astype(np.int64))
    order = np.argsort(g.col_idx, kind="stable")
    col_ptr = np.zeros(g.n + 1, np.uint64)
    col_ptr[1:] = np.cumsum(np.bincount(g.col_idx.astype(np.int64), minlength=g.n))
    return col_ptr.astype(np.uint32), rows[order]


@pytest.mark.parametrize("symmetric", [False, True])
def test_static_entry_point_matches_khop_count_twice(symmetric):
    torch.cuda.set_device(0)
    g = gen.rmat(14, 16, seed=11, symmetrize=symmetric)
    G = kh.Graph.from_csr(g)
    seeds = gen.seeds(g, 96, seed=12)
    seeds[5] = g.n + 3                          # out of range: UINT64_MAX
    d_seeds = _dev_u32(seeds)
    rp, ci = _dev_u32(g.row_ptr), _dev_u32(g.col_idx)
    cp_h, ri_h = _csc(g)
    cp, ri = _dev_u32(cp_h), _dev_u32(ri_h)
    stream = torch.cuda.current_stream().cuda_stream
    # the CSC as separate arrays; for the symmetric graph also the CSR arrays
    # passed again as the CSC (the entry point's declared-symmetric branch)
    cscs = [(cp, ri)] + ([(rp, ci)] if symmetric else [])
    for k in (6, 2):                         # two calls in a row, each CSC form
        want, _ = oracle.khop_counts(g, seeds, k)
        assert want[5] == U64MAX
        ref = kh.as_u64(G.count(seeds, k))
        np.testing.assert_array_equal(ref, want)
        for c_p, r_i in cscs:
            out = torch.empty(seeds.size, dtype=torch.int64, device="cuda")
            kh.khop_count_static(g.n, rp.data_ptr(), ci.data_ptr(), c_p.data_ptr(), r_i.data_ptr(),
                                 g.nnz, d_seeds.data_ptr(), seeds.size, k, out.data_ptr(), stream)
            torch.cuda.synchronize()
            np.testing.assert_array_equal(kh.as_u64(out), want)   # integers: exact
            np.testing.assert_array_equal(kh.as_u64(out), ref)
    # push-only form (no CSC) agrees as well
    out = torch.empty(seeds.size, dtype=torch.int64, device="cuda")
    kh.khop_count_static(g.n, rp.data_ptr(), ci.data_ptr(), None, None, g.nnz,
                         d_seeds.data_ptr(), seeds.size, 3, out.data_ptr(), stream)
    torch.cuda.synchronize()
    want, _ = oracle.khop_counts(g, seeds, 3)
    np.testing.assert_array_equal(kh.as_u64(out), want)
    np.testing.assert_array_equal(kh.as_u64(out), kh.as_u64(G.count(seeds, 3)))
    G.close()


def test_static_entry_point_rejects_oversized_graphs():
    torch.cuda.set_device(0)
    x = torch.zeros(8, dtype=torch.int32, device="cuda")
    out = torch.empty(1, dtype=torch.int64, device="cuda")
    for n, nnz in (((1 << 20) + 1, 4), (16, (1 << 26) + 1)):
        with pytest.raises(kh.KhopError) as e:
            kh.khop_count_static(n, x.data_ptr(), x.data_ptr(), None, None, nnz, x.data_ptr(),
                                 1, 1, out.data_ptr(), 0)
        assert e.value.status == kh.EINVAL
