"""Parity on the full-size power-law graph (41.6M vertices, 1.47e9 edges).

This is the benchmark's Twitter-shaped workload, in the benchmark's launch
configuration (the graph tuned as the benchmark tunes it, bench.tune_graph).  Every
count of the paper protocol (300/300/10/10 seeds at k = 1/2/3/6, one plain
launch) and every count of the batched leg (1024 seeds, k mixed over
{1,2,3,6}, 64 and 128 lanes per traversal) is compared with the oracle.

Building the graph takes about two minutes and ~30 GB of host memory the
first time; gen.cached() then keeps a verified copy on disk.  The test runs
wherever the host has the memory for it and skips (saying why) where it has
not.
"""
import numpy as np
import pytest

import gen
import oracle

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
kh = pytest.importorskip("paper_1905_01294_gb300")

CHUNGLU = dict(n=41_600_000, edges=1_470_000_000, w_max=3e6, seed=4)
HOST_BYTES = 48 << 30     # generation peak (~30 GB) plus the oracle's per-thread arrays
DEVICE_BYTES = 24 << 30   # CSR + CSC (12.4 GB) plus traversal and batch state


def _mem_available():
    """Host memory this process may still use: MemAvailable, capped by the
    cgroup's limit (v2 memory.max, or v1 limit_in_bytes) minus its usage."""
    avail = 0
    try:
        with open("/proc/meminfo") as f:
            for line in f:
                if line.startswith("MemAvailable:"):
                    avail = int(line.split()[1]) * 1024
    except OSError:
        pass
    for lim, cur in (("/sys/fs/cgroup/memory.max", "/sys/fs/cgroup/memory.current"),
                     ("/sys/fs/cgroup/memory/memory.limit_in_bytes",
                      "/sys/fs/cgroup/memory/memory.usage_in_bytes")):
        try:
            with open(lim) as f:
                t = f.read().strip()
            if t == "max":
                continue
            with open(cur) as f:
                used = int(f.read().strip())
            avail = min(avail, int(t) - used)
        except (OSError, ValueError):
            continue
    return avail


def test_chunglu_41M_every_count_equals_the_oracle():
    if not torch.cuda.is_available():
        pytest.fail("CUDA device required for -m gpu tests")
    avail = _mem_available()
    if avail < HOST_BYTES:
        pytest.skip(f"host has {avail >> 30} GiB available, the graph needs {HOST_BYTES >> 30} GiB")
    torch.cuda.set_device(0)
    free, _ = torch.cuda.mem_get_info()
    if free < DEVICE_BYTES:
        pytest.skip(f"device has {free >> 30} GiB free, the graph needs {DEVICE_BYTES >> 30} GiB")
    import bench
    g = gen.cached("chunglu", **CHUNGLU)
    assert g.nnz >= 1_470_000_000 and g.n == 41_600_000
    G = kh.Graph.from_csr(g)
    bench.tune_graph(G, g)
    # the paper protocol, one plain launch: counts, TE and per-hop counts
    seeds, ks = bench.paper_queries(g)
    want_c, want_te, want_ph = oracle.khop_counts(g, seeds, ks, per_hop=True)
    res = G.count_ex(seeds, ks, te=True, hop_stride=want_ph.shape[1])
    torch.cuda.synchronize()
    np.testing.assert_array_equal(kh.as_u64(res["counts"]), want_c)
    np.testing.assert_array_equal(kh.as_u64(res["te"]), want_te)
    np.testing.assert_array_equal(kh.as_u64(res["per_hop"]).reshape(want_ph.shape), want_ph)
    # the batched leg: 1024 mixed queries
    bs = gen.seeds(g, 1024, seed=2)
    bk = gen.mixed_ks(1024, seed=2)
    want, _ = oracle.khop_counts(g, bs, bk, with_te=False)
    for mode in (kh.MODE_BATCHED64, kh.MODE_BATCHED128):
        got = kh.as_u64(G.count_mixed(bs, bk, mode=mode))
        np.testing.assert_array_equal(got, want, err_msg=f"mode {mode}")
    assert G.error_bits() == 0
    G.close()
