"""The multi-GPU path of bench.py is replicas only (independent queries, no
collective on the data path): these gloo tests run its cross-rank reduction and
its rank handling as two CPU processes."""
import importlib.util
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _bench():
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    b = _bench()
    # rank r ran 620 * (r + 1) queries in 0.5 * (r + 1) seconds
    out = b.over_ranks(dist, 0.5 * (rank + 1), 620 * (rank + 1), "cpu")
    q.put((rank, out))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_reduce_to_max_time_and_summed_queries():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    for r in (0, 1):
        t, n, qps = res[r]
        assert t == 1.0 and n == 620 * 3 and qps == 1860.0


def test_single_process_reduction_is_identity():
    b = _bench()
    assert b.over_ranks(None, 2.0, 100, "cpu") == (2.0, 100, 50.0)


def test_reference_arm_other_ranks_exit_quietly(capsys, monkeypatch):
    b = _bench()
    monkeypatch.setenv("RANK", "1")

    class A:
        scale, steps, warmup, gpus = 10, 1, 1, 2
    assert b.run_reference(A) == 0
    assert capsys.readouterr().out == ""
