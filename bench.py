"""Benchmark: k-hop neighbourhood count on one GB300 (or N replicas).

Workload (default): the paper's single-request protocol (Sec. III: 300 seeds
for the 1- and 2-hop queries, 10 seeds for the 3- and 6-hop queries, run one
after another) on a synthetic Graph500-shaped Kronecker graph of scale 21
(2,097,152 vertices, edge factor 16, A/B/C/D = .57/.19/.19/.05, seed 1,
symmetrized, self-loops removed, duplicates collapsed), uint32 CSR.  One step
= those 620 queries on the plain single-query path (one persistent launch).

Also reported: the 64-lane batched form on 4096 seeds with k mixed over
{1,2,3,6}, and the continuous-batching server under an open-loop Poisson
request stream.

Metric: queries/sec (and GTEPS, p50/p99/p99.9 latency).  `value` is measured
with CUDA events on the launching stream, inputs resident in HBM, L2 flushed
between steps (a 256 MiB write).  `e2e` is the same metric through the public
API with the seeds and ks copied from pinned host memory and the counts copied
back, inside the timed region.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
"""
from __future__ import annotations

import argparse
import json
import os
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import gen  # noqa: E402

PAPER_QUERIES = ((1, 300), (2, 300), (3, 10), (6, 10))   # (k, seeds), run sequentially


def workload_graph(scale: int):
    t0 = time.time()
    g = gen.rmat(scale, 16, 0.57, 0.19, 0.19, seed=1, symmetrize=True)
    return g, time.time() - t0


# The Twitter-shaped power-law graph: Chung-Lu, 41.6M vertices, 1.47e9 distinct
# directed edges, out/in weights of density ~ w^-2 up to 3e6 (seed 4).
CHUNGLU = dict(n=41_600_000, edges=1_470_000_000, w_max=3e6, seed=4)


def tune_graph(G, g):
    """The launch configuration every leg times (and the full-size parity
    tests check): the batched path's parameters tuned on 1024 seeds with k
    mixed over {1,2,3,6}, like the batched leg; the plain path's grid shape,
    push tile and direction parameters on 620 queries drawn like the paper
    protocol, like the headline.  Both samples come from seed stream 9, not
    the measured seeds.  Returns the khop_tuning in effect."""
    tb = G.autotune(gen.seeds(g, 1024, seed=9), ks=gen.mixed_ks(1024, seed=9))
    s9, k9 = paper_queries(g, seed=9)
    tp = G.autotune(s9, ks=k9)
    G.set_tuning(direction=tp.direction, alpha=tp.alpha, beta=tp.beta, block_threads=tp.block_threads,
                 blocks_per_sm=tp.blocks_per_sm, push_tile=tp.push_tile, batch_alpha=tb.batch_alpha,
                 batch_beta=tb.batch_beta, batch_push_tile=tb.batch_push_tile)
    return G.tuning()


def workload(args):
    """(graph, workload name, batched query count)"""
    t0 = time.time()
    if args.workload == "chunglu":
        g = gen.cached("chunglu", **CHUNGLU)
        name = (f"chunglu-n41.6M-m{g.nnz}-wmax3e6-seed4 directed plain 300/300/10/10 seeds "
                f"k=1/2/3/6")
        return g, name, 1024, time.time() - t0
    g = gen.rmat(args.scale, 16, 0.57, 0.19, 0.19, seed=1, symmetrize=True)
    return g, f"kronecker-s{args.scale}-ef16-sym plain 300/300/10/10 seeds k=1/2/3/6", 4096, \
        time.time() - t0


def paper_queries(g, scale_seeds=1.0, seed=2):
    """300/300/10/10 seeds (seed stream 2 for the measured queries, uniform
    over out-degree > 0); the first 300 draws serve k = 1 and 2, the first 10
    serve k = 3 and 6."""
    s = gen.seeds(g, 300, seed=seed)
    seeds, ks = [], []
    for k, cnt in PAPER_QUERIES:
        c = max(1, int(round(cnt * scale_seeds)))
        seeds.append(s[:c])
        ks.append(np.full(c, k, np.uint32))
    return np.concatenate(seeds).astype(np.uint32), np.concatenate(ks)


KERNEL_SOURCES = {   # a kernel's code and the graph layout it reads
    "plain_kernel": ("khop_plain.cu", "khop_internal.cuh", "khop_graph.cu"),
    "batch_kernel": ("khop_batch.cu", "khop_internal.cuh", "khop_graph.cu"),
}


def kernel_source_sha(kernel):
    """sha256 over the source files a kernel is built from."""
    import hashlib
    h = hashlib.sha256()
    for f in KERNEL_SOURCES[kernel]:
        with open(os.path.join(ROOT, "paper_1905_01294_gb300", "csrc", f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def captured_traffic(kernel, workload):
    """DRAM bytes per launch of `kernel` on this benchmark's workload, from the
    committed ncu summary profiles/roofline_traffic.md, or None if the kernel's
    source changed since that capture or the capture was taken on another
    workload (the summary holds the default scale-21 Kronecker workload)."""
    if workload != "kronecker21":
        return None
    path = os.path.join(ROOT, "profiles", "roofline_traffic.md")
    try:
        text = open(path).read()
    except OSError:
        return None
    import re
    m = re.search(rf"^- {kernel}: dram_bytes_per_launch=(\d+) source_sha256=([0-9a-f]+)", text, re.M)
    if not m or m.group(2) != kernel_source_sha(kernel):
        return None
    return int(m.group(1))


def over_ranks(dist, t_local, queries_local, device):
    """Whole-job throughput of independent replicas: the slowest rank's time
    (MAX) and every rank's queries (SUM).  Returns (t_max, queries, qps)."""
    import torch
    t = torch.tensor([float(t_local)], dtype=torch.float64, device=device)
    q = torch.tensor([float(queries_local)], dtype=torch.float64, device=device)
    if dist is not None:
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        dist.all_reduce(q, op=dist.ReduceOp.SUM)
    return float(t.item()), int(q.item()), float(q.item()) / float(t.item())


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 200 ms."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.rows = []
        self.proc = None
        cmd = ["nvidia-smi", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
               "-lms", "200"]
        if uuid:
            cmd += ["-i", uuid]
        try:
            self.proc = subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.DEVNULL,
                                         text=True)
        except Exception:
            self.proc = None
            return
        self.t = threading.Thread(target=self._read, daemon=True)
        self.t.start()

    def _read(self):
        for line in self.proc.stdout:
            parts = [x.strip() for x in line.split(",")]
            if len(parts) >= 9:
                self.rows.append(parts)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        self.t.join(timeout=2)
        if not self.rows:
            return None
        sm = [float(r[1]) for r in self.rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in self.rows if r[2].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in self.rows for i in range(4)
                          if r[5 + i].lower().startswith("active")})
        return {"sm_mhz": float(np.median(sm)) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(self.rows)}


def percentiles(x):
    x = np.asarray(x, dtype=np.float64)
    if x.size == 0:
        return {}
    return {"p50": float(np.percentile(x, 50)), "p99": float(np.percentile(x, 99)),
            "p999": float(np.percentile(x, 99.9)), "mean": float(x.mean())}


# ---------------------------------------------------------------------------
def cpu_baseline(g, seeds, ks, budget_s=25.0):
    """The oracle as it stands, one query at a time on one host thread (the
    paper's one-query-one-core model), on a bounded sample of the workload:
    for each k, the first seeds of that k until the k's share of the time
    budget is used.  Returns queries/s for the workload's k mix."""
    import oracle
    per_k = {}
    t_all = time.time()
    for k, cnt in PAPER_QUERIES:
        sel = seeds[ks == k]
        done, spent = 0, 0.0
        while done < sel.size and spent < budget_s / len(PAPER_QUERIES):
            t0 = time.perf_counter()
            oracle.khop_counts(g, sel[done:done + 1], k, nthreads=1)
            spent += time.perf_counter() - t0
            done += 1
        per_k[k] = (done, spent)
    t_workload = sum(per_k[k][1] / per_k[k][0] * (ks == k).sum() for k, _ in PAPER_QUERIES
                     if per_k[k][0])
    sample = ", ".join(f"k={k}: {per_k[k][0]} queries" for k, _ in PAPER_QUERIES)
    return {"value": float(seeds.size / t_workload), "unit": "queries/s", "cores": 1,
            "kind": "oracle",
            "sample": f"{sample} of the 620-query workload, one host thread, "
                      f"{time.time() - t_all:.1f} s; rate weighted by the workload's k mix"}


def cpu_pool_baseline(g, seeds, ks, sample):
    """The oracle as it stands on every host core, one query per thread (a
    thread pool: the paper's concurrency model for many clients), over the
    first `sample` queries of the batched workload.  Returns queries/s."""
    import oracle
    oracle.build()
    n = int(min(sample, seeds.size))
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    oracle.khop_counts(g, seeds[:n], ks[:n], nthreads=cores, with_te=False)
    dt = time.perf_counter() - t0
    return {"value": n / dt, "unit": "queries/s", "cores": cores, "kind": "oracle",
            "sample": f"the first {n} of the batched leg's queries (k mixed), one query per "
                      f"host thread at a time, {dt:.1f} s"}


def push_equivalent_bytes(te, below, width):
    """Bytes a push-only traversal of the same queries streams (the reference
    against which a direction choice that saves bytes shows up as speed):
    per query 4 * TE + (2W + 8) * |{u : dist(s, u) < k}| -- the expanded
    vertices' edge indices, row offsets and queue entries."""
    te = np.asarray(te, dtype=np.float64)
    below = np.asarray(below, dtype=np.float64)
    return float(np.sum(4.0 * te + (2.0 * width + 8.0) * below))


def workload_config(wname, g, queries_per_step, world):
    """The `config` object both arms print for the same workload."""
    return {"workload": wname, "n": int(g.n), "nnz": int(g.nnz),
            "queries_per_step": int(queries_per_step),
            "protocol": "sequential: one query at a time, in the paper's order",
            "l2": "GPU arm: flushed between steps (256 MiB write); the edge array (254 MB at "
                  "scale 21) exceeds the 129 MB L2",
            "parallelism": "replicas" if world > 1 else "single"}


REFERENCE_BUDGET_S = 180.0   # the reference arm's warm-up + timed steps, about


def run_reference(args):
    """The CPU reference arm: the oracle as it stands, one query at a time on
    one host thread, over the same workload and queries as the GPU arm.  Each
    step runs every query of the step and is timed whole; if K + W full steps
    (~4.4 s each at scale 21) would exceed the budget, each step takes the
    same leading fraction of every k's seeds instead (the k mix kept), and
    `queries_per_step`, `value` and `ms_per_step` describe what ran."""
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    if rank != 0:
        return 0
    g, wname, _, _ = workload(args)
    seeds, ks = paper_queries(g)
    import oracle
    oracle.build()
    # time one full pass of each k's first query to size the steps
    t_q = {}
    for k, _c in PAPER_QUERIES:
        s0 = seeds[ks == k][:1]
        t0 = time.perf_counter()
        oracle.khop_counts(g, s0, k, nthreads=1)
        t_q[k] = time.perf_counter() - t0
    est = sum(t_q[k] * c for k, c in PAPER_QUERIES)
    frac = min(1.0, REFERENCE_BUDGET_S / max(est * (args.steps + args.warmup), 1e-9))
    sel_s, sel_k = [], []
    for k, c in PAPER_QUERIES:
        m = max(1, int(round(c * frac)))
        sel_s.append(seeds[ks == k][:m])
        sel_k.append(np.full(m, k, np.uint32))
    ss, sk = np.concatenate(sel_s), np.concatenate(sel_k)

    def step():
        for s, k in zip(ss.tolist(), sk.tolist()):
            oracle.khop_counts(g, [s], k, nthreads=1)

    for _ in range(args.warmup):
        step()
    t0 = time.perf_counter()
    for _ in range(args.steps):
        step()
    t_work = time.perf_counter() - t0
    value = ss.size * args.steps / t_work
    ms = t_work / args.steps * 1e3
    sample = (f"every one of the {ss.size} queries of each step, timed whole" if frac >= 1.0 else
              f"{ss.size} of the 620 queries per step (the leading {frac:.2f} of each k's seeds)")
    line = {"impl": "reference", "metric": "k-hop queries/sec (plain sequential, paper protocol)",
            "value": value, "unit": "queries/s", "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
            "config": workload_config(wname, g, ss.size, world),
            "cpu_baseline": {"value": value, "unit": "queries/s", "cores": 1, "kind": "oracle",
                             "sample": f"{sample}, one host thread (the oracle: a FIFO BFS with "
                                       "a hop limit)"},
            "e2e": {"value": value, "unit": "queries/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line))
    return 0


# ---------------------------------------------------------------------------
def batched_leg(kh, torch, G, g, dev, stream, steps, warmup, flush, peak, nq=4096, gname="",
                wkey="kronecker21"):
    """The batched multi-source form: nq seeds (seed 2) with k uniform over
    {1,2,3,6}, 64 queries per uint64 lane word, one persistent launch per
    step.  Compared with the plain single-query path on the same queries."""
    seeds = gen.seeds(g, nq, seed=2)
    ks = gen.mixed_ks(nq, seed=2)
    d_s = torch.from_numpy(seeds.view(np.int32)).to(dev)
    d_k = torch.from_numpy(ks.view(np.int32)).to(dev)
    d_o = torch.empty(nq, dtype=torch.int64, device=dev)
    d_p = torch.empty(nq, dtype=torch.int64, device=dev)
    d_te = torch.empty(nq, dtype=torch.int64, device=dev)

    def call(st):
        kh.khop_count_mixed(G.handle, d_s.data_ptr(), d_k.data_ptr(), nq, d_o.data_ptr(),
                            kh.MODE_BATCHED64, st.cuda_stream)

    call(stream)                      # first call allocates the batch state
    torch.cuda.synchronize()
    graph = torch.cuda.CUDAGraph()    # then the whole call is one captured graph
    side = torch.cuda.Stream()
    with torch.cuda.graph(graph, stream=side):
        call(side)

    def step():
        graph.replay()

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ms, byts = [], 0
    for i in range(steps):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        step()
        b.record(stream)
        b.synchronize()
        ms.append(a.elapsed_time(b))
        byts += kh.khop_batch_stats(G.handle)["bytes"]
    st = kh.khop_batch_stats(G.handle)
    got = kh.as_u64(d_o).copy()
    # the plain path on the same queries (one pass), with TE for GTEPS
    flush.fill_(7)
    a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    a.record(stream)
    kh.khop_count_ex(G.handle, d_s.data_ptr(), d_k.data_ptr(), nq, d_p.data_ptr(),
                     d_te.data_ptr(), None, None, 0, stream.cuda_stream)
    b.record(stream)
    b.synchronize()
    plain_ms = a.elapsed_time(b)
    if not np.array_equal(got, kh.as_u64(d_p)):
        raise SystemExit("batched counts differ from the plain path")
    te = int(kh.as_u64(d_te).sum())
    t = sum(ms) * 1e-3
    achieved = byts / t / 1e9
    # the same queries 128 per traversal (two lane words per vertex), same tuning
    kh.khop_count_mixed(G.handle, d_s.data_ptr(), d_k.data_ptr(), nq, d_o.data_ptr(),
                        kh.MODE_BATCHED128, stream.cuda_stream)
    torch.cuda.synchronize()
    ms128 = []
    for i in range(steps):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        kh.khop_count_mixed(G.handle, d_s.data_ptr(), d_k.data_ptr(), nq, d_o.data_ptr(),
                            kh.MODE_BATCHED128, stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        ms128.append(a.elapsed_time(b))
    if not np.array_equal(got, kh.as_u64(d_o)):
        raise SystemExit("128-lane counts differ from the 64-lane ones")
    lanes128 = {"value": nq * steps / (sum(ms128) * 1e-3), "unit": "queries/s",
                "ms_per_step": float(np.mean(ms128)), "mode": "KHOP_MODE_BATCHED128 (direct calls)"}
    # and 256 per traversal (four lane words per vertex)
    kh.khop_count_mixed(G.handle, d_s.data_ptr(), d_k.data_ptr(), nq, d_o.data_ptr(),
                        kh.MODE_BATCHED256, stream.cuda_stream)
    torch.cuda.synchronize()
    ms256 = 0.0
    for i in range(steps):
        flush.fill_(i & 0xFF)
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        kh.khop_count_mixed(G.handle, d_s.data_ptr(), d_k.data_ptr(), nq, d_o.data_ptr(),
                            kh.MODE_BATCHED256, stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        ms256 += a.elapsed_time(b)
    if not np.array_equal(got, kh.as_u64(d_o)):
        raise SystemExit("256-lane counts differ from the 64-lane ones")
    lanes256 = {"value": nq * steps / (ms256 * 1e-3), "unit": "queries/s",
                "ms_per_step": ms256 / steps, "mode": "KHOP_MODE_BATCHED256 (direct calls)"}
    # six-hop traversals alone: 1024 seeds (seed 4) at k = 6, 64 per lane word
    n6 = min(1024, nq)
    s6 = torch.from_numpy(gen.seeds(g, n6, seed=4).view(np.int32)).to(dev)
    k6 = torch.full((n6,), 6, dtype=torch.int32, device=dev)
    o6 = torch.empty(n6, dtype=torch.int64, device=dev)
    six = {"queries": n6}
    for mode, name in ((kh.MODE_BATCHED64, "lanes64"), (kh.MODE_BATCHED128, "lanes128"),
                       (kh.MODE_BATCHED256, "lanes256")):
        kh.khop_count_mixed(G.handle, s6.data_ptr(), k6.data_ptr(), n6, o6.data_ptr(), mode,
                            stream.cuda_stream)
        torch.cuda.synchronize()
        ms6, b6 = 0.0, 0
        for i in range(steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            kh.khop_count_mixed(G.handle, s6.data_ptr(), k6.data_ptr(), n6, o6.data_ptr(), mode,
                                stream.cuda_stream)
            b.record(stream)
            b.synchronize()
            ms6 += a.elapsed_time(b)
            b6 += kh.khop_batch_stats(G.handle)["bytes"]
        ach = b6 / (ms6 * 1e-3) / 1e9
        six[name] = {"value": n6 * steps / (ms6 * 1e-3), "unit": "queries/s",
                     "ms_per_call": ms6 / steps,
                     "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                  "frac": ach / peak}}
    return {"workload": f"{gname}, {nq} seeds (seed 2), k uniform over {{1,2,3,6}}, "
                        "64 queries per uint64 lane word, persistent launch replayed from a "
                        "captured CUDA graph",
            "value": nq * steps / t, "unit": "queries/s", "ms_per_step": float(np.mean(ms)),
            "gteps": te * steps / t / 1e9,
            "plain_same_queries": {"value": nq / (plain_ms * 1e-3), "unit": "queries/s",
                                   "ms": plain_ms},
            "speedup_vs_plain": (nq * steps / t) / (nq / (plain_ms * 1e-3)),
            "batches_per_step": st["batches"], "rounds_per_step": st["rounds"],
            "pull_rounds_per_step": st["pull_rounds"],
            "roofline": {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                         "frac": achieved / peak, "traffic": captured_traffic("batch_kernel", wkey),
                         "kernel": "batch_kernel (64-lane bit-sliced persistent traversal)"},
            "lanes128": lanes128, "lanes256": lanes256, "six_hop": six}


K_MIX = ((1, 0.4), (2, 0.3), (3, 0.2), (6, 0.1))


SUSTAINED = 0.98   # a rate is sustained when this fraction of it is served


def best_and_sustained(points):
    """The sweep point with the highest achieved rate, and the one with the
    highest offered rate that was sustained (None if none was)."""
    best = max(points, key=lambda x: x["achieved_qps"])
    held = [p for p in points if p["achieved_qps"] >= SUSTAINED * p["offered_qps"]]
    return best, (max(held, key=lambda x: x["offered_qps"]) if held else None)


def serving_leg(kh, G, g, plain_mean_us_by_k, nreq=100000,
                rates=(25e3, 50e3, 100e3, 150e3, 200e3, 300e3, 400e3), G2=None, g2=None, names=""):
    """Open-loop Poisson request stream (seed 3), k from {1:.4, 2:.3, 3:.2,
    6:.1}, uniform seeds over out-degree > 0, served by the continuous-
    batching server; the arrival rate rises until the server saturates
    (achieves less than 0.9 of the offered rate).  With a second resident
    graph, a seeded fair coin sends each request to one of the two.
    Latency = completion time - scheduled arrival time.  `value` is the best
    achieved rate; latency is also reported at the highest offered rate the
    server sustained, i.e. served at >= SUSTAINED of the offered rate (at 0.9 a
    rate whose queue still grows over the run passes, with a p50 of tens of
    milliseconds)."""
    plain_rate = 1.0 / sum(p * plain_mean_us_by_k[k] * 1e-6 for k, p in K_MIX)
    points, checked = [], False
    for rate in rates:
        t_arr, ks, sd = gen.poisson_stream(g, nreq, rate, seed=3, k_probs=K_MIX)
        on2 = np.zeros(nreq, bool)
        if G2 is not None:
            on2 = (gen.rand_array(gen.subkey(3, 11), 0, nreq) >> np.uint64(63)).astype(bool)
            _, _, sd2 = gen.poisson_stream(g2, nreq, rate, seed=5, k_probs=K_MIX)
            sd = np.where(on2, sd2, sd).astype(np.uint32)
        srv = kh.Server()
        srv.submit_many(G, sd[:256][~on2[:256]], ks[:256][~on2[:256]])   # warm-up: slots allocated
        if G2 is not None:
            srv.submit_many(G2, sd[:256][on2[:256]], ks[:256][on2[:256]])
        warm, tw = 0, time.time()
        while warm < 256 and time.time() - tw < 30:
            warm += len(srv.poll_arrays(4096, 100000))
        tickets = np.zeros(nreq, np.uint64)
        done = []
        t0 = time.monotonic_ns()
        i = 0
        while i < nreq:
            now = (time.monotonic_ns() - t0) * 1e-9
            j = int(np.searchsorted(t_arr, now, side="right"))
            if j > i:
                if G2 is None:
                    tickets[i:j] = srv.submit_many(G, sd[i:j], ks[i:j])
                else:   # in arrival order, one graph's run at a time
                    a = i
                    while a < j:
                        b = a + 1
                        while b < j and on2[b] == on2[a]:
                            b += 1
                        tickets[a:b] = srv.submit_many(G2 if on2[a] else G, sd[a:b], ks[a:b])
                        a = b
                i = j
            done.append(srv.poll_arrays(8192, 0))
        ndone = sum(len(x) for x in done)
        tw = time.time()
        while ndone < nreq and time.time() - tw < 120:
            x = srv.poll_arrays(8192, 100000)
            done.append(x)
            ndone += len(x)
        counters = srv.counters()
        srv.close()
        res = np.concatenate(done)
        res = res[np.argsort(res["ticket"])]
        if not np.array_equal(res["ticket"], tickets) or (res["status"] != 0).any():
            raise SystemExit("serving: missing or failed requests")
        lat_us = (res["t_done_ns"].astype(np.int64) - t0 - (t_arr * 1e9).astype(np.int64)) * 1e-3
        span = (int(res["t_done_ns"].max()) - t0) * 1e-9
        if not checked:
            # each served count equals the same query alone on the plain path
            alone = np.zeros(nreq, np.uint64)
            alone[~on2] = kh.as_u64(G.count_mixed(sd[~on2], ks[~on2], mode=kh.MODE_PLAIN))
            if G2 is not None and on2.any():
                alone[on2] = kh.as_u64(G2.count_mixed(sd[on2], ks[on2], mode=kh.MODE_PLAIN))
            if not np.array_equal(res["count"], alone):
                raise SystemExit("serving: a served count differs from the query alone")
            checked = True
        pt = {"offered_qps": rate, "achieved_qps": nreq / span, "latency_us": percentiles(lat_us),
              "latency_us_by_k": {str(k): percentiles(lat_us[ks == k]) for k, _ in K_MIX},
              "server": {k: v for k, v in counters.items()
                         if k in ("steps", "joined_running", "plain_launches", "pull_steps",
                                  "slots_allocated", "max_lanes_busy")}}
        points.append(pt)
        if pt["achieved_qps"] < 0.9 * rate:
            break
    best, top = best_and_sustained(points)
    return {"workload": f"{names} resident, open-loop Poisson (seed 3), "
                        f"{nreq} requests per rate, k ~ {{1:.4, 2:.3, 3:.2, 6:.1}}",
            "value": best["achieved_qps"], "unit": "queries/s",
            "sustained_qps": top["achieved_qps"] if top else None,
            "latency_us_at_sustained": top["latency_us"] if top else None,
            "latency_us_at_sustained_offered_qps": top["offered_qps"] if top else None,
            "plain_sequential_same_mix_qps": plain_rate,
            "speedup_vs_plain": best["achieved_qps"] / plain_rate,
            "sweep": points}


def variants_leg(kh, torch, dev, stream, scale, steps, warmup, flush):
    """The paper protocol (300/300/10/10 seeds at k = 1/2/3/6) on the directed
    scale-`scale` R-MAT graph (edges kept one-way) counted along out-edges
    (Sec. III's A^T q), in-edges (A q) and both (A OR A^T); default tuning,
    one plain launch per step, L2 flushed between steps."""
    g = gen.rmat(scale, 16, seed=1)
    seeds, ks = paper_queries(g)
    nq = seeds.size
    d_seeds = torch.from_numpy(seeds.view(np.int32)).to(dev)
    d_ks = torch.from_numpy(ks.view(np.int32)).to(dev)
    d_out = torch.empty(nq, dtype=torch.int64, device=dev)
    res = {"workload": f"kronecker-s{scale}-ef16 directed (nnz {g.nnz}), 620 paper-protocol queries, "
                       "default tuning", "unit": "queries/s"}
    for name, kw in (("out", {}), ("in", {"reverse": True}), ("either", {"undirected": True})):
        Gv = kh.Graph.from_csr(g, **kw)

        def step():
            kh.khop_count_mixed(Gv.handle, d_seeds.data_ptr(), d_ks.data_ptr(), nq, d_out.data_ptr(),
                                kh.MODE_PLAIN, stream.cuda_stream)

        for _ in range(warmup):
            step()
        torch.cuda.synchronize()
        ms = 0.0
        for i in range(steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            step()
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
        counts = kh.as_u64(d_out)
        res[name] = {"value": nq * steps / (ms * 1e-3), "mean_count": float(counts.mean()),
                     "ms_per_step": ms / steps}
        Gv.close()
    return res


def listing_leg(kh, torch, G, g, seeds, ks, counts, dev, stream):
    """The neighbourhoods themselves (khop_neighbourhood_list: ascending ids)
    for the paper protocol's (seed, k) pairs at k = 3, 6 and the first 50 at
    k = 2: sets/s and ids/s over one call each, every size checked against
    the plain count; then khop_levels (hop levels and (MIN, SECOND) parents
    of all n vertices) for the same pairs."""
    ids = torch.empty(g.n, dtype=torch.int32, device=dev)
    size = torch.zeros(1, dtype=torch.int64, device=dev)
    pick = [i for i in range(seeds.size) if ks[i] in (3, 6)] + \
        [i for i in range(seeds.size) if ks[i] == 2][:50]
    for i in pick[:3]:   # warm-up
        kh.khop_neighbourhood_list(G.handle, int(seeds[i]), int(ks[i]), ids.data_ptr(), g.n,
                                   size.data_ptr(), stream.cuda_stream)
    torch.cuda.synchronize()
    ms, total = 0.0, 0
    for i in pick:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        kh.khop_neighbourhood_list(G.handle, int(seeds[i]), int(ks[i]), ids.data_ptr(), g.n,
                                   size.data_ptr(), stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        ms += a.elapsed_time(b)
        sz = int(size.item())
        if sz != int(counts[i]) + 1:
            raise SystemExit("neighbourhood size differs from the count")
        total += sz
    # BFS levels and (MIN, SECOND) parents of the same pairs (khop_levels)
    lv = torch.empty(g.n, dtype=torch.int32, device=dev)
    par = torch.empty(g.n, dtype=torch.int32, device=dev)
    ms_l = 0.0
    for i in pick:
        a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        a.record(stream)
        kh.khop_levels(G.handle, int(seeds[i]), int(ks[i]), lv.data_ptr(), par.data_ptr(), stream.cuda_stream)
        b.record(stream)
        b.synchronize()
        ms_l += a.elapsed_time(b)
    return {"workload": f"{len(pick)} paper-protocol (seed, k) pairs at k = 2/3/6, one call each",
            "value": len(pick) / (ms * 1e-3), "unit": "sets/s", "ids_per_s": total / (ms * 1e-3),
            "mean_size": total / len(pick),
            "levels_and_parents_per_s": len(pick) / (ms_l * 1e-3)}


def measure(args, kh, torch, dev, dist, world, rank, local, g, G, wname, wkey, batched_nq, tuning,
            steps, warmup, serving_kw=None, cpu_budget_s=25.0, directions=True, listing=True,
            pool_sample=512):
    """One workload measured on its resident graph G: the paper protocol on
    the plain path (the headline metric's timed steps), its end-to-end form,
    rooflines, and the batched, listing, direction and serving legs.  Returns
    the JSON line's fields."""
    seeds, ks = paper_queries(g)
    nq = seeds.size
    stream = torch.cuda.current_stream()
    d_seeds = torch.from_numpy(seeds.view(np.int32)).to(dev)
    d_ks = torch.from_numpy(ks.view(np.int32)).to(dev)
    d_out = torch.empty(nq, dtype=torch.int64, device=dev)
    d_te = torch.empty(nq, dtype=torch.int64, device=dev)
    d_stats = torch.empty(nq * kh.QUERY_STATS_WORDS, dtype=torch.int64, device=dev)
    flush = torch.empty(256 << 20, dtype=torch.uint8, device=dev)

    def step():
        kh.khop_count_ex(G.handle, d_seeds.data_ptr(), d_ks.data_ptr(), nq, d_out.data_ptr(),
                         d_te.data_ptr(), d_stats.data_ptr(), None, 0, stream.cuda_stream)

    for _ in range(warmup):
        step()
    torch.cuda.synchronize()
    ref_counts = kh.as_u64(d_out).copy()

    uuid = None
    try:
        uuid = "GPU-" + str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    sampler = ClockSampler(uuid) if rank == 0 else None
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(steps)]
    lat, te_sum, bytes_sum = [], 0, 0
    lat_by_k = {k: [] for k, _ in PAPER_QUERIES}
    bytes_by_k = {k: 0 for k, _ in PAPER_QUERIES}
    for i in range(steps):
        flush.fill_(i & 0xFF)                       # L2 flush between steps (not timed)
        evs[i][0].record(stream)
        step()
        evs[i][1].record(stream)
        evs[i][1].synchronize()
        rec = kh.stats_records(d_stats)
        dt = (rec["t_end_ns"] - rec["t_start_ns"]).astype(np.float64) * 1e-3
        lat.extend(dt.tolist())
        for k, _ in PAPER_QUERIES:
            lat_by_k[k].extend(dt[ks == k].tolist())
            bytes_by_k[k] += int(rec["bytes"][ks == k].sum())
        te_sum += int(rec["te"].sum())
        bytes_sum += int(rec["bytes"].sum())
        if not np.array_equal(kh.as_u64(d_out), ref_counts):
            raise SystemExit("counts changed between steps")
    torch.cuda.synchronize()
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_total, queries_total, value = over_ranks(dist, sum(step_ms) * 1e-3, nq * steps, dev)
    if dist is not None:
        dist.barrier()
    clocks = sampler.stop() if sampler else None
    gteps = te_sum * world / t_total / 1e9

    # e2e: public API, pinned host inputs, counts back to the host, per step
    h_seeds = torch.from_numpy(seeds.view(np.int32)).pin_memory()
    h_ks = torch.from_numpy(ks.view(np.int32)).pin_memory()
    h_out = torch.empty(nq, dtype=torch.int64).pin_memory()
    e_seeds = torch.empty_like(d_seeds)
    e_ks = torch.empty_like(d_ks)
    e_out = torch.empty_like(d_out)
    e_t = 0.0
    for i in range(steps):
        flush.fill_(i & 0xFF)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        e_seeds.copy_(h_seeds, non_blocking=True)
        e_ks.copy_(h_ks, non_blocking=True)
        kh.khop_count_mixed(G.handle, e_seeds.data_ptr(), e_ks.data_ptr(), nq, e_out.data_ptr(),
                            kh.MODE_PLAIN, stream.cuda_stream)
        h_out.copy_(e_out, non_blocking=True)
        stream.synchronize()
        e_t += time.perf_counter() - t0
        if not np.array_equal(h_out.numpy().view(np.uint64), ref_counts):
            raise SystemExit("e2e counts differ")
    _, _, e2e_qps = over_ranks(dist, e_t, nq * steps, dev)
    e2e = {"value": e2e_qps, "unit": "queries/s",
           "h2d_bytes_per_step": int(seeds.nbytes + ks.nbytes),
           "d2h_bytes_per_step": int(nq * 8)}

    peak, peak_kind = load_peaks()
    achieved = bytes_sum / t_total / 1e9   # per GPU: one rank's kernel bytes over the max time
    traffic = captured_traffic("plain_kernel", wkey)
    roofline = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s",
                "frac": achieved / peak, "traffic": traffic,
                "kernel": "plain_kernel (persistent push/pull traversal)",
                "peak_kind": peak_kind,
                # the captured DRAM bytes per step over this run's mean step time
                "dram_gbs": (traffic / (t_total / steps) / 1e9) if traffic else None}
    # push-equivalent bytes: |{u : dist(s, u) < k}| = count(s, k - 1) + 1, from
    # one untimed plain call at k - 1; TE from the last timed step
    try:   # an auxiliary figure: the headline line is printed whatever happens here
        d_kp = torch.from_numpy((np.maximum(ks, 1) - 1).astype(np.uint32).view(np.int32)).to(dev)
        d_cp = torch.empty(nq, dtype=torch.int64, device=dev)
        kh.khop_count_mixed(G.handle, d_seeds.data_ptr(), d_kp.data_ptr(), nq, d_cp.data_ptr(),
                            kh.MODE_PLAIN, stream.cuda_stream)
        torch.cuda.synchronize()
        b_ref = push_equivalent_bytes(kh.as_u64(d_te), kh.as_u64(d_cp).astype(np.float64) + 1.0,
                                      4 if g.nnz < 2**32 else 8)
        a_ref = b_ref * steps / t_total / 1e9
        roofline["push_equivalent"] = {"bytes_per_step": b_ref, "achieved": a_ref,
                                       "frac": a_ref / peak}
    except Exception as exc:   # noqa: BLE001
        print(f"push-equivalent bytes not computed: {exc}", file=sys.stderr)
        roofline["push_equivalent"] = None
    # per k: the queries' algorithmic bytes over their device-timestamp latencies
    roofline_by_k = {}
    for k, _ in PAPER_QUERIES:
        t_k = float(np.sum(lat_by_k[k])) * 1e-6
        if t_k > 0:
            a_k = bytes_by_k[k] / t_k / 1e9
            roofline_by_k[str(k)] = {"achieved": a_k, "frac": a_k / peak,
                                     "bytes_per_query": bytes_by_k[k] / max(1, len(lat_by_k[k]))}

    extras = {}
    if not args.no_extras:
        extras["batched"] = batched_leg(kh, torch, G, g, dev, stream, steps, warmup,
                                        flush, peak, nq=batched_nq, gname=wname.split(" ")[0],
                                        wkey=wkey)
        if listing:
            extras["listing"] = listing_leg(kh, torch, G, g, seeds, ks, ref_counts, dev, stream)
        if directions:
            extras["directions"] = variants_leg(kh, torch, dev, stream, args.scale, steps,
                                                warmup, flush)
            extras["mxv"] = mxv_leg(kh, torch, G, g, stream, steps, flush, peak)
        if serving_kw is not None:
            mean_by_k = {k: float(np.mean(v)) for k, v in lat_by_k.items()}
            extras["serving"] = serving_leg(kh, G, g, mean_by_k, **serving_kw)
    lat_p = percentiles(lat)
    line = {
        "metric": "k-hop queries/sec (plain sequential, paper protocol)",
        "value": value, "unit": "queries/s", "n_gpus": world, "steps": steps,
        "warmup": warmup, "ms_per_step": float(np.mean(step_ms)),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u32",
        "data": "synthetic",
        "config": workload_config(wname, g, nq, world),
        "tuning": tuning,
        "gteps": gteps,
        "latency_us": lat_p,
        "latency_us_by_k": {str(k): percentiles(v) for k, v in lat_by_k.items()},
        "e2e": e2e,
        "roofline": roofline,
        "roofline_by_k": roofline_by_k,
        "gpu_launches": steps,   # one persistent plain_kernel launch per step
        "clocks": clocks,
    }
    line.update(extras)
    if rank == 0 and world == 1 and not args.no_cpu:
        line["cpu_baseline"] = cpu_baseline(g, seeds, ks, budget_s=cpu_budget_s)
        if "batched" in line:
            try:   # an auxiliary baseline: the headline line is printed whatever happens here
                line["batched"]["cpu_pool"] = cpu_pool_baseline(
                    g, gen.seeds(g, batched_nq, seed=2), gen.mixed_ks(batched_nq, seed=2),
                    sample=pool_sample)
            except Exception as exc:   # noqa: BLE001
                print(f"thread-pool oracle baseline not measured: {exc}", file=sys.stderr)
    return line


def power_law_leg(args, kh, torch, dev, dist, world, rank, local, G2, g2):
    """The 41.6M-vertex, 1.47e9-edge power-law graph (read from the on-disk
    cache when present): the paper protocol on the plain path, 1024 batched
    queries, and serving with both graphs resident (20k requests per rate)."""
    t0 = time.time()
    gl = gen.cached("chunglu", **CHUNGLU)
    t_gen = time.time() - t0
    GL = kh.Graph.from_csr(gl)
    t = tune_graph(GL, gl)
    tuning = {f: (getattr(t, f) if isinstance(getattr(t, f), int) else round(getattr(t, f), 3))
              for f, _ in t._fields_}
    name = (f"chunglu-n41.6M-m{gl.nnz}-wmax3e6-seed4 directed plain 300/300/10/10 seeds "
            f"k=1/2/3/6")
    sub = measure(args, kh, torch, dev, dist, world, rank, local, gl, GL, name, "chunglu", 1024,
                  tuning, min(args.steps, 5), min(args.warmup, 3),
                  serving_kw=None if args.no_serving else dict(
                      G2=G2, g2=g2, nreq=20000, rates=(2.5e3, 5e3, 10e3, 20e3, 40e3, 80e3, 160e3),
                      names="chunglu-41.6M/1.47e9 and kronecker-s21"),
                  cpu_budget_s=10.0, directions=False, listing=False, pool_sample=64)
    sub["graph_load_s"] = t_gen
    GL.close()
    return sub


def mxv_leg(kh, torch, G, g, stream, steps, flush, peak):
    """khop_mxv over the whole graph for each semiring (x: seeded random
    values, a third of them the "no entry" identity; no mask), and OR_AND as
    a BFS step (the frontier at distance 2 from a seed, the visited set as the
    complemented mask).  Algorithmic bytes per call: 2W n (column offsets) +
    8 n (y) + (4 + 8) per in-edge examined (index, x gather) + n/8 (mask)."""
    rng = np.random.default_rng(11)
    W = 4 if g.nnz < 2**32 else 8
    res = {"workload": f"{g.n} vertices, {g.nnz} edges, one call per step, L2 flushed between steps",
           "unit": "calls/s"}
    cases = []
    for sr, name in ((kh.SR_OR_AND, "or_and"), (kh.SR_PLUS_TIMES, "plus_times"),
                     (kh.SR_MIN_SECOND, "min_second"), (kh.SR_MAX_SECOND, "max_second")):
        x = rng.integers(1, 2**40, g.n, dtype=np.uint64)
        x[rng.random(g.n) < 0.33] = np.uint64(2**64 - 1) if sr == kh.SR_MIN_SECOND else np.uint64(0)
        cases.append((name, sr, torch.from_numpy(x.view(np.int64)).cuda(), None))
    s0 = int(gen.seeds(g, 1, seed=13)[0])
    lv, _ = G.levels(s0, 2, parents=False)
    lvh = lv.cpu().numpy()
    q = (lvh == 2).astype(np.uint64)
    vis = np.nonzero(lvh >= 0)[0]
    words = np.zeros((g.n + 31) // 32, np.uint32)
    np.bitwise_or.at(words, vis >> 5, np.uint32(1) << (vis & 31).astype(np.uint32))
    cases.append(("or_and_bfs_step", kh.SR_OR_AND, torch.from_numpy(q.view(np.int64)).cuda(),
                  torch.from_numpy(words.view(np.int32)).cuda()))
    y = torch.empty(g.n, dtype=torch.int64, device="cuda")
    for name, sr, xd, md in cases:
        call = lambda: kh.khop_mxv(G.handle, sr, xd.data_ptr(), md.data_ptr() if md is not None else None,
                                   1 if md is not None else 0, y.data_ptr(), stream.cuda_stream)
        call()
        torch.cuda.synchronize()
        scanned = kh.khop_mxv_stats(G.handle)
        ms = 0.0
        for i in range(steps):
            flush.fill_(i & 0xFF)
            a, b = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            a.record(stream)
            call()
            b.record(stream)
            b.synchronize()
            ms += a.elapsed_time(b)
        t = ms * 1e-3 / steps
        byts = 2 * W * g.n + 8 * g.n + 12 * scanned + (g.n // 8 if md is not None else 0)
        ach = byts / t / 1e9
        res[name] = {"value": 1.0 / t, "us_per_call": t * 1e6, "in_edges_scanned": scanned,
                     "roofline": {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s",
                                  "frac": ach / peak}}
    return res


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--scale", type=int, default=21)
    ap.add_argument("--workload", default="kronecker21", choices=["kronecker21", "chunglu"],
                    help="kronecker21: the scale-21 Graph500-shaped graph (default); chunglu: "
                         "the 41.6M-vertex, 1.47e9-edge power-law graph")
    ap.add_argument("--no-cpu", action="store_true", help="skip the CPU baseline leg")
    ap.add_argument("--no-extras", action="store_true", help="plain path only")
    ap.add_argument("--no-serving", action="store_true", help="skip the serving sweep")
    ap.add_argument("--no-large", action="store_true",
                    help="skip the power-law (41.6M-vertex) leg of the default run")
    ap.add_argument("--case", choices=["plain6", "batch6", "mxv"],
                    help="run one launch of a small case (for a profiler) and exit: plain6 = "
                         "10 six-hop queries on the plain path, batch6 = 128 six-hop queries "
                         "(two 64-lane batches), mxv = two PLUS_TIMES khop_mxv calls over the graph "
                         "(the first also lists the hub chunks: plan, vertex and chunk kernels, "
                         "then vertex and chunk kernels)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import paper_1905_01294_gb300 as kh

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    torch.cuda.set_device(local)
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    dev = torch.device("cuda", local)
    kh.lib()

    g, wname, batched_nq, t_gen = workload(args)
    seeds, ks = paper_queries(g)
    nq = seeds.size
    G = kh.Graph.from_csr(g)
    if not args.case:
        t = tune_graph(G, g)
        tuning = {f: (getattr(t, f) if isinstance(getattr(t, f), int) else round(getattr(t, f), 3))
                  for f, _ in t._fields_}
    if args.case == "mxv":
        x = np.random.default_rng(11).integers(1, 2**40, g.n, dtype=np.uint64)
        y = G.mxv(kh.SR_PLUS_TIMES, x)
        y = G.mxv(kh.SR_PLUS_TIMES, x)
        torch.cuda.synchronize()
        print(json.dumps({"case": "mxv", "y_head": kh.as_u64(y)[:4].tolist()}))
        G.close()
        return 0
    if args.case:
        cs = gen.seeds(g, 128 if args.case == "batch6" else 10, seed=2)
        out = G.count_mixed(cs, np.full(cs.size, 6, np.uint32),
                            mode=kh.MODE_BATCHED64 if args.case == "batch6" else kh.MODE_PLAIN)
        torch.cuda.synchronize()
        print(json.dumps({"case": args.case, "queries": int(cs.size),
                          "counts_head": kh.as_u64(out)[:4].tolist()}))
        G.close()
        return 0
    line = measure(args, kh, torch, dev, dist, world, rank, local, g, G, wname, args.workload,
                   batched_nq, tuning, args.steps, args.warmup,
                   serving_kw=None if (args.no_extras or args.no_serving) else (
                       dict(names=wname.split(" ")[0]) if args.workload == "kronecker21" else
                       dict(G2=None, names=wname.split(" ")[0], rates=(2.5e3, 5e3, 10e3, 20e3, 40e3, 80e3))),
                   directions=args.workload == "kronecker21",
                   pool_sample=512 if args.workload == "kronecker21" else 128)
    if args.workload == "kronecker21" and not args.no_extras and not args.no_large:
        # the Twitter-shaped power-law graph (41.6M vertices, 1.47e9 edges), with
        # the scale-21 graph still resident for two-graph serving
        try:
            line["chunglu"] = power_law_leg(args, kh, torch, dev, dist, world, rank, local, G, g)
        except Exception as exc:   # noqa: BLE001 -- the headline line is printed regardless
            print(f"power-law leg not measured: {exc}", file=sys.stderr)
            line["chunglu"] = {"unavailable": str(exc)[:300]}
    if rank == 0:
        print(json.dumps(line))
    G.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
