"""bench.py's reference arm times the CPU oracle alone: it runs without a GPU,
prints one JSON line with the contract's keys, and only rank 0 prints."""
import json
import os
import subprocess
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
KEYS = ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
        "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e")


def _run(env_extra, wall=None):
    import time
    env = dict(os.environ, **env_extra)
    t0 = time.time()
    r = subprocess.run([sys.executable, "bench.py", "--impl", "reference", "--scale", "12",
                        "--steps", "2", "--warmup", "1"], cwd=ROOT, env=env, capture_output=True,
                       text=True, timeout=300)
    if wall is not None:
        wall.append(time.time() - t0)
    assert r.returncode == 0, r.stderr[-2000:]
    return [ln for ln in r.stdout.splitlines() if ln.strip()]


def test_reference_arm_prints_one_contract_line():
    wall = []
    lines = _run({}, wall)
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference"
    for k in KEYS:
        assert k in d, k
    assert d["value"] > 0 and d["unit"] == "queries/s" and d["higher_is_better"] is True
    assert d["steps"] == 2 and d["warmup"] == 1
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["value"] == d["value"]
    assert d["e2e"]["value"] == d["value"]
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0
    # the timed region really ran: every query of each step, inside the process's lifetime
    assert d["config"]["queries_per_step"] == 620
    assert d["steps"] * d["ms_per_step"] * 1e-3 < wall[0]
    assert abs(d["value"] - 620 / (d["ms_per_step"] * 1e-3)) < 1e-6 * d["value"]
    # the same config object as the GPU arm prints for this workload
    b = _bench()
    assert set(d["config"]) == set(b.workload_config("w", _G(), 620, 1))


def _G():
    import gen
    return gen.path_graph(3)


def test_reference_arm_other_ranks_print_nothing():
    assert _run({"RANK": "1", "WORLD_SIZE": "2"}) == []


def _bench():
    import importlib.util
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(ROOT, "bench.py"))
    m = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(m)
    return m


def test_thread_pool_oracle_baseline():
    import gen
    b = _bench()
    g = gen.rmat(12, 16, seed=1, symmetrize=True)
    r = b.cpu_pool_baseline(g, gen.seeds(g, 256, seed=2), gen.mixed_ks(256, seed=2), sample=64)
    assert r["value"] > 0 and r["cores"] >= 1 and r["kind"] == "oracle" and "64" in r["sample"]


def test_push_equivalent_bytes_closed_form():
    """A directed path 0 -> 1 -> ... -> 9 from vertex 0 at k = 3 expands
    vertices 0, 1, 2 (dist < 3) with one out-edge each: 4 * 3 + (2W + 8) * 3."""
    import gen
    import oracle
    b = _bench()
    g = gen.path_graph(10)
    c, te = oracle.khop_counts(g, [0], [3])
    below, _ = oracle.khop_counts(g, [0], [2])
    got = b.push_equivalent_bytes(te, below.astype(float) + 1.0, 4)
    assert int(te[0]) == 3 and got == 4 * 3 + (2 * 4 + 8) * 3
