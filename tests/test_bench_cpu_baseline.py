"""The bench's CPU baseline on every host core: spawned processes, each
stepping the unchanged oracle on its own band of the workload, started
together.  Checked on the CPU with small bands: the pool reports the cell
updates of all bands and the worker keeps its command protocol."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_oracle_pool_counts_every_band_and_times_the_slowest():
    sys.path.insert(0, ROOT)
    import bench

    with bench.OraclePool(2, rows=8) as pool:
        cells, dt = pool.step(2)
        assert cells == 2 * 2048 * 8 * 2
        assert dt > 0
        cells1, _ = pool.step(1)
        assert cells1 == 2 * 2048 * 8


def test_band_worker_protocol_in_process():
    """The worker announces itself once its oracle is built, then answers each
    step command after the barrier with that step's time, and exits on None."""
    import queue
    import threading

    sys.path.insert(0, ROOT)
    import bench

    cmd, res = queue.Queue(), queue.Queue()
    for n in (1, 2, None):
        cmd.put(n)
    bench._oracle_band_worker(3, 8, cmd, res, threading.Barrier(1))
    got = [res.get_nowait() for _ in range(3)]
    assert got[0] == (3, 0.0)
    assert [b for b, _ in got] == [3, 3, 3] and all(dt > 0 for _, dt in got[1:])
    assert res.empty()


def test_reference_arm_prints_one_contract_line():
    """`bench.py --impl reference` on the CPU: one JSON line with the
    benchmark's keys, the oracle as the reference, its own e2e figure."""
    import json
    import subprocess

    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "1"], capture_output=True, text=True, timeout=600, cwd=ROOT)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "scaling",
              "vs_baseline", "dtype", "data", "config", "impl", "cpu_baseline", "e2e"):
        assert k in d, k
    assert d["impl"] == "reference" and d["steps"] == 2 and d["warmup"] == 1 and d["value"] > 0
    assert d["unit"] == "MLUPS" and d["higher_is_better"] is True and d["vs_baseline"] is None
    assert d["config"]["workload"]
    cb = d["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == d["value"] and cb["sample"]
    assert d["e2e"] == {"value": d["value"], "unit": "MLUPS", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}
