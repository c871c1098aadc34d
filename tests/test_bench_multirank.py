"""bench.py's multi-rank aggregation on CPU with two gloo ranks: the slowest rank's time
sets the step time and the value counts every rank's work."""
import os
import socket

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    ms_local = 100.0 if rank == 0 else 250.0
    out = bench.aggregate(ms_local, 10, 1_000_000, world, "cpu")
    q.put((rank, out))
    dist.destroy_process_group()


def test_two_rank_aggregation():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
    for rank in (0, 1):
        ms_per_step, value = res[rank]
        assert ms_per_step == pytest.approx(25.0)
        assert value == pytest.approx(2 * 1_000_000 / 0.025 / 1e9)


def test_reference_arm_json_line():
    """bench.py --impl reference (the FP64 oracle on the host cores) prints one JSON line with
    the contract's keys, at a small level so the check stays short."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--level", "2",
                          "--steps", "2", "--warmup", "1", "--cpu-seconds", "1"],
                         capture_output=True, text=True, timeout=600, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [l for l in out.stdout.splitlines() if l.strip().startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["unit"] == "GDoF/s" and d["value"] > 0 and d["higher_is_better"]
    assert d["steps"] == 2 and d["warmup"] == 1 and d["ms_per_step"] > 0
    assert {"value", "unit", "cores", "kind", "sample"} <= set(d["cpu_baseline"]) and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert {"apply_L2_gdofs", "apply_L3_gdofs", "apply_L4_gdofs", "solve_L2_s"} <= set(d["oracle_levels"])
    assert d["cpu_baseline_all_cores"]["value"] > 0 and d["cpu_baseline_all_cores"]["cores"] >= 1
