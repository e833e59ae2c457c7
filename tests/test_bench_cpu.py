"""Host-side pieces of bench.py: replica aggregation over gloo ranks (world size 2, CPU) and
the reference arm's JSON line (the CPU oracle on a small workload)."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, ws, port, q):
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws)})
    sys.path.insert(0, ROOT)
    import torch.distributed as tdist

    import bench

    tdist.init_process_group("gloo", rank=rank, world_size=ws)
    t = bench.max_over_ranks(1.0 + rank, ws)
    v = bench.whole_job_value(100.0, ws, t)
    tdist.destroy_process_group()
    q.put((rank, t, v))


def test_replica_aggregation_gloo_world2():
    import multiprocessing as mp
    import socket

    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    res = sorted(q.get(timeout=5) for _ in range(2))
    assert all(t == 2.0 for _, t, _ in res)  # max over ranks
    assert all(v == 100.0 for _, _, v in res)  # 2 replicas x 100 units / 2 s


def test_reference_arm_json_line():
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload", "tiny",
                          "--steps", "2", "--warmup", "1"], capture_output=True, text=True, timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr
    lines = [l for l in out.stdout.splitlines() if l.strip()]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better", "impl",
              "cpu_baseline", "e2e", "config"):
        assert k in d
    assert d["impl"] == "reference" and d["value"] > 0 and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
