"""The benchmark's host-side parts without a GPU: the reference (oracle) arm's JSON line,
and the max-over-ranks timing reduction with two gloo ranks."""
import json
import os
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_reference_arm_prints_one_json_line():
    if ROOT not in sys.path:
        sys.path.insert(0, ROOT)
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "2",
                        "--warmup", "0", "--cpu-sample-bands", "1"], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "band-applies/s"
    import bench
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] == bench.host_cores()
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["higher_is_better"] is True
    # ms_per_step is the measured mean step of what ran: bands per step / value
    bands = d["config"]["sample_bands_per_step"]
    assert abs(d["ms_per_step"] - 1e3 * bands / d["value"]) <= 1e-6 * d["ms_per_step"]
    assert d["config"]["workload"] == bench.WORKLOAD


def _worker(rank, world, port, q):
    import torch
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    sys.path.insert(0, ROOT)
    import bench
    out = bench.max_over_ranks([1.0 + rank, 5.0 - rank], torch.device("cpu"))
    q.put((rank, out))
    dist.destroy_process_group()


def test_max_over_ranks_two_gloo_ranks():
    import multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = 29500 + os.getpid() % 1000
    ps = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in ps:
        p.start()
    res = dict(q.get(timeout=120) for _ in ps)
    for p in ps:
        p.join(timeout=60)
    assert res[0] == [2.0, 5.0] and res[1] == [2.0, 5.0]
