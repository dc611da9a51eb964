"""The N > 1 launch of bench.py on CPU (gloo, world size 2).

The worlds of different ranks are independent ("replicas only": no
collective on the data path); the only collectives are the timing barrier and
the final reduction, where the job's time is the slowest rank's and its work
the sum over ranks.  These tests run that reduction on two gloo ranks, and the
reference arm under torch.distributed.run, where rank 0 alone prints one line.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_stats(rank: int):
    # times (ms, s) then units (agent-steps, cell-steps, e2e agent-steps)
    return [10.0 * (rank + 1), 3.0 - rank, 1000.0 + rank, 80000.0, 7.0 * (rank + 1)]


def _reduce_worker(rank, world_size, port, out_dir):
    import torch
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world_size)
    try:
        stats = torch.tensor(_rank_stats(rank), dtype=torch.float64)
        got = bench.reduce_over_ranks(stats, dist, n_times=2)
        with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
            json.dump(got, f)
    finally:
        dist.destroy_process_group()


def test_reduce_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.start_processes(_reduce_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws,
                       join=True, start_method="spawn")
    per = [_rank_stats(r) for r in range(ws)]
    want = [max(p[0] for p in per), max(p[1] for p in per)] + \
        [sum(p[i] for p in per) for i in range(2, 5)]
    for r in range(ws):
        with open(tmp_path / f"rank{r}.json") as f:
            assert json.load(f) == pytest.approx(want, rel=0, abs=0)


def test_reduce_without_process_group():
    import torch
    sys.path.insert(0, ROOT)
    import bench
    stats = torch.tensor(_rank_stats(0), dtype=torch.float64)
    assert bench.reduce_over_ranks(stats, None, n_times=2) == _rank_stats(0)


def test_reference_arm_two_ranks():
    """Rank 1 exits 0 without work or output; rank 0 prints one JSON line."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "3", "--warmup", "3", "--workload", "small_20x40", "--cpu-cores", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["unit"] == "agent-steps/s"
    assert line["cpu_baseline"]["kind"] == "oracle" and line["cpu_baseline"]["cores"] == 1
    assert line["e2e"]["h2d_bytes_per_step"] == 0 and line["e2e"]["value"] == line["value"]
    assert line["config"]["parallelism"] == "replicas2"
