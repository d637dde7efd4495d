"""The N > 1 path of bench.py on CPU: two gloo ranks (no GPU).

Proteins are independent, so ranks shard the batch with no data-path
collective; the only exchange is the max over ranks of the step time.  These
tests check the sharding (disjoint seeds, N x batch distinct proteins), the
max-over-ranks reduction and the whole-job rate, and that the reference arm
under torchrun prints exactly one line, from rank 0.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    seeds = bench.shard_seeds(4, rank)
    everyone = [None] * world
    dist.all_gather_object(everyone, seeds)
    # a slow rank: its time must win
    elapsed = bench.max_over_ranks(1.0 + 2.0 * rank, dist, "cpu")
    rate = bench.job_rate(4, world, 3, elapsed)
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"seeds": everyone, "elapsed": elapsed, "rate": rate}, f)
    dist.destroy_process_group()


def test_two_gloo_ranks_shard_and_take_the_max(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True,
                       start_method="spawn")
    r0 = json.load(open(tmp_path / "rank0.json"))
    r1 = json.load(open(tmp_path / "rank1.json"))
    assert r0 == r1
    s0, s1 = r0["seeds"]
    assert len(s0) == len(s1) == 4 and not set(s0) & set(s1)
    assert r0["elapsed"] == 3.0                      # the slower rank's time
    assert r0["rate"] == pytest.approx(4 * 2 * 3 / 3.0)


def test_reference_arm_under_torchrun_prints_once():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py",
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--cpu-sample-aa", "10"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
