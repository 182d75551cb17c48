"""The multi-process path of bench.py on the CPU: two gloo ranks.

Back-projection shards into independent problems, so N GPUs run N replicas
(each rank reconstructs its own data) and the only collective is the
all-reduce (MAX) of the step time; the JSON value is all ranks' updates
over the slowest rank's time. The reference arm runs on rank 0 alone. These
tests run that logic as two processes on 127.0.0.1 with the gloo backend.
"""
import json
import os
import socket
import subprocess
import sys

import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", init_method=f"tcp://127.0.0.1:{port}", rank=rank, world_size=world)
    local_ms = [40.0, 55.0][rank]            # rank 1 is the slowest
    slowest = bench.max_over_ranks(local_ms, world, "cpu")
    value = bench.replica_value(6.657e10, world, slowest)
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump({"slowest": slowest, "value": value}, f)


def test_two_gloo_ranks_take_the_slowest_time(tmp_path):
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(world)]
    for r in res:
        assert r["slowest"] == 55.0                       # every rank sees the maximum
        assert abs(r["value"] - 2 * 6.657e10 / 0.055 / 1e9) < 1e-6


def test_single_rank_needs_no_collective():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(12.5, 1) == 12.5
    assert abs(bench.replica_value(1e9, 1, 1.0) - 1000.0) < 1e-9


def test_reference_arm_prints_on_rank_zero_only():
    """bench.py --impl reference under a non-zero RANK exits 0 without output
    (the other ranks of a torchrun launch do no work)."""
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "1"], capture_output=True, text=True, env=env, timeout=120)
    assert r.returncode == 0, r.stderr
    assert r.stdout.strip() == ""
