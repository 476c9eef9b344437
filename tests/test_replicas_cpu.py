"""The N > 1 host path of bench.py on CPU (gloo, world size 2).

On several GPUs every rank runs an independent replica of the workload (the
power does not shard without a per-level exchange): the ranks meet at a
barrier around the timed region, the slowest rank's time sets the
throughput (max over ranks), and rank 0 alone prints the JSON line.  These
tests run that logic as two CPU processes."""
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
    import argparse
    os.environ.update(WORLD_SIZE=str(world), RANK=str(rank), LOCAL_RANK=str(rank),
                      MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    import torch.distributed as dist
    w, r, local = bench.dist_setup(argparse.Namespace(impl="reference"))
    assert (w, r, local) == (world, rank, rank)
    assert dist.get_backend() == "gloo"
    bench.barrier(w)
    # each rank's time; the job's time is the slowest rank's
    got = bench.max_over_ranks(w, 10.0 + 3.0 * rank, "cpu")
    bench.barrier(w)
    dist.destroy_process_group()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"max": got}, f)


def test_barrier_and_max_over_ranks_gloo(tmp_path):
    import torch.multiprocessing as mp
    world, port = 2, _free_port()
    mp.start_processes(_rank_main, args=(world, port, str(tmp_path)), nprocs=world, join=True,
                       start_method="spawn")
    for r in range(world):
        with open(tmp_path / ("rank%d.json" % r)) as f:
            assert json.load(f)["max"] == 13.0


def test_max_over_ranks_is_identity_alone():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(1, 4.25) == 4.25


def test_reference_arm_under_torchrun_prints_once():
    # `bench.py --impl reference` launched as two ranks: rank 0 times the
    # oracle on a bounded sample and prints one line; rank 1 exits 0 without work
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), os.path.join(ROOT, "bench.py"),
           "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "3", "--ref-budget", "0.2",
           "--workload", "stoch64"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=240, env=env)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [l for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1, p.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2
    assert line["value"] > 0 and line["cpu_baseline"]["kind"] == "oracle"
    assert line["config"]["parallelism"] == "replicas"
