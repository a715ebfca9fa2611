"""The N > 1 path of the benchmark on CPU ranks (gloo, world size 2): the
replica harness's collectives (barrier, maximum over ranks), the whole-job
aggregate, and the reference arm under torchrun (rank 0 alone runs the
oracle and prints one line; the other rank exits 0 without work).  The
step path itself shards into independent replicas and has no collective."""
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
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)
    r = bench.Ranks(dist, "cpu")
    r.barrier()
    elapsed = 0.25 * (rank + 1)          # rank 1 is the slow one
    slowest = r.max(elapsed)
    rate = bench.whole_job_rate(r.world, 1000.0, slowest)
    r.barrier()
    with open(os.path.join(out_dir, "rank%d.json" % rank), "w") as f:
        json.dump({"rank": r.rank, "world": r.world, "slowest": slowest, "rate": rate}, f)
    dist.destroy_process_group()


def test_replica_collectives_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / ("rank%d.json" % k))) for k in range(2)]
    for k, r in enumerate(res):
        assert r["rank"] == k and r["world"] == 2
        assert r["slowest"] == 0.5            # the maximum, on every rank
        assert r["rate"] == 2 * 1000.0 / 0.5  # all ranks' units over the slowest rank's time


def test_single_process_ranks_are_trivial():
    sys.path.insert(0, ROOT)
    import bench
    r = bench.Ranks()
    r.barrier()
    assert (r.world, r.rank, r.max(3.5)) == (1, 0, 3.5)
    assert bench.whole_job_rate(1, 10.0, 2.0) == 5.0


def test_reference_arm_under_torchrun_two_ranks(tmp_path):
    env = dict(os.environ, OMP_NUM_THREADS="2")
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node=2",
           "--master-addr=127.0.0.1", "--master-port=%d" % _free_port(), "--log-dir", str(tmp_path / "logs"),
           "--redirects", "3", os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2",
           "--steps", "1", "--warmup", "0", "--side", "64"]
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    outs = {}
    for root, _, files in os.walk(tmp_path / "logs"):
        for fn in files:
            if fn == "stdout.log":
                rank = int(os.path.basename(root))
                outs[rank] = open(os.path.join(root, fn)).read().strip().splitlines()
    assert sorted(outs) == [0, 1]
    assert outs[1] == []                      # the other rank does no work and prints nothing
    assert len(outs[0]) == 1
    line = json.loads(outs[0][0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle"
