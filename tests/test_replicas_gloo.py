"""Multi-GPU path on the CPU (gloo, world size 2): the run is replicas only.
Each rank runs its own simulation (own seed); ranks exchange nothing but a
barrier and the max-over-ranks time, and the reported value is the units all
ranks processed over that time.  The reference arm prints its line on rank 0
only; the other ranks exit 0 without work.
"""
import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    import bench
    import workloads
    w, r, _ = bench.dist_env()
    dist = bench.init_dist(w, "gloo")
    bench.barrier(dist)
    t = bench.reduce_max(1.5 + r, dist)               # rank 1 is the slowest
    run = bench.replica_run(workloads.BIG_NDGP, r, 23)
    with open(os.path.join(out_dir, f"rank{r}.json"), "w") as f:
        json.dump({"max_t": t, "seed": run.seed, "Np": run.Np, "nsteps": run.nsteps,
                   "value": bench.whole_job_throughput(100.0, w, t)}, f)
    bench.barrier(dist)
    dist.destroy_process_group()


def test_two_gloo_ranks_share_only_the_timer(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    res = [json.load(open(tmp_path / f"rank{r}.json")) for r in range(2)]
    assert res[0]["max_t"] == res[1]["max_t"] == 2.5
    assert res[0]["value"] == res[1]["value"] == pytest.approx(100.0 * 2 / 2.5)
    assert res[0]["seed"] != res[1]["seed"]            # independent replicas
    assert res[0]["Np"] == res[1]["Np"] and res[0]["nsteps"] == res[1]["nsteps"] == 30


def test_reference_arm_under_torchrun_prints_one_line():
    port = _free_port()
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(port), "bench.py", "--impl", "reference",
           "--workload", "small", "--steps", "1", "--warmup", "0"]
    p = subprocess.run(cmd, cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [json.loads(l) for l in p.stdout.splitlines() if l.startswith("{")]
    assert len(lines) == 1 and lines[0]["impl"] == "reference"
    assert lines[0]["n_gpus"] == 2 and lines[0]["value"] > 0 and lines[0]["cpu_baseline"]["kind"] == "oracle"
