"""The N > 1 path of bench.py on CPU with two gloo ranks: each rank anneals its own
replica set (replicas only: different seeds, no data exchange), and the job's time
is the slowest rank's time."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    import bench
    import oracle
    from paper_1806_08815_gb300 import instances
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    q = instances.sk_bimodal(24, 1)
    beta = instances.beta_linear(0.1, 3.0, 300)
    r = oracle.da_anneal(q.Q, beta, R=4, seed=bench.rank_seed(rank), inc=0.0)
    t = bench.max_over_ranks(0.5 + rank, dist, "cpu")
    out[rank] = (bench.rank_seed(rank), t, r["x_best"].tobytes())
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_replicas_only():
    import torch.multiprocessing as mp
    import oracle
    oracle.build()
    world = 2
    port = _free_port()
    with mp.Manager() as mgr:
        out = mgr.dict()
        mp.spawn(_rank_main, args=(world, port, out), nprocs=world, join=True)
        res = dict(out)
    seeds = {res[r][0] for r in range(world)}
    assert len(seeds) == world
    assert all(res[r][1] == 1.5 for r in range(world))       # max over ranks of 0.5 and 1.5
    assert res[0][2] != res[1][2]                              # independent replica sets


def test_bench_spawns_its_ranks_for_gpus_n():
    """`bench.py --gpus 2` without a launcher starts two ranks itself (torch.distributed.run);
    with the reference arm, rank 0 alone runs and prints one line that names 2 GPUs."""
    import json
    import subprocess
    import sys
    import oracle
    oracle.build()
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("WORLD_SIZE", "RANK", "LOCAL_RANK")}
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--impl", "reference", "--gpus", "2",
                        "--steps", "1", "--warmup", "0"], capture_output=True, text=True, env=env, timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [ln for ln in r.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, r.stdout
    line = json.loads(lines[0])
    assert line["impl"] == "reference" and line["n_gpus"] == 2 and line["value"] > 0
