"""The N > 1 bench path on CPU with gloo (world size 2): every rank runs its own replica of the
transform ("replicas only": the apply has no exchange step on these single-GPU machines), rank 0
builds and saves the plan, the other ranks load it, and the timing is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, cache, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    class Args:
        workload = "sphere4096"
        plan_cache = cache

    plan, _, built = bench.get_plan(Args(), dist, rank)
    ex = plan.export()
    digest = float(np.sum(ex["transfer"][:1000])) + float(np.sum(ex["ranks"]))
    digests = [None] * world
    dist.all_gather_object(digests, (rank, built, digest, plan.info()["stored_entries"]))
    top = bench.max_over_ranks(1.0 + rank, dist)
    if rank == 0:
        np.save(out, np.array([[d[0], d[1], d[2], d[3]] for d in digests] + [[top, 0, 0, 0]], dtype=np.float64))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_share_one_plan_and_take_the_max_time(mht_lib, tmp_path):
    import torch.multiprocessing as mp
    cache = str(tmp_path / "plan.bin")
    out = str(tmp_path / "digests.npy")
    mp.spawn(_worker, args=(2, _free_port(), cache, out), nprocs=2, join=True)
    d = np.load(out)
    assert d[0, 1] == 1 and d[1, 1] == 0          # rank 0 built, rank 1 loaded
    assert d[0, 2] == d[1, 2] and d[0, 3] == d[1, 3]  # the same factors on both ranks
    assert d[2, 0] == 2.0                          # maximum over ranks


def test_bench_gpus_n_starts_n_replicas_itself(mht_lib):
    """`bench.py --gpus 2` without a launcher re-executes itself under torch.distributed.run:
    two ranks (world size 2, local ranks 0 and 1) report through gloo."""
    import json
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    env = {k: v for k, v in os.environ.items() if k not in ("RANK", "WORLD_SIZE", "LOCAL_RANK", "MASTER_PORT")}
    out = subprocess.run([sys.executable, os.path.join(root, "bench.py"), "--gpus", "2", "--workload", "ranks"],
                         capture_output=True, text=True, timeout=300, env=env, cwd=root)
    assert out.returncode == 0, out.stderr[-2000:]
    line = json.loads([x for x in out.stdout.splitlines() if x.startswith("{")][-1])
    assert sorted(tuple(r) for r in line["ranks"]) == [(0, 2, 0), (1, 2, 1)]
