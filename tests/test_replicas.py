"""Replica sharding across ranks: host logic on CPU with gloo, world size 2."""
import os
import socket

import numpy as np
import pytest

from paper_2303_02724_gb300 import fields as F
from paper_2303_02724_gb300 import replicas


def test_shard_complete_disjoint_balanced():
    sizes = [int(np.prod(e)) for (e, _, _) in F.batch_specs(3, 256)]
    for world in (1, 2, 4, 8):
        parts = replicas.shard(sizes, world)
        flat = sorted(i for p in parts for i in p)
        assert flat == list(range(len(sizes)))
        loads = [sum(sizes[i] for i in p) for p in parts]
        assert max(loads) <= max(sizes) + sum(sizes) / world  # LPT bound
        assert replicas.shard(sizes, world) == parts  # deterministic


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        specs = F.batch_specs(3, 64, scale=0.05)
        sizes = [int(np.prod(e)) for (e, _, _) in specs]
        mine = replicas.my_share(sizes, rank, world)
        # every rank "processes" its own fields (no data exchange) and reports
        verts = sum(sizes[i] for i in mine)
        t = 1.0 + rank  # per-rank step time
        tmax = replicas.reduce_max(t)
        vsum = replicas.reduce_sum(verts)
        got = [None] * world
        dist.all_gather_object(got, mine)
        with open(os.path.join(out_dir, f"rank{rank}.txt"), "w") as f:
            f.write(f"{tmax} {vsum} {sum(sizes)} {sorted(i for g in got for i in g) == list(range(len(sizes)))}")
    finally:
        dist.destroy_process_group()


def test_two_ranks_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn")
    for r in range(2):
        tmax, vsum, total, complete = open(tmp_path / f"rank{r}.txt").read().split()
        assert float(tmax) == 2.0          # the max over ranks
        assert float(vsum) == float(total)  # the shards cover the batch once
        assert complete == "True"
