"""Multi-GPU layout is replicas only: each rank runs its own copy of the
workload and bench.py reports all ranks' cell updates over the slowest rank's
time.  The reduction runs here on CPU ranks (gloo, world size 2)."""
import json
import os
import socket
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ms_local = 10.0 + 5.0 * rank  # rank 1 is the slow one
    ms, mlups = bench.replica_mlups(ms_local, cells=1000, steps=50, world=world, device="cpu")
    with open(os.path.join(out_dir, f"r{rank}.json"), "w") as fh:
        json.dump({"ms": ms, "mlups": mlups}, fh)
    dist.destroy_process_group()


def test_replica_aggregate_gloo(tmp_path):
    torch = pytest.importorskip("torch")
    import torch.multiprocessing as mp
    world = 2
    mp.spawn(_rank, args=(world, _free_port(), str(tmp_path)), nprocs=world, join=True)
    res = [json.load(open(tmp_path / f"r{r}.json")) for r in range(world)]
    for r in res:
        assert r["ms"] == 15.0  # max over ranks
        assert abs(r["mlups"] - world * 1000 * 50 / 15e-3 / 1e6) < 1e-9
