"""The multi-replica bench path on CPU: two gloo ranks (world size 2) run
bench.replica_totals, the only cross-rank step of `bench.py --gpus N` (each
rank solves an independent replica; there is no collective in the data
path): the whole-job units are the sum over ranks and the time is the
slowest rank's."""
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


def _rank(rank, world, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ws, r, local = bench._dist()
    units, ms = bench.replica_totals(dist, units=1000 * (rank + 1), ms=10.0 + 5.0 * rank, device="cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out, f"rank{rank}.json"), "w") as f:
        json.dump({"units": units, "ms": ms, "ws": ws, "rank": r, "local": local}, f)


def test_two_gloo_replicas(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        d = json.load(open(tmp_path / f"rank{rank}.json"))
        assert d["units"] == 3000.0 and d["ms"] == 15.0
        assert d["ws"] == 2 and d["rank"] == rank and d["local"] == rank


def test_single_process_totals_are_local():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.replica_totals(None, 7, 2.5, "cpu") == (7.0, 2.5)
