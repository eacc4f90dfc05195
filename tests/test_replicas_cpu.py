"""The multi-GPU path of the benchmark is replicas (each rank reconstructs
its own batch, no collective on the data path); its host logic -- the
slowest rank's time, distinct per-rank inputs, rank-0-only reference arm --
runs here as two gloo ranks on the CPU."""
import os
import socket
import sys

import numpy as np
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
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    slowest = bench.reduce_max(1.5 + rank, dist, "cpu")
    y, lam = bench.make_inputs(1, rank)
    args = type("A", (), dict(steps=1, warmup=1, oracle_iters=10, sigma=0.13, rho=0.95))()
    ref = bench.run_reference(args, rank, world) if rank != 0 else "rank0"
    np.savez(os.path.join(out_dir, "r%d.npz" % rank), slowest=slowest, y=y[0, :4, :16],
             ref_none=ref is None)
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    port = _free_port()
    mp.start_processes(_rank_main, args=(2, port, str(tmp_path)), nprocs=2, start_method="spawn", join=True)
    r0 = np.load(tmp_path / "r0.npz")
    r1 = np.load(tmp_path / "r1.npz")
    # every rank reports the slowest rank's time
    assert float(r0["slowest"]) == 2.5 and float(r1["slowest"]) == 2.5
    # replicas reconstruct different scans
    assert not np.array_equal(r0["y"], r1["y"])
    # the reference arm runs on rank 0 only
    assert bool(r1["ref_none"])


def test_reduce_max_without_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_max(3.0, None, "cpu") == 3.0

