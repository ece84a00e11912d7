"""Multi-process host logic on CPU (gloo, world size 2).

1. The benchmark's timing rule: every rank times its own replica and rank 0
   reports the maximum over ranks.
2. Sharding the path over ranks: histories are independent, so each rank can
   accumulate N and M over its share and an all-reduce sum gives exactly the
   whole scan's counts (and from them the same decisions).  Checked with the
   oracle on each rank's shard.
"""
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_1402_1720_gb300 import synth


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import oracle
    # 1. max over ranks of per-rank step times
    t = torch.tensor([1.5 + rank], dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    # 2. sharded accumulation
    w = synth.make_config(1, fraction=0.2)
    g, h = w.geometry, w.histories
    share = h.take(np.arange(rank, len(h), world))
    acc = oracle.accumulate(g, share)
    N = torch.from_numpy(acc["N"].astype(np.int64))
    M = torch.from_numpy(acc["M"].astype(np.int64))
    dist.all_reduce(N, op=dist.ReduceOp.SUM)
    dist.all_reduce(M, op=dist.ReduceOp.SUM)
    if rank == 0:
        np.save(os.path.join(out_dir, "N.npy"), N.numpy())
        np.save(os.path.join(out_dir, "M.npy"), M.numpy())
        np.save(os.path.join(out_dir, "tmax.npy"), t.numpy())
    dist.destroy_process_group()


def test_two_rank_sharding_and_timing(tmp_path, oracle_mod):
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    assert float(np.load(tmp_path / "tmax.npy")[0]) == 2.5
    w = synth.make_config(1, fraction=0.2)
    whole = oracle_mod.run(w.geometry, w.histories)
    N = np.load(tmp_path / "N.npy").astype(np.uint32)
    M = np.load(tmp_path / "M.npy").astype(np.uint32)
    assert np.array_equal(N, whole["N"]) and np.array_equal(M, whole["M"])
    dims = (w.geometry.nx, w.geometry.ny, w.geometry.nz)
    assert np.array_equal(oracle_mod.msc_decide(N, dims), whole["H2"])
    assert np.array_equal(oracle_mod.sm_decide(M, dims)["H3"], whole["H3"])
