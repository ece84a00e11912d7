"""Sharding a scan over ranks through the library (gloo, world size 2).

Histories are independent and N, M are sums over them (Eq. 3.4, 3.9), so a
scan can be split: each rank runs the library on its share (here both ranks
share the one GPU; their kernels never wait on one another), the counts are
summed over ranks with an all-reduce on the host, each rank loads the sums
into its scan (hd_scan_set_counts) and finalizes.  Every rank must then hold
the hulls and thresholds of the whole scan as the oracle computes them.
"""
import os
import socket

import numpy as np
import pytest

from paper_1402_1720_gb300 import synth

torch = pytest.importorskip("torch")
pytestmark = pytest.mark.gpu

if not torch.cuda.is_available():  # pragma: no cover - CPU container
    pytest.skip("needs a CUDA GPU", allow_module_level=True)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    from paper_1402_1720_gb300 import hulld
    hulld.load()
    torch.cuda.set_device(0)
    w = synth.make_config(1)
    g, h = w.geometry, w.histories
    share = h.take(np.arange(rank, len(h), world))
    with hulld.Scan(g) as s:
        s.add([torch.from_numpy(a).cuda() for a in share.arrays()])
        torch.cuda.synchronize()
        local = s.stats()
        N = torch.from_numpy(s.counts(hulld.HD_MSC).astype(np.int64))
        M = torch.from_numpy(s.counts(hulld.HD_SM).astype(np.int64))
        dist.all_reduce(N, op=dist.ReduceOp.SUM)
        dist.all_reduce(M, op=dist.ReduceOp.SUM)
        hulld.hd_scan_set_counts(s.handle, hulld.HD_MSC, N.numpy().astype(np.uint32))
        hulld.hd_scan_set_counts(s.handle, hulld.HD_SM, M.numpy().astype(np.uint32))
        s.finalize()
        torch.cuda.synchronize()
        mt, slope, index = s.thresholds()
        out = {"N": s.counts(hulld.HD_MSC), "M": s.counts(hulld.HD_SM),
               "H1": s.mask(hulld.HD_SC), "H2": s.mask(hulld.HD_MSC), "H3": s.mask(hulld.HD_SM),
               "Mt": mt, "index": index}
        st = s.stats()
    n_in = torch.tensor([local["n_in"]], dtype=torch.int64)
    dist.all_reduce(n_in, op=dist.ReduceOp.SUM)
    np.savez(os.path.join(out_dir, f"rank{rank}.npz"), n_in=n_in.numpy(),
             steps=np.array([st["steps_miss"], st["steps_hit"]]), **out)
    dist.destroy_process_group()


def test_two_rank_library_shards_equal_whole_scan(tmp_path, oracle_mod):
    import torch.multiprocessing as mp
    world = 2
    mp.start_processes(_worker, args=(world, _free_port(), str(tmp_path)), nprocs=world,
                       join=True, start_method="spawn")
    w = synth.make_config(1)
    ref = oracle_mod.run(w.geometry, w.histories, threads=8)
    for r in range(world):
        got = np.load(tmp_path / f"rank{r}.npz")
        assert int(got["n_in"][0]) == len(w.histories)
        assert int(got["steps"][0]) == ref["stats"]["steps_miss"]
        assert int(got["steps"][1]) == ref["stats"]["steps_hit"]
        for k in ("N", "M", "H1", "H2", "H3", "Mt", "index"):
            assert np.array_equal(got[k], ref[k]), (r, k)
