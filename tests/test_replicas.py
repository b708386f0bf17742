"""The multi-GPU form is replicas only (each rank an independent simulation,
no collective on the data path): the bench's whole-job figures take the
slowest rank's time and the sum of all ranks' units.  Checked with two gloo
ranks on the CPU."""
import os
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _rank(rank, ws, port, out):
    import torch
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    torch.distributed.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    sec = [0.5, 0.8][rank]
    units = [1e9, 3e9][rank]
    esec = [1.0, 0.9][rank]
    eu = [2e9, 5e9][rank]
    out[rank] = bench.combine_ranks(sec, units, esec, eu, "cpu")
    torch.distributed.barrier()
    torch.distributed.destroy_process_group()


def test_two_gloo_ranks_combine_to_whole_job_figures():
    ctx = mp.get_context("spawn")
    with ctx.Manager() as m:
        out = m.dict()
        port = 29500 + (os.getpid() % 1000)
        ps = [ctx.Process(target=_rank, args=(r, 2, port, out)) for r in range(2)]
        for p in ps:
            p.start()
        for p in ps:
            p.join(120)
        assert all(p.exitcode == 0 for p in ps)
        for r in range(2):
            assert out[r] == pytest.approx((0.8, 4e9, 1.0, 7e9))
