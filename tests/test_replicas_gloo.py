"""The multi-GPU form is replicas only (one independent field per rank, no
data-path collective).  Its host logic runs here on CPU with two `gloo`
ranks: every rank gets its own seeded field, and the job's step time is the
slowest rank's, the job's value the cells of all ranks over that time."""
import os
import socket
import sys

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank(rank, ws, port, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        w, r, _ = bench._dist()
        ms = bench.slowest_rank_ms(10.0 + 5.0 * r, w)           # rank 1 is the slow one
        rho = bench.workload_density(8, r)
        digest = torch.tensor([float(np.float64(rho).sum())], dtype=torch.float64)
        gathered = [torch.zeros(1, dtype=torch.float64) for _ in range(w)]
        dist.all_gather(gathered, digest)
        out[r] = (ms, bench.whole_job_cells_per_s(w, 8, ms), [float(g) for g in gathered])
    finally:
        dist.destroy_process_group()


def test_two_replicas_time_as_the_slowest_and_solve_distinct_fields():
    ws = 2
    port = _free_port()
    with mp.get_context("spawn").Manager() as mgr:       # no fork of a threaded process
        out = mgr.dict()
        mp.spawn(_rank, args=(ws, port, out), nprocs=ws, join=True)
        res = dict(out)
    for r in range(ws):
        ms, value, digests = res[r]
        assert ms == pytest.approx(15.0)
        assert value == pytest.approx(ws * 8 ** 3 / 0.015)
        assert digests[0] != digests[1]             # one independent field per rank


def test_single_process_is_unchanged():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.slowest_rank_ms(12.5, 1) == 12.5
    assert bench.whole_job_cells_per_s(1, 256, 50.0) == pytest.approx(256 ** 3 / 0.05)

