"""The multi-GPU path of the benchmark is replicas with no collective on the data path:
each rank steps its own cases; ranks meet only to take the job's time (the maximum over
ranks) and the units processed (the sum).  These host-side pieces run here as two gloo
ranks on the CPU."""
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

from conftest import ROOT


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    from synth import cases
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t = bench.max_over_ranks([1.0 + rank, 10.0 - rank], dist)
        bc = cases.batch_cases(seed=bench.batch_seed(rank), n=64)
        cells = sum(c["nx"] * c["nr"] for c, _ in bc)
        total = bench.total_over_ranks(cells, dist)
        out.put((rank, t, cells, total, [c["T_amb"] for c, _ in bc[:4]]))
    finally:
        dist.destroy_process_group()


def test_two_ranks_time_is_max_and_units_are_summed():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    (r0, t0, c0, tot0, amb0), (r1, t1, c1, tot1, amb1) = res
    assert t0 == t1 == [2.0, 10.0]                   # max over ranks, the same on every rank
    assert tot0 == tot1 == c0 + c1                   # whole-job units
    assert amb0 != amb1                              # each rank steps its own cases


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks([1.5, 2.5], None) == [1.5, 2.5]
    assert bench.total_over_ranks(7, None) == 7
    assert bench.batch_seed(0) != bench.batch_seed(1)
