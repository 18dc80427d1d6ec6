"""Multi-GPU runs are independent replicas (one instance, batch or request
stream per rank, no collective on the data path); the only cross-rank steps
are the host-side barrier and the max / sum reductions of bench.py's timing.
These run here as two gloo ranks on the CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, ws, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist

    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench

    bench.barrier(ws)
    # per-rank wall times and unit counts: the job time is the slowest rank,
    # the job's units are every rank's
    t = bench.max_over_ranks(1.5 + rank, ws)
    u = bench.sum_over_ranks(100.0 * (rank + 1), ws)
    # every rank draws its own instance (seed offset by rank)
    wl = dict(bench.WORKLOADS["vc-er-n2000-m8000"])
    g = bench.make_graph(wl, rank)
    out[rank] = (t, u, int(g.eu[:50].sum()))
    dist.destroy_process_group()


def test_two_replicas_timing_reductions():
    ws = 2
    mgr = mp.get_context("spawn").Manager()
    out = mgr.dict()
    port = _free_port()
    mp.start_processes(_rank, args=(ws, port, out), nprocs=ws, start_method="spawn", join=True)
    assert out[0][:2] == out[1][:2] == (2.5, 300.0)
    assert out[0][2] != out[1][2], "replicas must solve different instances"


def test_dist_setup_single_process_needs_no_group():
    import bench

    class A:
        impl = "thetis"

    os.environ.pop("WORLD_SIZE", None)
    ws, rank, local = bench.dist_setup(A())
    assert (ws, rank, local) == (1, 0, 0)
    assert bench.max_over_ranks(3.0, 1) == 3.0 and bench.sum_over_ranks(3.0, 1) == 3.0
