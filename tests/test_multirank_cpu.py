"""The benchmark's multi-rank path on CPU ranks (gloo, world size 2): every
rank advances an independent lattice (here the FP64 oracle stands in for the
GPU), the timing is the maximum over ranks, and whole-job throughput scales
with the number of ranks (weak scaling, no data-path collective)."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        import bench
        from oracle import oracle as O
        from paper_2501_16000_gb300 import workloads as W
        # each rank: its own independent lattice, no exchange of populations
        case = W.LatticeCase(nx=24, ny=16, tau=0.7, case="shear", u0=0.05, m=1 + rank, n=1)
        p = O.params(case.nx, case.ny, case.tau)
        f = O.run(O.init_equilibrium(p, *case.fields()), p, 10)
        mass = float(f.sum())
        elapsed = 100.0 + 50.0 * rank            # per-rank "times"
        out[rank] = (bench.max_over_ranks(elapsed), mass,
                     bench.weak_scaling_mlups(world, case.nodes, 10, bench.max_over_ranks(elapsed)))
    finally:
        dist.destroy_process_group()


def test_two_ranks_max_timing_and_weak_scaling():
    pytest.importorskip("torch.distributed")
    world = 2
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True,
                       start_method="spawn")
    assert out[0][0] == out[1][0] == 150.0               # the slowest rank sets the time
    assert abs(out[0][1] - 24 * 16) < 1e-9 and abs(out[1][1] - 24 * 16) < 1e-9
    assert np.isclose(out[0][2], 2 * 24 * 16 * 10 / 0.150 / 1e6)


def test_single_process_is_identity():
    import bench
    assert bench.max_over_ranks(3.5) == 3.5
    assert np.isclose(bench.weak_scaling_mlups(1, 1000, 10, 1.0), 10.0)
