"""One lattice split into y-slabs over CPU ranks (gloo): the per-step halo
exchange of ``slabs`` (3 populations x nx each way) with the FP64 oracle as
each rank's collision and streaming ends bitwise equal to the oracle on the
whole lattice.  World sizes 2 (both neighbours are the same rank) and 3
(uneven slabs), OReg and BGK."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

NX, NY, STEPS = 12, 10, 6


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _state(seed=7):
    """A non-uniform state: equilibria of random fields plus a random stress-
    carrying perturbation (so the OReg projection has work to do)."""
    from oracle import oracle as O
    rng = np.random.default_rng(seed)
    p = O.params(NX, NY, 0.7)
    rho = 1.0 + 0.05 * rng.standard_normal((NY, NX))
    ux, uy = 0.03 * rng.standard_normal((2, NY, NX))
    f = O.init_equilibrium(p, rho, ux, uy)
    return f + 1e-3 * rng.standard_normal(f.shape)


def _worker(rank, world, port, coll, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O
        from paper_2501_16000_gb300 import slabs
        c = O.OREG if coll == "oreg" else O.BGK
        y0, y1 = slabs.slab_rows(NY, world, rank)
        f = _state()[:, y0:y1, :].copy()

        def collide_slab(s):
            post = np.empty_like(s)
            for y in range(s.shape[1]):
                for x in range(s.shape[2]):
                    post[:, y, x] = O.collide(s[:, y, x], 0.7, coll=c)
            return post

        for _ in range(STEPS):
            f = slabs.step(f, collide_slab, O.stream)
        out[rank] = (y0, y1, f)
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("coll", ["oreg", "bgk"])
@pytest.mark.parametrize("world", [2, 3])
def test_slabs_equal_the_whole_lattice_bitwise(world, coll):
    pytest.importorskip("torch.distributed")
    from oracle import oracle as O
    mgr = mp.Manager()
    out = mgr.dict()
    mp.start_processes(_worker, args=(world, _free_port(), coll, out), nprocs=world, join=True,
                       start_method="spawn")
    p = O.params(NX, NY, 0.7, coll=O.OREG if coll == "oreg" else O.BGK)
    want = O.run(_state(), p, STEPS)
    got = np.empty_like(want)
    rows = []
    for r in range(world):
        y0, y1, f = out[r]
        got[:, y0:y1, :] = f
        rows.append((y0, y1))
    assert rows[0][0] == 0 and rows[-1][1] == NY
    assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
    assert np.array_equal(got, want)


def test_slab_plan():
    """Row partition and halo directions: the up/down sets are the c_y = +1 /
    -1 directions, slabs tile the rows with heights differing by at most one,
    and a single slab exchanges with itself (the periodic lattice)."""
    from paper_2501_16000_gb300 import slabs
    assert slabs.UP == (2, 5, 6) and slabs.DOWN == (4, 7, 8)
    for ny in (1, 5, 10, 17):
        for world in range(1, min(ny, 6) + 1):
            parts = [slabs.slab_rows(ny, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == ny
            h = [b - a for a, b in parts]
            assert max(h) - min(h) <= 1 and min(h) >= 1
    with pytest.raises(ValueError):
        slabs.slab_rows(3, 4, 0)
    post = np.arange(9 * 4 * 5, dtype=float).reshape(9, 4, 5)
    up, down = slabs.pack_halos(post)
    ext = slabs.extend(post, up, down)
    assert ext.shape == (9, 6, 5)
    assert np.array_equal(ext[[2, 5, 6], 0], post[[2, 5, 6], -1])
    assert np.array_equal(ext[[4, 7, 8], -1], post[[4, 7, 8], 0])
    assert not ext[[0, 1, 3, 4, 7, 8], 0].any() and not ext[[0, 1, 2, 3, 5, 6], -1].any()
