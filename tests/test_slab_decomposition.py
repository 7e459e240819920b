"""Domain decomposition of the step into y-slabs, on the CPU with `gloo` ranks.

Each rank owns a band of rows of a y-periodic problem and steps it on its
band plus two halo rows on each side, through the package's slab module
(paper_1810_07802_gb300.slab: Band, DistExchange), with the FP64 oracle as
the band stepper in place of the GPU solver.  What one step of a cell reads
determines the halo: the update of row j needs psi-bar-plus of rows
j-1 .. j+1 (face reconstruction, Eq. 27), and psi-bar-plus of row j-1 needs
phi (all of f) on rows j-2 .. j (the gradient and Laplacian stencils), with g
and (phi u)^{n-1} on row j-1 itself.  So before every step each rank receives
from its neighbours their two edge rows; rows farther out never reach its own
rows.  The exchange is a pair of point-to-point send/receives per neighbour
(no collective).  The bands' rows, gathered after the steps, must equal the
single-domain oracle bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

from paper_1810_07802_gb300 import slab  # noqa: E402

HALO = slab.HALO


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


class OracleBand:
    """The FP64 oracle on a band's problem, with the stepper interface of
    slab.Band (rows of the stored planes f, g and (phi u)^{n-1} in and out of
    [20][nrows][nx] CPU tensors)."""

    def __init__(self, cfg, fields):
        from oracle.oracle import Oracle

        self.o = Oracle(cfg, **fields)
        self.nx = cfg["nx"]
        self.n = 0

    def row_buffer(self, nrows):
        import torch

        return torch.empty((20, nrows, self.nx), dtype=torch.float64)

    def get_rows(self, row0, nrows, buf):
        import torch

        f, g, h = self.o.state()
        buf.copy_(torch.from_numpy(np.concatenate([f, g, h])[:, row0:row0 + nrows]))

    def set_rows(self, row0, nrows, buf):
        f, g, h = self.o.state()
        a = buf.numpy()
        f[:, row0:row0 + nrows], g[:, row0:row0 + nrows], h[:, row0:row0 + nrows] = a[:9], a[9:18], a[18:]
        self.o.set_state(f, g, h, self.n)

    def step(self, n):
        self.o.step(n)
        self.n += n


def _problem():
    from paper_1810_07802_gb300 import workloads as W

    return W.random_state(21, 26, seed=13, rho_ratio=100.0)


def _rank_main(rank, world, port, steps, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg, fl = _problem()
        r0, r1 = slab.bands(cfg["ny"], world)[rank]
        band = slab.Band(OracleBand(*slab.band_problem(cfg, fl, r0, r1)), r0, r1)
        slab.step_bands(slab.DistExchange(band, rank, world), [band], steps)
        f, g, h = band.stepper.o.state()
        own = slice(HALO, HALO + band.n_own)
        q.put((rank, r0, r1, f[:, own].copy(), g[:, own].copy(), h[:, own].copy()))
    finally:
        dist.destroy_process_group()


def _single_domain(steps):
    from oracle.oracle import Oracle

    cfg, fl = _problem()
    ref = Oracle(cfg, **fl)
    ref.step(steps)
    return cfg, ref.state()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_with_halo_exchange_equal_the_single_domain(world):
    import torch.multiprocessing as mp

    steps = 7
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    cfg, (F, G, H) = _single_domain(steps)
    covered = np.zeros(cfg["ny"], dtype=int)
    for rank, r0, r1, f, g, h in parts:
        assert np.array_equal(f, F[:, r0:r1]), rank
        assert np.array_equal(g, G[:, r0:r1]), rank
        assert np.array_equal(h, H[:, r0:r1]), rank
        covered[r0:r1] += 1
    assert (covered == 1).all()


def test_local_exchange_of_three_bands():
    """The in-process exchange (the one the GPU test uses) with oracle bands:
    three bands equal the single-domain oracle bit for bit."""
    steps = 5
    cfg, fl = _problem()
    band_list = [slab.Band(OracleBand(*slab.band_problem(cfg, fl, r0, r1)), r0, r1)
                 for r0, r1 in slab.bands(cfg["ny"], 3)]
    slab.step_bands(slab.LocalExchange(band_list), band_list, steps)
    _, (F, G, H) = _single_domain(steps)
    for b in band_list:
        f, g, h = b.stepper.o.state()
        own = slice(HALO, HALO + b.n_own)
        assert np.array_equal(f[:, own], F[:, b.r0:b.r1])
        assert np.array_equal(g[:, own], G[:, b.r0:b.r1])
        assert np.array_equal(h[:, own], H[:, b.r0:b.r1])


def test_one_halo_row_fewer_breaks_the_equality():
    """The halo is no wider than needed: with only one row of f received
    below, the band's first row differs from the single-domain result."""
    from oracle.oracle import Oracle

    cfg, fl = _problem()
    ny = cfg["ny"]
    full = Oracle(cfg, **fl)
    F, G, H = full.state()
    r0, r1 = 0, 13
    idx = np.arange(r0 - HALO, r1 + HALO) % ny
    f, g, h = F[:, idx, :].copy(), G[:, idx, :].copy(), H[:, idx, :].copy()
    f[:, 0, :] = 0.0                       # the second f row below is not sent
    band = Oracle(dict(cfg, ny=r1 - r0 + 2 * HALO), **{k: (None if v is None else v[idx, :]) for k, v in fl.items()})
    band.set_state(f, g, h, 0)
    band.step(1)
    full.step(1)
    got = band.state()[0][:, HALO]
    assert not np.array_equal(got, full.state()[0][:, r0])


def test_bands_rejects_thin_bands_and_walls():
    with pytest.raises(ValueError):
        slab.bands(5, 3)
    cfg, fl = _problem()
    with pytest.raises(ValueError):
        slab.band_problem(dict(cfg, bc_y="wall"), fl, 0, 10)
