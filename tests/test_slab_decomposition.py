"""Domain decomposition of the step into y-slabs, on the CPU with `gloo` ranks.

Each rank owns a band of rows and steps it on its band plus halo rows on each
side that has a neighbour, through the package's slab module
(paper_1810_07802_gb300.slab: Band, DistExchange, LocalExchange), with the
FP64 oracle as the band stepper in place of the GPU solver.  What one step of
a cell reads determines the halo: the update of row j needs psi-bar-plus of
rows j-1 .. j+1 (face reconstruction, Eq. 27), and psi-bar-plus of row j-1
needs phi (all of f) on rows j-2 .. j (the gradient and Laplacian stencils),
with g and (phi u)^{n-1} on row j-1 itself: two rows.  The upwind face reads
the profile of the cell a direction leaves, one row further: three rows.
Periodic problems are cut into periodic bands; problems with no-slip walls
into walled bands whose inner walls touch only their outermost halo row.
The exchange is a pair of point-to-point send/receives per neighbour (no
collective).  The bands' rows, gathered after the steps, must equal the
single-domain oracle bit for bit, and their combined reductions the oracle's.
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

    def reduce_rows(self, row0, nrows):
        """The sums behind the oracle's reduction over rows [row0, row0 + nrows),
        against the whole grid kept at the previous call (numpy, FP64)."""
        m = self.o.macros()
        phi, ux, uy = m["phi"], m["ux"], m["uy"]
        rows = slice(row0, row0 + nrows)
        u2 = ux[rows] ** 2 + uy[rows] ** 2
        sums = np.array([phi[rows].sum(), (phi[rows] ** 2).sum(), 0.0, u2.sum(), 0.0, np.sqrt(u2).max()])
        had = getattr(self, "_snap", None) is not None
        if had:
            p0, a0, b0 = self._snap
            sums[2] = ((phi[rows] - p0[rows]) ** 2).sum()
            sums[4] = ((ux[rows] - a0[rows]) ** 2 + (uy[rows] - b0[rows]) ** 2).sum()
        self._snap = (phi.copy(), ux.copy(), uy.copy())
        return sums, had


KINDS = ("periodic", "wall", "upwind", "wall_upwind")


def _problem(kind="periodic"):
    """A rough coupled state, periodic or walled in y, with the central or
    the upwind reconstruction."""
    from paper_1810_07802_gb300 import workloads as W

    cfg, fl = W.random_state(21, 26, seed=13, rho_ratio=100.0, bc_y="wall" if "wall" in kind else "periodic")
    if "upwind" in kind:
        cfg = dict(cfg, recon="upwind")
    return cfg, fl


def _band_list(cfg, fl, world, halo=None):
    h = slab.halo_rows(cfg) if halo is None else halo
    return [slab.Band(OracleBand(*slab.band_problem(cfg, fl, r0, r1, halo)), r0, r1, cfg, halo)
            for r0, r1 in slab.bands(cfg["ny"], world, h)]


def _rank_main(rank, world, port, steps, kind, q):
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg, fl = _problem(kind)
        r0, r1 = slab.bands(cfg["ny"], world, slab.halo_rows(cfg))[rank]
        band = slab.Band(OracleBand(*slab.band_problem(cfg, fl, r0, r1)), r0, r1, cfg)
        ex = slab.DistExchange(band, rank, world)
        slab.step_bands(ex, [band], steps)
        red = [ex.reduce()]
        slab.step_bands(ex, [band], 3)
        red.append(ex.reduce())
        slab.step_bands(ex, [band], 1)   # the halo exchange before the next step: band state = after steps + 4
        f, g, h = band.stepper.o.state()
        own = band.own
        q.put((rank, r0, r1, f[:, own].copy(), g[:, own].copy(), h[:, own].copy(), red))
    finally:
        dist.destroy_process_group()


def _single_domain(steps, kind="periodic"):
    """The single-domain oracle after steps + 4 steps, with its reductions
    after `steps` and after `steps` + 3."""
    from oracle.oracle import Oracle

    cfg, fl = _problem(kind)
    ref = Oracle(cfg, **fl)
    ref.step(steps)
    red = [ref.reduce()]
    ref.step(3)
    red.append(ref.reduce())
    ref.step(1)
    return cfg, ref.state(), red


def _assert_same_reductions(got, want):
    """phi mass, both residuals and max |u| of the bands against the single
    domain (the sums run over the cells in another order)."""
    for (m, rp, ru, um), (m0, rp0, ru0, um0) in zip(got, want):
        assert m == pytest.approx(m0, rel=1e-13)
        assert rp == pytest.approx(rp0, rel=1e-10)
        assert ru == pytest.approx(ru0, rel=1e-10)
        assert um == um0
    assert got[0][1] == 1.0 and got[1][1] < 1.0


@pytest.mark.parametrize("world,kind", [(1, "periodic"), (1, "wall"), (2, "periodic"), (3, "periodic"),
                                        (2, "wall"), (3, "wall_upwind"), (4, "wall_upwind"), (2, "upwind")])
def test_slabs_with_halo_exchange_equal_the_single_domain(world, kind):
    """gloo ranks, one band each: the bands' own rows and their all-reduced
    reductions equal the single-domain oracle's, bit for bit (the reductions
    to the rounding of a different summation order)."""
    import torch.multiprocessing as mp

    steps = 7
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, steps, kind, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = [q.get(timeout=300) for _ in range(world)]
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    cfg, (F, G, H), red = _single_domain(steps, kind)
    covered = np.zeros(cfg["ny"], dtype=int)
    for rank, r0, r1, f, g, h, band_red in parts:
        _assert_same_reductions(band_red, red)
        assert np.array_equal(f, F[:, r0:r1]), (kind, rank)
        assert np.array_equal(g, G[:, r0:r1]), (kind, rank)
        assert np.array_equal(h, H[:, r0:r1]), (kind, rank)
        covered[r0:r1] += 1
    assert (covered == 1).all()


@pytest.mark.parametrize("kind", KINDS)
def test_local_exchange_of_three_bands(kind):
    """The in-process exchange (the one the GPU test uses) with oracle bands:
    three bands equal the single-domain oracle bit for bit."""
    steps = 5
    cfg, fl = _problem(kind)
    band_list = _band_list(cfg, fl, 3)
    ex = slab.LocalExchange(band_list)
    slab.step_bands(ex, band_list, steps)
    red = [slab.reduce_local(ex, band_list)]
    slab.step_bands(ex, band_list, 3)
    red.append(slab.reduce_local(ex, band_list))
    slab.step_bands(ex, band_list, 1)
    _, (F, G, H), red0 = _single_domain(steps, kind)
    _assert_same_reductions(red, red0)
    for b in band_list:
        f, g, h = b.stepper.o.state()
        assert np.array_equal(f[:, b.own], F[:, b.r0:b.r1]), (kind, b.r0)
        assert np.array_equal(g[:, b.own], G[:, b.r0:b.r1]), (kind, b.r0)
        assert np.array_equal(h[:, b.own], H[:, b.r0:b.r1]), (kind, b.r0)


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


@pytest.mark.parametrize("kind", ["upwind", "wall_upwind"])
def test_upwind_needs_three_halo_rows(kind):
    """The upwind face takes the profile of the cell a direction leaves, one
    row further out than the central face: bands with the central scheme's
    two halo rows no longer equal the single domain, with three they do (the
    test above)."""
    cfg, fl = _problem(kind)
    band_list = _band_list(cfg, fl, 3, halo=2)
    slab.step_bands(slab.LocalExchange(band_list), band_list, 3)
    from oracle.oracle import Oracle

    ref = Oracle(cfg, **fl)
    ref.step(3)
    F = ref.state()[0]
    assert any(not np.array_equal(b.stepper.o.state()[0][:, b.own], F[:, b.r0:b.r1]) for b in band_list)


def test_bands_reject_thin_bands_and_position_dependent_velocity():
    with pytest.raises(ValueError):
        slab.bands(5, 3)
    with pytest.raises(ValueError):
        slab.bands(8, 3, halo=3)
    from paper_1810_07802_gb300 import workloads as W

    cfg, fl = W.zalesak_disk(L=36, R=12.0, slot=3.0, U=0.04)
    assert cfg.get("velocity_field") not in (None, "uniform")
    with pytest.raises(ValueError):
        slab.band_problem(cfg, fl, 0, 12)
    cfg, fl = _problem()
    with pytest.raises(ValueError):
        slab.band_problem(dict(cfg, bc_y="slip"), fl, 0, 10)
    with pytest.raises(ValueError):
        slab.band_layout(cfg, 20, 30)
