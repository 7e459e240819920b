"""Domain decomposition of the step into y-slabs, on the CPU with `gloo` ranks.

Each rank owns a band of rows of a y-periodic problem and steps it with the
FP64 oracle on its band plus two halo rows on each side.  What one step of a
cell reads determines the halo: the update of row j needs psi-bar-plus of rows
j-1 .. j+1 (face reconstruction, Eq. 27), and psi-bar-plus of row j-1 needs
phi (all of f) on rows j-2 .. j (the gradient and Laplacian stencils), with g
and (phi u)^{n-1} on row j-1 itself.  So before every step each rank receives
from its neighbours two rows of f, one row of g and one row of (phi u)^{n-1}
on each side; rows farther out never reach its own rows.  The exchange is a
pair of point-to-point send/receives per neighbour (no collective).  The
bands' rows, gathered after the steps, must equal the single-domain oracle
bit for bit.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HALO = 2


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _bands(ny, world):
    edges = np.linspace(0, ny, world + 1).round().astype(int)
    return [(int(edges[r]), int(edges[r + 1])) for r in range(world)]


def _exchange(dist, torch, rank, world, f, g, h, n_own):
    """Fill the halo rows of (f, g, h) ([planes][n_own + 2 HALO][nx]) from the
    neighbouring ranks' own rows: f two rows, g and h one row per side."""
    up, down = (rank + 1) % world, (rank - 1) % world
    lo, hi = HALO, HALO + n_own            # own rows [lo, hi)

    def rows(a, r0, r1):
        return torch.from_numpy(np.ascontiguousarray(a[:, r0:r1, :]))

    # what each side needs: f 2 rows, g and h 1 row
    send_up = [rows(f, hi - 2, hi), rows(g, hi - 1, hi), rows(h, hi - 1, hi)]
    send_down = [rows(f, lo, lo + 2), rows(g, lo, lo + 1), rows(h, lo, lo + 1)]
    recv_below = [torch.empty_like(t) for t in send_up]      # the lower neighbour's top rows
    recv_above = [torch.empty_like(t) for t in send_down]    # the upper neighbour's bottom rows
    # tags tell the two directions apart (with two ranks both neighbours are one rank)
    ops = []
    for k, t in enumerate(send_up):
        ops.append(dist.P2POp(dist.isend, t, up, tag=k))
    for k, t in enumerate(recv_above):
        ops.append(dist.P2POp(dist.irecv, t, up, tag=3 + k))
    for k, t in enumerate(send_down):
        ops.append(dist.P2POp(dist.isend, t, down, tag=3 + k))
    for k, t in enumerate(recv_below):
        ops.append(dist.P2POp(dist.irecv, t, down, tag=k))
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    f[:, lo - 2:lo, :] = recv_below[0].numpy()
    g[:, lo - 1:lo, :] = recv_below[1].numpy()
    h[:, lo - 1:lo, :] = recv_below[2].numpy()
    f[:, hi:hi + 2, :] = recv_above[0].numpy()
    g[:, hi:hi + 1, :] = recv_above[1].numpy()
    h[:, hi:hi + 1, :] = recv_above[2].numpy()


def _rank_main(rank, world, port, steps, q):
    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    from oracle.oracle import Oracle
    from paper_1810_07802_gb300 import workloads as W

    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        cfg, fl = W.random_state(21, 26, seed=13, rho_ratio=100.0)
        nx, ny = cfg["nx"], cfg["ny"]
        r0, r1 = _bands(ny, world)[rank]
        n_own = r1 - r0
        # this rank's initial state: the single-domain oracle's initial state
        # (R7, built cell by cell) restricted to its band and halo rows
        full = Oracle(cfg, **fl)
        F, G, H = full.state()
        idx = np.arange(r0 - HALO, r1 + HALO) % ny
        f, g, h = F[:, idx, :].copy(), G[:, idx, :].copy(), H[:, idx, :].copy()
        band = Oracle(dict(cfg, ny=n_own + 2 * HALO), **{k: (None if v is None else v[idx, :])
                                                          for k, v in fl.items()})
        for n in range(steps):
            _exchange(dist, torch, rank, world, f, g, h, n_own)
            band.set_state(f, g, h, n)
            band.step(1)
            f, g, h = band.state()
        q.put((rank, r0, r1, f[:, HALO:HALO + n_own].copy(), g[:, HALO:HALO + n_own].copy(),
               h[:, HALO:HALO + n_own].copy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_slabs_with_halo_exchange_equal_the_single_domain(world):
    import torch.multiprocessing as mp

    sys.path.insert(0, ROOT)
    from oracle.oracle import Oracle
    from paper_1810_07802_gb300 import workloads as W

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
    cfg, fl = W.random_state(21, 26, seed=13, rho_ratio=100.0)
    ref = Oracle(cfg, **fl)
    ref.step(steps)
    F, G, H = ref.state()
    covered = np.zeros(cfg["ny"], dtype=int)
    for rank, r0, r1, f, g, h in parts:
        assert np.array_equal(f, F[:, r0:r1]), rank
        assert np.array_equal(g, G[:, r0:r1]), rank
        assert np.array_equal(h, H[:, r0:r1]), rank
        covered[r0:r1] += 1
    assert (covered == 1).all()


def test_one_halo_row_fewer_breaks_the_equality():
    """The halo is no wider than needed: with only one row of f received
    below, the band's first row differs from the single-domain result
    (single process, the exchange done by hand)."""
    sys.path.insert(0, ROOT)
    from oracle.oracle import Oracle
    from paper_1810_07802_gb300 import workloads as W

    cfg, fl = W.random_state(21, 26, seed=13, rho_ratio=100.0)
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
