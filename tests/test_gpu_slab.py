"""The y-slab decomposition on the GPU: bands of one problem (periodic or
walled in y), each a Solver on its rows plus two halo rows (three with the
upwind reconstruction) on each side that has a neighbour, their halo rows
refreshed before every step through dugks_get_rows / dugks_set_rows (device
buffers, exchanged in one process).  (With one GPU per box the same bands over NCCL
between GPUs are not run here: one rank on the NCCL backend is, and the
exchange protocol on several ranks is covered with gloo in
test_slab_decomposition, bit for bit against the oracle.)

On the GPU a cell's result depends on where the tile grid falls at the
round-off level: the same problem shifted cyclically by three rows and
shifted back differs by up to 4.4e-16 (FP64) and one FP32 unit in the last
place after 7 steps.  A band moves the tile grid the same way, so bands are
compared with the single-domain solver to round-off, against that shifted
run as the control, and with the FP64 oracle at the parity bar.  A stale halo
row changes the band's own rows by about 1e-2 in these random states
(8.8e-3 measured), far above either bound."""
import numpy as np
import pytest

from paper_1810_07802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

# max |band - single domain| over the stored distributions after 7 steps
ROUNDOFF = {"fp64": 1e-14, "fp32": 4e-7}


@pytest.fixture(scope="module")
def S():
    from paper_1810_07802_gb300 import build, solver

    build.build()
    solver.lib()
    return solver


@pytest.mark.parametrize("precision,world", [("fp64", 2), ("fp64", 3), ("fp32", 2), ("fp32", 3)])
def test_bands_equal_the_single_domain(S, precision, world):
    from paper_1810_07802_gb300 import slab

    cfg, f = W.random_state(150, 70, seed=31, rho_ratio=100.0)
    cfg = dict(cfg, precision=precision)
    if precision == "fp32":
        cfg["phi_ref"] = 0.5
    steps = 7
    with S.Solver(cfg, **f) as whole:
        whole.step(steps)
        ref = whole.distributions()
    shifted = {k: (None if v is None else np.roll(v, 3, axis=0)) for k, v in f.items()}
    with S.Solver(cfg, **shifted) as s:
        s.step(steps)
        control = max(float(np.abs(np.roll(a, -3, axis=1) - b).max()) for a, b in zip(s.distributions(), ref))
    band_list = []
    for r0, r1 in slab.bands(cfg["ny"], world):
        bcfg, bfields = slab.band_problem(cfg, f, r0, r1)
        band_list.append(slab.Band(S.Solver(bcfg, **bfields), r0, r1, cfg))
    slab.step_bands(slab.LocalExchange(band_list), band_list, steps)
    worst = 0.0
    covered = np.zeros(cfg["ny"], dtype=int)
    for b in band_list:
        got = b.stepper.distributions()
        own = b.own
        for g, r in zip(got, ref):
            worst = max(worst, float(np.abs(g[:, own] - r[:, b.r0:b.r1]).max()))
        covered[b.r0:b.r1] += 1
        b.stepper.close()
    print("\n%s, %d bands: max |band - single domain| %.2e, grid shifted by 3 rows %.2e" % (
        precision, world, worst, control), end="")
    assert (covered == 1).all()
    assert worst <= ROUNDOFF[precision], (worst, control)
    assert control <= ROUNDOFF[precision], control


def test_a_stale_halo_row_is_far_above_the_bound(S):
    """The bound detects a halo fault: with the outermost halo row of f left
    stale (zeroed deviations) before each step, the band's own rows move far
    beyond round-off."""
    from paper_1810_07802_gb300 import slab

    cfg, f = W.random_state(150, 70, seed=31, rho_ratio=100.0)
    steps = 7
    with S.Solver(cfg, **f) as whole:
        whole.step(steps)
        ref = whole.distributions()
    band_list = []
    for r0, r1 in slab.bands(cfg["ny"], 2):
        bcfg, bfields = slab.band_problem(cfg, f, r0, r1)
        band_list.append(slab.Band(S.Solver(bcfg, **bfields), r0, r1, cfg))
    exchange = slab.LocalExchange(band_list)
    b0 = band_list[0]
    row = b0.stepper.row_buffer(1)

    def faulty():
        exchange()
        b0.stepper.get_rows(0, 1, row)
        row[:9].zero_()
        b0.stepper.set_rows(0, 1, row)

    slab.step_bands(faulty, band_list, steps)
    got = b0.stepper.distributions()
    own = b0.own
    err = max(float(np.abs(g[:, own] - r[:, b0.r0:b0.r1]).max()) for g, r in zip(got, ref))
    print("\nstale halo row: max |band - single domain| %.2e" % err, end="")
    for b in band_list:
        b.stepper.close()
    assert err > 1e3 * ROUNDOFF["fp64"], err


@pytest.mark.parametrize("kind", ["periodic", "wall", "upwind", "wall_upwind"])
def test_fp64_bands_match_the_oracle(S, kind):
    """FP64 bands against the single-domain FP64 oracle at the parity bar:
    periodic and walled problems (walled bands: no halo at the problem's
    walls, the bands' inner walls beyond their halo rows), with the central
    reconstruction (two halo rows) and the upwind one (three)."""
    from oracle.oracle import Oracle
    from paper_1810_07802_gb300 import slab

    cfg, f = W.random_state(150, 70, seed=31, rho_ratio=100.0, bc_y="wall" if "wall" in kind else "periodic")
    if "upwind" in kind:
        cfg = dict(cfg, recon="upwind")
    steps = 7
    ref = Oracle(cfg, **f)
    ref.step(steps)
    F, G, Hh = ref.state()
    band_list = []
    for r0, r1 in slab.bands(cfg["ny"], 3, slab.halo_rows(cfg)):
        bcfg, bfields = slab.band_problem(cfg, f, r0, r1)
        band_list.append(slab.Band(S.Solver(bcfg, **bfields), r0, r1, cfg))
    slab.step_bands(slab.LocalExchange(band_list), band_list, steps)
    for b in band_list:
        got = b.stepper.distributions()
        own = b.own
        for g, r in zip(got, (F, G, Hh)):
            assert np.abs(g[:, own] - r[:, b.r0:b.r1]).max() <= 1e-10, (kind, b.r0)
        b.stepper.close()


def test_fp32_walled_bands_equal_the_single_domain(S):
    """FP32-shifted bands of a walled problem against the single-domain FP32
    solver, to the round-off bound of the periodic case."""
    from paper_1810_07802_gb300 import slab

    cfg, f = W.random_state(150, 70, seed=31, rho_ratio=100.0, bc_y="wall")
    cfg = dict(cfg, precision="fp32", phi_ref=0.5)
    with S.Solver(cfg, **f) as whole:
        whole.step(7)
        ref = whole.distributions()
    band_list = []
    for r0, r1 in slab.bands(cfg["ny"], 3):
        bcfg, bfields = slab.band_problem(cfg, f, r0, r1)
        band_list.append(slab.Band(S.Solver(bcfg, **bfields), r0, r1, cfg))
    assert band_list[0].lo == 0 and band_list[-1].hi == 0
    slab.step_bands(slab.LocalExchange(band_list), band_list, 7)
    worst = 0.0
    for b in band_list:
        for g, r in zip(b.stepper.distributions(), ref):
            worst = max(worst, float(np.abs(g[:, b.own] - r[:, b.r0:b.r1]).max()))
        b.stepper.close()
    print("\nfp32 walled, 3 bands: max |band - single domain| %.2e" % worst, end="")
    assert worst <= ROUNDOFF["fp32"], worst


def test_row_copies_round_trip_and_reject_bad_rows(S):
    """get_rows / set_rows move the stored rows exactly; rows outside the grid
    are refused."""
    import torch

    cfg, f = W.random_state(40, 20, seed=5)
    with S.Solver(cfg, **f) as s:
        s.step(2)
        before = s.get_state()
        buf = s.row_buffer(3)
        s.get_rows(5, 3, buf)
        s.set_rows(5, 3, buf)
        torch.cuda.synchronize()
        assert np.array_equal(before, s.get_state())
        with pytest.raises(S.DugksError):
            s.get_rows(18, 3, buf)
        with pytest.raises(ValueError):
            s.get_rows(0, 2, buf)


def test_reduce_rows_over_every_row_is_reduce(S):
    """dugks_reduce_rows over all rows, combined, is dugks_reduce bit for bit
    (the same kernel over the same cells), with and without a previous call."""
    from paper_1810_07802_gb300 import slab

    cfg, f = W.random_state(150, 70, seed=31, rho_ratio=100.0)
    with S.Solver(cfg, **f) as a, S.Solver(cfg, **f) as b:
        for n in (3, 4):
            a.step(n)
            b.step(n)
            want = a.reduce()
            sums, had = b.reduce_rows(0, cfg["ny"])
            assert slab.combine(sums, had) == want
        with pytest.raises(S.DugksError):
            b.reduce_rows(60, 11)


def test_band_reductions_equal_the_single_domain(S):
    """phi mass, the Eq. 44 residuals and max |u| of three FP64 bands, from
    their own-row sums after a halo exchange, against the single-domain
    solver's reduction, after 7 steps (no previous fields) and 3 more."""
    from paper_1810_07802_gb300 import slab

    cfg, f = W.random_state(150, 70, seed=31, rho_ratio=100.0)
    with S.Solver(cfg, **f) as whole:
        whole.step(7)
        want = [whole.reduce()]
        whole.step(3)
        want.append(whole.reduce())
    band_list = []
    for r0, r1 in slab.bands(cfg["ny"], 3):
        bcfg, bfields = slab.band_problem(cfg, f, r0, r1)
        band_list.append(slab.Band(S.Solver(bcfg, **bfields), r0, r1, cfg))
    ex = slab.LocalExchange(band_list)
    slab.step_bands(ex, band_list, 7)
    got = [slab.reduce_local(ex, band_list)]
    slab.step_bands(ex, band_list, 3)
    got.append(slab.reduce_local(ex, band_list))
    for b in band_list:
        b.stepper.close()
    for (m, rp, ru, um), (m0, rp0, ru0, um0) in zip(got, want):
        assert m == pytest.approx(m0, rel=1e-13)
        assert rp == pytest.approx(rp0, rel=1e-9)
        assert ru == pytest.approx(ru0, rel=1e-9)
        assert um == pytest.approx(um0, rel=1e-12)
    assert got[0][1] == 1.0 and got[1][1] < 1.0


def test_one_rank_over_nccl_equals_the_single_domain(S):
    """DistExchange on the NCCL backend with one rank (the one GPU of the
    box): the periodic band is its own neighbour, its halo rows come from its
    own edge rows, and the reductions are all-reduced as CUDA tensors.  The
    band equals the single-domain solver to round-off, and so do its
    reductions.  (Exchanges between GPUs need more than one.)"""
    import datetime
    import socket

    import torch.distributed as dist

    from paper_1810_07802_gb300 import slab

    with socket.socket() as sk:
        sk.bind(("127.0.0.1", 0))
        port = sk.getsockname()[1]
    cfg, f = W.random_state(150, 70, seed=31, rho_ratio=100.0)
    with S.Solver(cfg, **f) as whole:
        whole.step(7)
        want = whole.reduce()
        ref = whole.distributions()
    dist.init_process_group("nccl", init_method="tcp://127.0.0.1:%d" % port, rank=0, world_size=1,
                            timeout=datetime.timedelta(seconds=60))
    try:
        bcfg, bfields = slab.band_problem(cfg, f, 0, cfg["ny"])
        band = slab.Band(S.Solver(bcfg, **bfields), 0, cfg["ny"], cfg)
        ex = slab.DistExchange(band, 0, 1)
        slab.step_bands(ex, [band], 7)
        got = ex.reduce()
        dists = band.stepper.distributions()
        band.stepper.close()
    finally:
        dist.destroy_process_group()
    worst = max(float(np.abs(g[:, band.own] - r).max()) for g, r in zip(dists, ref))
    assert worst <= ROUNDOFF["fp64"], worst
    m, rp, ru, um = got
    assert m == pytest.approx(want[0], rel=1e-13)
    assert rp == 1.0 and ru == 1.0
    assert um == pytest.approx(want[3], rel=1e-12)
