"""The y-slab decomposition on the GPU: bands of one periodic problem, each a
Solver on its rows plus two halo rows per side, their halo rows refreshed
before every step through dugks_get_rows / dugks_set_rows (device buffers,
exchanged in one process).  Every band's own rows equal the single-domain
solver's bit for bit, FP64 and FP32-shifted, for two and three bands.  (With
one GPU per box the same bands over NCCL between GPUs are not run here; the
exchange protocol on ranks is covered with gloo in test_slab_decomposition.)"""
import numpy as np
import pytest

from paper_1810_07802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_1810_07802_gb300 import build, solver

    build.build()
    solver.lib()
    return solver


@pytest.mark.parametrize("precision,world", [("fp64", 2), ("fp64", 3), ("fp32", 2)])
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
    band_list = []
    for r0, r1 in slab.bands(cfg["ny"], world):
        bcfg, bfields = slab.band_problem(cfg, f, r0, r1)
        band_list.append(slab.Band(S.Solver(bcfg, **bfields), r0, r1))
    slab.step_bands(slab.LocalExchange(band_list), band_list, steps)
    for b in band_list:
        got = b.stepper.distributions()
        own = slice(slab.HALO, slab.HALO + b.n_own)
        for name, g, r in zip(("f", "g", "phiu"), got, ref):
            assert np.array_equal(g[:, own], r[:, b.r0:b.r1]), (precision, world, b.r0, name)
        b.stepper.close()


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
