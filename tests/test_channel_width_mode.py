"""The layered channel of Sec. IV.B at the paper's viscosity ratio (1000),
on the FP64 oracle: why the absolute viscosity is a reading.

The paper gives only mu_H / mu_L.  With mu_H = 10 the viscous layer's
tau_g = 3 mu_H / rho = 30 lets a mode across the 4-cell width of the channel
grow once the channel is tall enough (Ny = 192 here), from any seed: x 12
per 1,000 steps.  With mu_H = 5 (the value the paper-case tests use) the
same seed stays at its size, and at Ny = 128 neither grows it (mu_H = 10
damps it to round-off).  The x-uniform state is seeded
with 1e-12 noise in u, the size round-off gives the GPU's tiles.  Amplitude:
max over the cells of |u_x - (row mean of u_x)|.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07802_gb300 import workloads as W


def _mode_amplitudes(ny, mu_h, chunks=5, chunk=1000):
    cfg, f = W.layered_poiseuille(ny=ny, mu_ratio=1000.0, mu_h=mu_h, start_from_analytic=True)
    r = np.random.default_rng(1)
    f = dict(f, ux0=f["ux0"] + 1e-12 * r.standard_normal(f["ux0"].shape))
    o = Oracle(cfg, **f)
    amps = []
    for _ in range(chunks):
        o.step(chunk)
        u = o.macros()["ux"]
        amps.append(float(np.abs(u - u.mean(axis=1, keepdims=True)).max()))
    return amps


def test_the_width_mode_grows_at_mu_h_10_and_not_at_5():
    grow = _mode_amplitudes(192, 10.0)
    keep = _mode_amplitudes(192, 5.0)
    # about 0.25 % per step: x 12 or more per 1,000 steps once it dominates
    assert grow[-1] > 1e3 * grow[0], grow
    assert all(b > 5 * a for a, b in zip(grow[1:], grow[2:])), grow
    assert max(keep) < 1e-10 and keep[-1] < 2 * keep[0], keep


@pytest.mark.parametrize("mu_h", [10.0, 5.0])
def test_a_shorter_channel_keeps_the_seed(mu_h):
    amps = _mode_amplitudes(128, mu_h, chunks=4)
    assert max(amps) < 1e-10 and amps[-1] < 2 * amps[0], amps
