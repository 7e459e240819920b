"""Linear stability of the hydrodynamic model at a planar interface, as a
function of density ratio, interface width W and the readings of the passages
the paper leaves open (Sec. II.B, Eqs. 31-36).

The quantity measured is the spectral radius of the one-step Jacobian of the
g-model (g~ -> g~, phi frozen at a tanh interface at rest).  A value above 1
is a mode that grows by that factor every step.  The oracle provides it
directly (finite differences of its own step); `planar_scheme` restates the
step for fields uniform in x, with switchable readings, and is checked here
against the oracle first.

Findings the tests hold fixed:
  * density ratio <= 30: stable for W = 4 and 5 under both viscosity rules;
  * density ratio 1000 with the paper's bubble parameters (W = 5, one
    kinematic viscosity for the whole field, Sec. IV.A, i.e. Eq. 36 with
    mu_H / mu_L = rho_H / rho_L): stable, in every mode of a 2-D grid;
  * density ratio 1000 at W = 4: unstable (1.026 per step with the linear
    rule, 1.075 with the reciprocal one), and no alternative reading of the
    face macros, of the face density gradient or of the S^g_0 term dropped
    from Eq. 33 removes it; only scaling down the (dt/2) u . grad rho term of
    Eq. 33 does, which no passage supports.
"""
import numpy as np
import pytest

import planar_scheme as PS
from oracle import oracle as O

TOL_STABLE = 1e-6   # finite-difference noise on a neutral eigenvalue


def _cfg(P, visc, nx):
    return dict(nx=nx, ny=P.ny, model="coupled", cfl=P.cfl, mobility=P.mobility, width=P.width,
                rho_h=P.rho_h, rho_l=P.rho_l, mu_h=P.mu_h, mu_l=P.mu_l, sigma=P.sigma, visc=visc)


def _physics(ratio, width, ny=32, nu=0.1, **kw):
    return PS.Physics(ny=ny, width=width, rho_h=ratio, mu_h=ratio * nu, mu_l=nu, **kw)


def _oracle_g_jacobian(P, visc, nx, eps=1e-7):
    """Jacobian of one oracle step g~ -> g~ (phi frozen) on an nx x ny grid
    holding the planar interface in every column, all 9 nx ny components."""
    phi = np.tile(PS.planar_interface(P.ny, P.width)[:, None], (1, nx))
    o = O.Oracle(_cfg(P, visc, nx), phi)
    f, g, h = o.state()
    base = g.ravel().copy()

    def apply(v):
        o.set_state(f, v.reshape(g.shape), h, 1)
        o.step(1)
        return o.state()[1].ravel()

    J = np.zeros((base.size, base.size))
    for k in range(base.size):
        e = np.zeros(base.size)
        e[k] = eps
        J[:, k] = (apply(base + e) - apply(base - e)) / (2 * eps)
    return J


def _radius(J):
    return float(np.abs(np.linalg.eigvals(J)).max())


@pytest.mark.parametrize("visc", ["reciprocal", "linear"])
def test_restatement_is_the_oracle_step(visc):
    """With every reading at its default, planar_scheme.step is the oracle's
    step of an x-uniform state (a perturbed interface, not the first step)."""
    P = _physics(1000.0, 4.0, ny=24)
    rd = PS.Reading(visc=visc)
    rng = np.random.default_rng(7)
    f, g, h = PS.initial_state(P, rd, PS.planar_interface(P.ny, P.width))
    f = f + 1e-4 * rng.standard_normal(f.shape)
    g = g + 1e-4 * rng.standard_normal(g.shape)
    h = h + 1e-5 * rng.standard_normal(h.shape)
    nx = 3
    o = O.Oracle(_cfg(P, visc, nx), np.tile(PS.planar_interface(P.ny, P.width)[:, None], (1, nx)))
    rep = lambda a: np.repeat(a[:, :, None], nx, axis=2)
    o.set_state(rep(f), rep(g), rep(h), 5)
    o.step(1)
    fo, go, ho = o.state()
    fn, gn, hn = PS.step(P, rd, f, g, h)
    for k in range(nx):
        assert np.abs(fo[:, :, k] - fn).max() < 1e-15
        assert np.abs(go[:, :, k] - gn).max() < 1e-15
        assert np.abs(ho[:, :, k] - hn).max() < 1e-18


def test_oracle_jacobian_matches_restatement():
    """The x-uniform block of the oracle's Jacobian has the restatement's
    spectral radius (ratio 1000, W = 4, reciprocal rule: the unstable case)."""
    P = _physics(1000.0, 4.0, ny=24)
    phi = PS.planar_interface(P.ny, P.width)
    o = O.Oracle(_cfg(P, "reciprocal", 3), np.tile(phi[:, None], (1, 3)))
    f, g, h = o.state()
    base = g[:, :, 0].ravel().copy()

    def apply(v):
        G = np.repeat(v.reshape(9, P.ny, 1), 3, axis=2)
        o.set_state(f, G, h, 1)
        o.step(1)
        return o.state()[1][:, :, 0].ravel()

    J = np.zeros((base.size, base.size))
    for k in range(base.size):
        e = np.zeros(base.size)
        e[k] = 1e-7
        J[:, k] = (apply(base + e) - apply(base - e)) / 2e-7
    r_oracle = _radius(J)
    r_restated = PS.spectral_radius(P, PS.Reading(visc="reciprocal"))
    assert r_oracle > 1.05
    assert abs(r_oracle - r_restated) < 1e-6


@pytest.mark.parametrize("visc", ["reciprocal", "linear"])
@pytest.mark.parametrize("ratio", [1.0, 10.0, 30.0])
@pytest.mark.parametrize("width", [4.0, 5.0])
def test_moderate_density_ratios_are_stable(visc, ratio, width):
    assert PS.spectral_radius(_physics(ratio, width), PS.Reading(visc=visc)) < 1 + TOL_STABLE


def test_ratio_1000_stability_map():
    """The printed scheme at density ratio 1000: unstable at W = 4 under both
    viscosity rules and at W = 5 under the reciprocal rule; stable from W = 5
    with one kinematic viscosity for the whole field (the linear rule)."""
    r = {(v, w): PS.spectral_radius(_physics(1000.0, w), PS.Reading(visc=v))
         for v in ("reciprocal", "linear") for w in (4.0, 5.0, 6.0)}
    assert r[("reciprocal", 4.0)] > 1.05
    assert r[("reciprocal", 5.0)] > 1.02
    assert r[("linear", 4.0)] > 1.02
    assert r[("linear", 5.0)] < 1 + TOL_STABLE
    assert r[("linear", 6.0)] < 1 + TOL_STABLE


@pytest.mark.parametrize("visc", ["reciprocal", "linear"])
def test_no_alternative_reading_stabilises_width_4(visc):
    """Density ratio 1000, W = 4: the face macros taken with dt instead of h,
    face u and p as cell means, a compact face density difference, and the
    S^g_0 term of the derivation of Eq. 33 kept all leave a growing mode; the
    mode lives in the (dt/2) u . grad rho term of Eq. 33 (halving it removes
    it), which the paper prints as is."""
    P = _physics(1000.0, 4.0)
    alternatives = [dict(face_half="dt"), dict(face_up="mean"), dict(face_drho="compact"),
                    dict(cell_pressure_s0=1.0)]
    for kw in alternatives:
        assert PS.spectral_radius(P, PS.Reading(visc=visc, **kw)) > 1.02, kw
    assert PS.spectral_radius(P, PS.Reading(visc=visc, cell_pressure_drho=0.5)) < 1 + TOL_STABLE


def test_paper_bubble_parameters_stable_in_two_dimensions():
    """Every mode of a 4 x 24 grid (x-wavenumbers 0, pi/2 and pi) is stable at
    density ratio 1000 with the paper's bubble parameters (W = 5, M = 0.1,
    one kinematic viscosity 0.1 for the whole field: the linear rule)."""
    P = _physics(1000.0, 5.0, ny=24, mobility=0.1)
    assert _radius(_oracle_g_jacobian(P, "linear", 4)) < 1 + TOL_STABLE
