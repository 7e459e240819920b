"""One coupled DUGKS step restricted to fields that do not vary along x, with
switchable readings of the passages the paper leaves open -- an analysis aid
for the density-ratio stability study, not a second oracle.

For a state uniform in x the two-dimensional scheme of Sec. II.B reduces
exactly to a problem in y alone: the isotropic gradient becomes the central
difference (phi_{j+1} - phi_{j-1}) / 2, the nine-point Laplacian becomes
phi_{j+1} + phi_{j-1} - 2 phi_j, the x-faces carry equal fluxes on both sides
of a cell (their divergence vanishes), and the central reconstruction of a
y-face (Eq. 27) has no tangential slope.  With every switch at its default this
module computes what the oracle computes for such a state (the tests check it
to round-off); each switch replaces one reading by an alternative so that its
effect on the linear stability of a planar interface can be measured.

Readings that can be switched (defaults are the oracle's):
  cell_pressure_drho  factor on the (dt/2) u . grad rho term of Eq. 33 at a
                      cell centre (1 = as printed)
  cell_pressure_s0    add the -(dt/2) S^g_0 term that the derivation of Eq. 33
                      from Eq. 23a leaves out (0 = as printed)
  face_half           the half-step used by the face macros of u and p: "h"
                      (psi_bar is psi shifted by h/2 of collision and source)
                      or "dt" (Eqs. 32-33 applied at the face as printed)
  face_up             face u and p: "bar" (from the reconstructed g_bar) or
                      "mean" (mean of the two cells' u and p)
  face_drho           face grad rho: "mean" (of the two cells) or "compact"
                      (rho(phi_f) difference of the two cells)
  visc                "reciprocal" (Eq. 35) or "linear" (Eq. 36)
"""
from dataclasses import dataclass

import numpy as np

RT = 1.0 / 3.0
EX = np.array([0, 1, 1, 0, -1, -1, -1, 0, 1], dtype=np.float64)
EY = np.array([0, 0, 1, 1, 1, 0, -1, -1, -1], dtype=np.float64)
WQ = np.array([4 / 9, 1 / 9, 1 / 36, 1 / 9, 1 / 36, 1 / 9, 1 / 36, 1 / 9, 1 / 36])


@dataclass
class Reading:
    cell_pressure_drho: float = 1.0
    cell_pressure_s0: float = 0.0
    face_half: str = "h"
    face_up: str = "bar"
    face_drho: str = "mean"
    visc: str = "reciprocal"


@dataclass
class Physics:
    ny: int
    cfl: float = 0.5
    mobility: float = 0.02
    width: float = 4.0
    rho_h: float = 1000.0
    rho_l: float = 1.0
    mu_h: float = 100.0
    mu_l: float = 0.1
    sigma: float = 0.01


def _gamma(ux, uy):
    """Gamma_i(u) of Eq. 18 for arrays of points: shape (9, n)."""
    eu = EX[:, None] * ux + EY[:, None] * uy
    return WQ[:, None] * (1.0 + eu / RT + eu * eu / (2 * RT * RT) - (ux * ux + uy * uy) / (2 * RT))


def _props(P, rd, phi, dphiy, lap):
    """rho, d rho / dy, mu_phi, tau_g, theta, n_y, F_y at points (Eqs. 3-10, 34-36)."""
    beta, kappa = 12 * P.sigma / P.width, 1.5 * P.sigma * P.width
    rho = (P.rho_h - P.rho_l) * phi + P.rho_l
    drho = (P.rho_h - P.rho_l) * dphiy
    muphi = 4 * beta * phi * (phi - 1) * (phi - 0.5) - kappa * lap
    if rd.visc == "reciprocal":
        mu = 1.0 / (phi * (1 / P.mu_h - 1 / P.mu_l) + 1 / P.mu_l)
    else:
        mu = phi * (P.mu_h - P.mu_l) + P.mu_l
    tau = mu / (rho * RT)
    theta = 4 * phi * (1 - phi) / P.width
    ny_ = dphiy / np.sqrt(dphiy * dphiy + 1e-16)
    F = muphi * dphiy
    return rho, drho, tau, theta, ny_, F


def _geq(p, rho, ux, uy):
    rest = WQ.copy()
    rest[0] -= 1.0
    return p / RT * rest[:, None] + rho * (_gamma(ux, uy) - WQ[:, None])


def _sg(drho, F, ux, uy):
    gu = _gamma(ux, uy)
    ay = (gu - WQ[:, None]) * RT * drho + F * gu
    ax = np.zeros_like(ay)
    return ((EX[:, None] - ux) * ax + (EY[:, None] - uy) * ay) / RT


def _feq(phi, ux, uy):
    return WQ[:, None] * phi * (1 + (EX[:, None] * ux + EY[:, None] * uy) / RT)


def _sf(theta, ny_, Dx, Dy):
    return WQ[:, None] * theta * (EY[:, None] * ny_) + WQ[:, None] * (EX[:, None] * Dx + EY[:, None] * Dy) / RT


def _pressure(P, rd, sum_nonrest, half, ux, uy, rho, drho, s0_factor=0.0, F=None):
    g0 = _gamma(ux, uy)[0] - WQ[0]
    extra = 0.0
    if s0_factor:
        # S^g_0 with xi_0 = 0 (Eq. 19): -u . {(Gamma_0 - w_0) grad(rho RT) + F Gamma_0} / RT
        gu0 = _gamma(ux, uy)[0]
        s0 = -(uy * ((gu0 - WQ[0]) * RT * drho + F * gu0)) / RT
        extra = -s0_factor * half * s0
    return RT / (1 - WQ[0]) * (sum_nonrest + half * uy * drho + rho * g0 + extra)


def step(P, rd, f, g, phiu, first=False):
    """One step of x-uniform state arrays f, g: (9, ny); phiu: (2, ny).
    Returns the new (f, g, phiu).  `first` means step number 0 (d_t(phi u) = 0)."""
    ny, dt = P.ny, P.cfl
    h = 0.5 * dt
    up = lambda a: np.roll(a, -1, axis=-1)
    dn = lambda a: np.roll(a, 1, axis=-1)
    phi = f.sum(axis=0)
    dphiy = 0.5 * (up(phi) - dn(phi))
    lap = up(phi) + dn(phi) - 2 * phi
    rho, drho, tau, theta, ny_, F = _props(P, rd, phi, dphiy, lap)
    mx = (EX[:, None] * g).sum(axis=0)
    my = (EY[:, None] * g).sum(axis=0)
    ux = mx / rho
    uy = (my + 0.5 * dt * F) / rho
    s = g[1:].sum(axis=0)
    p = RT / (1 - WQ[0]) * (s + rd.cell_pressure_drho * 0.5 * dt * uy * drho
                            + rho * (_gamma(ux, uy)[0] - WQ[0]))
    if rd.cell_pressure_s0:
        gu0 = _gamma(ux, uy)[0]
        s0 = -(uy * ((gu0 - WQ[0]) * RT * drho + F * gu0)) / RT
        p = p + RT / (1 - WQ[0]) * (-rd.cell_pressure_s0 * 0.5 * dt * s0)
    if first:
        Dx = np.zeros(ny)
        Dy = np.zeros(ny)
    else:
        Dx = (phi * ux - phiu[0]) / dt
        Dy = (phi * uy - phiu[1]) / dt
    tau_f = P.mobility / RT
    # Eqs. 29-30
    feq, sf = _feq(phi, ux, uy), _sf(theta, ny_, Dx, Dy)
    geq, sg = _geq(p, rho, ux, uy), _sg(drho, F, ux, uy)
    fb = (2 * tau_f - h) / (2 * tau_f + dt) * f + 3 * h / (2 * tau_f + dt) * feq + 3 * tau_f * h / (2 * tau_f + dt) * sf
    gb = (2 * tau - h) / (2 * tau + dt) * g + 3 * h / (2 * tau + dt) * geq + 3 * tau * h / (2 * tau + dt) * sg
    ft = 4.0 / 3.0 * fb - f / 3.0
    gt = 4.0 / 3.0 * gb - g / 3.0
    # y-face below row j (between j-1 and j): Eq. 27 with the central profile
    rec = lambda B: 0.5 * (dn(B) + B) - h * EY[:, None] * (B - dn(B))
    fbar, gbar = rec(fb), rec(gb)
    phif = fbar.sum(axis=0)
    dphif = 0.5 * (dn(dphiy) + dphiy)
    lapf = 0.5 * (dn(lap) + lap)
    Dxf, Dyf = 0.5 * (dn(Dx) + Dx), 0.5 * (dn(Dy) + Dy)
    rhof, drhof, tauf, thetaf, nyf, Ff = _props(P, rd, phif, dphif, lapf)
    if rd.face_drho == "compact":
        drhof = (P.rho_h - P.rho_l) * (phi - dn(phi))
    half = h if rd.face_half == "h" else dt
    if rd.face_up == "bar":
        uxf = (EX[:, None] * gbar).sum(axis=0) / rhof
        uyf = ((EY[:, None] * gbar).sum(axis=0) + 0.5 * half * Ff) / rhof
        pf = _pressure(P, rd, gbar[1:].sum(axis=0), 0.5 * half, uxf, uyf, rhof, drhof,
                       rd.cell_pressure_s0, Ff)
    else:
        uxf, uyf, pf = 0.5 * (dn(ux) + ux), 0.5 * (dn(uy) + uy), 0.5 * (dn(p) + p)
    fe, fs = _feq(phif, uxf, uyf), _sf(thetaf, nyf, Dxf, Dyf)
    ge, gs = _geq(pf, rhof, uxf, uyf), _sg(drhof, Ff, uxf, uyf)
    fpsi = 2 * tau_f / (2 * tau_f + h) * fbar + h / (2 * tau_f + h) * fe + tau_f * h / (2 * tau_f + h) * fs
    gpsi = 2 * tauf / (2 * tauf + h) * gbar + h / (2 * tauf + h) * ge + tauf * h / (2 * tauf + h) * gs
    # Eq. 24: the flux through the face above row j minus the one below it
    fn = ft - dt * EY[:, None] * (up(fpsi) - fpsi)
    gn = gt - dt * EY[:, None] * (up(gpsi) - gpsi)
    return fn, gn, np.stack([phi * ux, phi * uy])


def initial_state(P, rd, phi):
    """R7: psi~ = psi_eq - dt/2 S at rest (u = 0, p = 0, d_t(phi u) = 0)."""
    up = lambda a: np.roll(a, -1)
    dn = lambda a: np.roll(a, 1)
    dphiy = 0.5 * (up(phi) - dn(phi))
    lap = up(phi) + dn(phi) - 2 * phi
    rho, drho, tau, theta, ny_, F = _props(P, rd, phi, dphiy, lap)
    z = np.zeros_like(phi)
    f = _feq(phi, z, z) - 0.5 * P.cfl * _sf(theta, ny_, z, z)
    g = _geq(z, rho, z, z) - 0.5 * P.cfl * _sg(drho, F, z, z)
    return f, g, np.zeros((2, P.ny))


def planar_interface(ny, width):
    """A layer of the light phase (phi = 0) of thickness ny/2 in the middle of a
    periodic column of the heavy one, with the tanh edges of Eq. 7."""
    y = np.arange(ny) + 0.5
    return 0.5 + 0.5 * np.tanh(2.0 * (np.abs(y - ny / 2.0) - ny / 4.0) / width)


def g_jacobian(P, rd, phi, eps=1e-7):
    """Jacobian of g~ -> g~ over one step (a step other than the first) at the
    rest state of the interface phi, with f~ and (phi u)^{n-1} held at that
    state (phi frozen).  Central differences in each component of g~."""
    f, g, phiu = initial_state(P, rd, phi)
    n = g.size
    J = np.zeros((n, n))
    base = g.ravel()
    for k in range(n):
        e = np.zeros(n)
        e[k] = eps
        gp = step(P, rd, f, (base + e).reshape(g.shape), phiu)[1].ravel()
        gm = step(P, rd, f, (base - e).reshape(g.shape), phiu)[1].ravel()
        J[:, k] = (gp - gm) / (2 * eps)
    return J


def spectral_radius(P, rd, phi=None):
    if phi is None:
        phi = planar_interface(P.ny, P.width)
    return float(np.abs(np.linalg.eigvals(g_jacobian(P, rd, phi))).max())
