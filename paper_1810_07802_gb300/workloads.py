"""Seeded synthetic inputs shaped like the paper's test problems.

This module only builds parameter dictionaries and initial fields (numpy
float64, shape (ny, nx), x fastest, cell centres at (i + 1/2, j + 1/2)).  It
holds none of the scheme's arithmetic, imports neither the CUDA library nor the
oracle, and is the one module both of them are fed from.

Parameter dictionary keys (all optional except nx, ny):
  nx, ny, model ("coupled" | "ac"), bc_x, bc_y ("periodic" | "wall"),
  visc ("reciprocal" | "linear"), gravity_mode (0 | 1), cfl, mobility, width,
  rho_h, rho_l, mu_h, mu_l, sigma, gx, gy, rho_ref, u0x, u0y,
  precision ("fp64" | "fp32"), phi_ref, p_ref.
"""
import math

import numpy as np

MASK64 = (1 << 64) - 1


def splitmix64_uniform(seed, n):
    """U[0,1) doubles from SplitMix64 (Steele, Lea & Flood, OOPSLA 2014),
    counter-based: value k is the generator's (k+1)-th output from `seed`."""
    k = np.arange(1, n + 1, dtype=np.uint64)
    with np.errstate(over="ignore"):
        z = np.uint64(seed & MASK64) + k * np.uint64(0x9E3779B97F4A7C15)
        z = (z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)
        z = (z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)
        z = z ^ (z >> np.uint64(31))
    return (z >> np.uint64(11)).astype(np.float64) * (1.0 / 9007199254740992.0)


def _centres(nx, ny):
    x = np.arange(nx, dtype=np.float64) + 0.5
    y = np.arange(ny, dtype=np.float64) + 0.5
    return np.meshgrid(x, y)  # each (ny, nx)


def _tanh_profile(z, width):
    """Equilibrium interface profile with phi_H = 1, phi_L = 0 (Eq. 7)."""
    return 0.5 + 0.5 * np.tanh(2.0 * z / width)


def _fields(phi, ux=None, uy=None, p=None):
    return {"phi0": phi, "ux0": ux, "uy0": uy, "p0": p}


def translation_circle(L=64, R=16.0, width=4.0, U=0.01, mobility=0.02, cfl=0.5):
    """Interface diagonal translation (Sec. III.A): a disc of phi = 1 moved by
    the uniform velocity (U, U) through a periodic L x L box."""
    X, Y = _centres(L, L)
    r = np.hypot(X - L / 2.0, Y - L / 2.0)
    cfg = dict(nx=L, ny=L, model="ac", cfl=cfl, mobility=mobility, width=width,
               u0x=U, u0y=U)
    return cfg, _fields(_tanh_profile(R - r, width))


def planar_slab(nx=64, ny=3, width=4.0, U=0.0, mobility=0.02, cfl=0.5, centre=None):
    """A slab of phi = 1 of half-width nx/4 with tanh edges, periodic in both
    directions, advected by (U, 0): a planar version of Sec. III.A."""
    X, _ = _centres(nx, ny)
    c = nx / 2.0 if centre is None else centre
    d = nx / 4.0 - np.abs(X - c)
    cfg = dict(nx=nx, ny=ny, model="ac", cfl=cfl, mobility=mobility, width=width,
               u0x=U, u0y=0.0)
    return cfg, _fields(_tanh_profile(d, width))


def zalesak_disk(L=256, R=100.0, slot=20.0, U=0.02, mobility=0.02, width=4.0, cfl=0.5):
    """Zalesak's slotted disk (Sec. III.B, Eq. 41): a disc of phi = 1 of radius R
    centred in the L x L box with a vertical slot of the given width cut from
    its bottom to 3/4 of its height (the paper's slot proportions are not
    printed); sharp initial step.  One revolution takes T = 2 L / U0."""
    X, Y = _centres(L, L)
    c = L / 2.0
    inside = np.hypot(X - c, Y - c) <= R
    cut = (np.abs(X - c) <= slot / 2.0) & (Y <= c + 0.5 * R)
    phi = np.where(inside & ~cut, 1.0, 0.0)
    cfg = dict(nx=L, ny=L, model="ac", cfl=cfl, mobility=mobility, width=width,
               velocity_field="rotation", vel_u0=U, vel_length=float(L))
    return cfg, _fields(phi)


def shear_elongation(L=256, U=0.02, mobility=0.01, width=4.0, cfl=0.5):
    """Interface elongation in a reversing shear flow (Sec. III.C, Eq. 42): a
    disc of radius L/5 at (0.5 L, 0.3 L); the field reverses after L0 / U0 and
    the disc returns at T = 2 L0 / U0."""
    X, Y = _centres(L, L)
    r = np.hypot(X - 0.5 * L, Y - 0.3 * L)
    cfg = dict(nx=L, ny=L, model="ac", cfl=cfl, mobility=mobility, width=width,
               velocity_field="shear", vel_u0=U, vel_length=float(L))
    return cfg, _fields(_tanh_profile(L / 5.0 - r, width))


def smoothed_deformation(L=512, U=0.02, mobility=0.02, width=4.0, cfl=0.5):
    """Deformation in a smoothed time-periodic shear flow (Sec. III.D, Eq. 43):
    a centred disc of radius L/5, period T = L0 / U0."""
    X, Y = _centres(L, L)
    r = np.hypot(X - 0.5 * L, Y - 0.5 * L)
    cfg = dict(nx=L, ny=L, model="ac", cfl=cfl, mobility=mobility, width=width,
               velocity_field="deformation", vel_u0=U, vel_length=float(L))
    return cfg, _fields(_tanh_profile(L / 5.0 - r, width))


def stationary_bubble(N=128, R=32.0, width=4.0, rho_ratio=1000.0, nu=0.1, sigma=0.01,
                      mobility=0.02, cfl=0.5, visc="linear"):
    """Light bubble (phi = 0) in heavy liquid, periodic N x N (Sec. IV.A, Eq. 45).
    Sec. IV.A keeps one kinematic viscosity nu for the whole field, so
    tau_g = nu / RT everywhere: with mu_H = rho_H nu and mu_L = rho_L nu that is
    the linear rule of Eq. 36 (reading R16), the default here."""
    X, Y = _centres(N, N)
    r = np.hypot(X - N / 2.0, Y - N / 2.0)
    rho_h, rho_l = rho_ratio, 1.0
    cfg = dict(nx=N, ny=N, model="coupled", cfl=cfl, mobility=mobility, width=width,
               rho_h=rho_h, rho_l=rho_l, mu_h=rho_h * nu, mu_l=rho_l * nu, sigma=sigma, visc=visc)
    return cfg, _fields(_tanh_profile(r - R, width))


def spinodal(N=2048, seed=20181018, rho_ratio=1000.0, nu_h=0.01, nu_ratio=10.0, sigma=0.001,
             width=4.0, mobility=0.02, cfl=0.5, amplitude=0.01, nx=None, ny=None):
    """Spinodal decomposition (Sec. IV.C): phi = 0.5 + amplitude (2U - 1) with
    U i.i.d. from SplitMix64(seed) in cell order; nu_L / nu_H = nu_ratio."""
    nx = N if nx is None else nx
    ny = N if ny is None else ny
    u = splitmix64_uniform(seed, nx * ny).reshape(ny, nx)
    phi = 0.5 + amplitude * (2.0 * u - 1.0)
    rho_h, rho_l = rho_ratio, 1.0
    cfg = dict(nx=nx, ny=ny, model="coupled", cfl=cfl, mobility=mobility, width=width,
               rho_h=rho_h, rho_l=rho_l, mu_h=rho_h * nu_h, mu_l=rho_l * nu_h * nu_ratio,
               sigma=sigma, phi_ref=0.5, p_ref=0.0)
    return cfg, _fields(phi)


def rayleigh_taylor(L=256, atwood=0.5, reynolds=3000.0, sqrt_gl=0.04, width=4.0,
                    sigma=5e-5, mobility=0.02, cfl=0.25, ny=None):
    """Rayleigh-Taylor instability (Sec. IV.D, Eqs. 48-49): L x 4L, periodic x,
    no-slip walls in y, heavy fluid on top of H(x) = 2L + 0.1 L cos(2 pi x / L).
    Equal kinematic viscosity in both phases with Re = rho_H L sqrt(gL) / mu_H."""
    ny = 4 * L if ny is None else ny
    X, Y = _centres(L, ny)
    H = ny / 2.0 + 0.1 * L * np.cos(2.0 * math.pi * X / L)
    rho_l = 1.0
    rho_h = rho_l * (1.0 + atwood) / (1.0 - atwood)
    g = sqrt_gl ** 2 / L
    nu = L * sqrt_gl / reynolds
    cfg = dict(nx=L, ny=ny, model="coupled", bc_y="wall", cfl=cfl, mobility=mobility,
               width=width, rho_h=rho_h, rho_l=rho_l, mu_h=rho_h * nu, mu_l=rho_l * nu,
               sigma=sigma, gravity_mode=1, gx=0.0, gy=-g, rho_ref=0.5 * (rho_h + rho_l))
    return cfg, _fields(_tanh_profile(Y - H, width))


def layered_poiseuille(ny=64, nx=4, mu_ratio=100.0, mu_h=1.0, uc=1e-4, width=4.0,
                       sigma=1e-3, mobility=0.02, cfl=0.5, start_from_analytic=False):
    """Layered Poiseuille flow (Sec. IV.B, Eq. 46): walls at y = 0 and y = ny,
    the viscous phase (phi = 1, mu_H) in the lower half, body force G_x with
    u_c = G_x h^2 / (mu_L + mu_H), rho_H = rho_L = 1."""
    mu_l = mu_h / mu_ratio
    h = ny / 2.0
    Gx = uc * (mu_l + mu_h) / h ** 2
    X, Y = _centres(nx, ny)
    phi = _tanh_profile(h - Y, width)
    cfg = dict(nx=nx, ny=ny, model="coupled", bc_y="wall", cfl=cfl, mobility=mobility,
               width=width, rho_h=1.0, rho_l=1.0, mu_h=mu_h, mu_l=mu_l, sigma=sigma,
               gravity_mode=0, gx=Gx, gy=0.0)
    ux = poiseuille_profile(Y, ny, mu_h, mu_l, Gx) if start_from_analytic else None
    return cfg, _fields(phi, ux)


def poiseuille_profile(y, ny, mu_h, mu_l, Gx):
    """Analytic layered Poiseuille velocity (Eq. 46) at heights y in [0, ny];
    the mu_L layer occupies the upper half."""
    h = ny / 2.0
    s = (np.asarray(y, dtype=np.float64) - h) / h
    upper = Gx * h * h / (2 * mu_l) * (-s * s - s * (mu_l - mu_h) / (mu_l + mu_h) + 2 * mu_l / (mu_l + mu_h))
    lower = Gx * h * h / (2 * mu_h) * (-s * s - s * (mu_l - mu_h) / (mu_l + mu_h) + 2 * mu_h / (mu_l + mu_h))
    return np.where(s > 0, upper, lower)


def taylor_green(N=32, U=1e-3, nu=0.1, cfl=0.5):
    """Single-phase decaying Taylor-Green vortex (phi = 1 everywhere, sigma = 0)."""
    X, Y = _centres(N, N)
    k = 2.0 * math.pi / N
    ux = -U * np.cos(k * X) * np.sin(k * Y)
    uy = U * np.sin(k * X) * np.cos(k * Y)
    p = -0.25 * U * U * (np.cos(2 * k * X) + np.cos(2 * k * Y))
    cfg = dict(nx=N, ny=N, model="coupled", cfl=cfl, mobility=0.02, width=4.0,
               rho_h=1.0, rho_l=1.0, mu_h=nu, mu_l=nu, sigma=0.0)
    return cfg, _fields(np.ones((N, N)), ux, uy, p)


def random_state(nx, ny, seed=1, rho_ratio=1000.0, model="coupled", bc_y="periodic",
                 amplitude=0.3, velocity=1e-3):
    """A rough, asymmetric coupled state for parity tests: an off-centre bubble
    with phi kept inside (0.03, 0.97) (so rho > 0 at any density ratio), plus
    cell noise, small random velocities and pressure."""
    u = splitmix64_uniform(seed, 4 * nx * ny).reshape(4, ny, nx)
    X, Y = _centres(nx, ny)
    r = np.hypot(X - 0.4 * nx, Y - 0.55 * ny)
    phi = 0.05 + 0.9 * _tanh_profile(r - 0.25 * min(nx, ny), 3.0) + amplitude * (u[0] - 0.5) * 0.1
    ux = velocity * (2 * u[1] - 1)
    uy = velocity * (2 * u[2] - 1)
    p = 1e-4 * (2 * u[3] - 1)
    cfg = dict(nx=nx, ny=ny, model=model, bc_y=bc_y, cfl=0.5, mobility=0.02, width=3.0,
               rho_h=rho_ratio, rho_l=1.0, mu_h=0.1 * rho_ratio, mu_l=0.05, sigma=0.01,
               gravity_mode=1, gx=1e-6, gy=-2e-6, rho_ref=0.5 * (rho_ratio + 1.0),
               u0x=0.01, u0y=-0.007)
    return cfg, _fields(phi, ux, uy, p)


def serving_trace(n=100, rate=50.0, seed=20181018, precision="fp32", burst=False,
                  steps=None):
    """A seeded stream of coupled solve requests shaped like the serving mix:
    layered Poiseuille (mu* = 100, Nx = 4, Ny in {64..512}), stationary bubbles
    (N in {64..512}, R = N/4, density ratio in {10, 100, 1000}, the paper's
    bubble width W = 5, with which ratio 1000 is stable) and spinodal
    boxes (N in {128..1024}), with Poisson arrivals of mean `rate` per second
    (all at t = 0 if burst).  Returns (kind, cfg, fields, steps, arrival)
    tuples.  Step budgets per kind: Poiseuille 400, bubble 100, spinodal 200
    (fixed budgets instead of a convergence test keep runs reproducible)."""
    steps = steps or {"poiseuille": 400, "bubble": 100, "spinodal": 200}
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for i in range(n):
        kind = ("poiseuille", "bubble", "spinodal")[int(rng.integers(3))]
        if kind == "poiseuille":
            cfg, f = layered_poiseuille(ny=int(rng.choice([64, 128, 256, 512])), nx=4, mu_ratio=100.0, mu_h=1.0)
        elif kind == "bubble":
            N = int(rng.choice([64, 128, 256, 512]))
            cfg, f = stationary_bubble(N=N, R=N / 4.0, width=5.0,
                                       rho_ratio=float(rng.choice([10.0, 100.0, 1000.0])))
        else:
            N = int(rng.choice([128, 256, 512, 1024]))
            cfg, f = spinodal(N=N, seed=seed + i)
        cfg["precision"] = precision
        if precision == "fp32":
            cfg.setdefault("phi_ref", 0.5)
        if not burst:
            t += float(rng.exponential(1.0 / rate))
        out.append((kind, cfg, f, steps[kind], 0.0 if burst else t))
    return out
