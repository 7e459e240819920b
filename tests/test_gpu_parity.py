"""GPU parity: the CUDA path (through the C ABI) against the FP64 CPU oracle.

FP64 bar: max |GPU - oracle| <= 1e-10 on phi, p, u (and on the stored
distributions) after the configured steps, on identical seeded inputs.
Sizes span several tiles and ragged tails (FP64 tiles are 16 x 16, FP32
tiles 32 x 8), tiny grids smaller than one tile, and walls.
"""
import numpy as np
import pytest

from oracle.oracle import Oracle
from paper_1810_07802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

TOL = 1e-10


@pytest.fixture(scope="module")
def S():
    from paper_1810_07802_gb300 import build, solver

    build.build()
    solver.lib()
    return solver


def run_both(S, cfg, fields, steps):
    with S.Solver(cfg, **fields) as s:
        s.step(steps)
        got = s.macros()
        dist = s.distributions()
    o = Oracle(cfg, **fields)
    o.step(steps)
    return got, o.macros(), dist, o.state()


def assert_parity(got, ref, dist=None, state=None, tol=TOL, what=""):
    for k in ("phi", "p", "ux", "uy"):
        err = np.abs(got[k] - ref[k]).max()
        assert err <= tol, "%s %s: max err %.3e" % (what, k, err)
    if dist is not None:
        for name, a, b in zip(("f", "g", "phiu"), dist, state):
            err = np.abs(a - b).max()
            assert err <= tol, "%s %s: max err %.3e" % (what, name, err)


@pytest.mark.parametrize("nx,ny,steps", [(37, 29, 1), (37, 29, 12), (16, 16, 3), (3, 3, 4),
                                         (5, 40, 6), (70, 9, 5), (33, 17, 20)])
def test_coupled_periodic_fp64(S, nx, ny, steps):
    cfg, f = W.random_state(nx, ny, seed=nx * 100 + ny)
    got, ref, dist, st = run_both(S, cfg, f, steps)
    assert_parity(got, ref, dist, st, what="%dx%d/%d" % (nx, ny, steps))


@pytest.mark.parametrize("nx,ny,steps,bc_y", [(150, 70, 6, "periodic"), (131, 53, 9, "wall"), (96, 40, 4, "periodic")])
def test_interior_tiles_fp64(S, nx, ny, steps, bc_y):
    """Grids large enough for interior tiles, whose input box is staged by TMA
    (edge tiles use plain loads): both paths in one run against the oracle."""
    cfg, f = W.random_state(nx, ny, seed=nx + 3 * ny, bc_y=bc_y)
    got, ref, dist, st = run_both(S, cfg, f, steps)
    assert_parity(got, ref, dist, st, what="interior %dx%d %s" % (nx, ny, bc_y))


@pytest.mark.parametrize("bc_y", ["periodic", "wall"])
def test_interior_tiles_fp32(S, bc_y):
    """FP32-shifted on a grid with interior (TMA-staged) tiles: within FP32
    round-off of the FP64 oracle after a few steps."""
    cfg, f = W.random_state(150, 70, seed=17, bc_y=bc_y)
    with S.Solver(dict(cfg, precision="fp32", phi_ref=0.5), **f) as s:
        s.step(6)
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(6)
    ref = o.macros()
    assert np.abs(got["phi"] - ref["phi"]).max() <= 2e-5
    assert np.abs(got["ux"] - ref["ux"]).max() <= 1e-7
    assert np.abs(got["p"] - ref["p"]).max() <= 1e-5


@pytest.mark.parametrize("nx,ny,steps", [(37, 29, 8), (20, 3, 5), (17, 33, 10), (40, 4, 3)])
def test_coupled_walls_fp64(S, nx, ny, steps):
    cfg, f = W.random_state(nx, ny, seed=7 + nx, bc_y="wall")
    got, ref, dist, st = run_both(S, cfg, f, steps)
    assert_parity(got, ref, dist, st, what="walls %dx%d" % (nx, ny))


@pytest.mark.parametrize("visc,grav", [("linear", 0), ("reciprocal", 0), ("linear", 1)])
def test_closure_options_fp64(S, visc, grav):
    cfg, f = W.random_state(24, 20, seed=5)
    cfg.update(visc=visc, gravity_mode=grav)
    got, ref, dist, st = run_both(S, cfg, f, 6)
    assert_parity(got, ref, dist, st, what="%s/%d" % (visc, grav))


@pytest.mark.parametrize("bc_y", ["periodic", "wall"])
def test_allen_cahn_only_fp64(S, bc_y):
    cfg, f = W.translation_circle(L=40, R=10.0, U=0.02)
    cfg["bc_y"] = bc_y
    got, ref, dist, st = run_both(S, cfg, f, 25)
    assert_parity(got, ref, dist, st, what="A-C " + bc_y)


@pytest.mark.parametrize("name,steps", [("rotation", 40), ("shear", 30), ("deformation", 30),
                                        ("shear_reversal", 420)])
def test_prescribed_velocity_fields_fp64(S, name, steps):
    """A-C-only model with the paper's rotation (Eq. 41), reversing shear (Eq. 42)
    and smoothed deformation (Eq. 43) fields, including a run across the shear's
    reversal time."""
    if name == "rotation":
        cfg, f = W.zalesak_disk(L=40, R=15.0, slot=4.0, U=0.04)
    elif name == "shear":
        cfg, f = W.shear_elongation(L=48, U=0.04)
    elif name == "deformation":
        cfg, f = W.smoothed_deformation(L=64, U=0.04)
    else:
        cfg, f = W.shear_elongation(L=16, U=0.08, width=2.0)
    got, ref, dist, st = run_both(S, cfg, f, steps)
    assert_parity(got, ref, dist, st, what=name)


def test_prescribed_velocity_fp32(S):
    cfg, f = W.smoothed_deformation(L=96, U=0.04)
    with S.Solver(dict(cfg, precision="fp32"), **f) as s:
        s.step(30)
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(30)
    ref = o.macros()
    assert np.abs(got["phi"] - ref["phi"]).max() <= 2e-5


def test_paper_workloads_fp64(S):
    """Reduced-size versions of the paper's problems: bubble, Poiseuille, RTI."""
    cases = [W.stationary_bubble(N=48, R=12.0, rho_ratio=1000.0),
             W.layered_poiseuille(ny=40, nx=4, mu_ratio=100.0),
             W.rayleigh_taylor(L=32, ny=64),
             W.taylor_green(N=32)]
    for cfg, f in cases:
        got, ref, dist, st = run_both(S, cfg, f, 30)
        assert_parity(got, ref, dist, st, what=str(cfg["nx"]) + "x" + str(cfg["ny"]))


def test_spinodal_full_size_one_step_fp64(S):
    """The 2048^2 spinodal box (the throughput workload) in the launch
    configuration the bench times: one step, every cell against the oracle."""
    cfg, f = W.spinodal(N=2048)
    got, ref, dist, st = run_both(S, cfg, f, 1)
    assert_parity(got, ref, what="2048^2")


def test_fp32_shifted_budget(S):
    """FP32 arithmetic on FP32 deviations from the rest state stays within the
    phi budget (relative L2 <= 1e-4) of the FP64 oracle on a bubble."""
    cfg, f = W.stationary_bubble(N=48, R=12.0, rho_ratio=10.0)
    cfg32 = dict(cfg, precision="fp32", phi_ref=0.5, p_ref=0.0)
    steps = 400
    with S.Solver(cfg32, **f) as s:
        s.step(steps)
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(steps)
    ref = o.macros()
    l2 = np.sqrt(((got["phi"] - ref["phi"]) ** 2).sum() / (ref["phi"] ** 2).sum())
    assert l2 <= 1e-4, l2
    assert np.abs(got["p"] - ref["p"]).max() <= 1e-2 * np.abs(ref["p"]).max() + 1e-6


def test_fp32_shifted_spinodal_full_size(S):
    """The bench workload in FP32: one step against the FP64 oracle."""
    cfg, f = W.spinodal(N=2048)
    with S.Solver(dict(cfg, precision="fp32"), **f) as s:
        s.step(1)
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(1)
    ref = o.macros()
    assert np.abs(got["phi"] - ref["phi"]).max() <= 1e-6
    l2 = np.sqrt(((got["phi"] - ref["phi"]) ** 2).sum() / (ref["phi"] ** 2).sum())
    assert l2 <= 1e-7, l2


def test_reduce_matches_oracle(S):
    cfg, f = W.random_state(30, 26, seed=9)
    with S.Solver(cfg, **f) as s:
        o = Oracle(cfg, **f)
        for n in (0, 3, 4):
            s.step(n)
            o.step(n)
            g = s.reduce()
            r = o.reduce()
            assert g[0] == pytest.approx(r[0], rel=1e-13)
            assert g[1] == pytest.approx(r[1], rel=1e-6, abs=1e-20)
            assert g[2] == pytest.approx(r[2], rel=1e-6, abs=1e-20)
            assert g[3] == pytest.approx(r[3], rel=1e-9)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_checkpoint_restart_bit_identical(S, precision):
    cfg, f = W.random_state(35, 21, seed=4, bc_y="wall")
    cfg["precision"] = precision
    with S.Solver(cfg, **f) as a:
        a.step(5)
        ck = a.get_state()
        a.step(7)
        want = a.macros()
        assert a.step_count == 12
    with S.Solver(cfg, **f) as b:
        b.set_state(ck)
        assert b.step_count == 5
        b.step(7)
        got = b.macros()
    for k in want:
        assert np.array_equal(want[k], got[k]), k


def test_nonphysical_state_reported(S):
    """phi below -1/999 at density ratio 1000 gives rho <= 0: the step records
    it in the device status word and the next synchronising call reports it."""
    cfg, f = W.spinodal(N=32)
    f["phi0"] = np.full((32, 32), -0.01)
    with S.Solver(cfg, **f) as s:
        s.step(1)
        with pytest.raises(S.DugksError) as e:
            s.sync()
        assert e.value.code == -5


def test_workspace_options_agree(S):
    """Library-allocated and torch-allocated workspaces give identical results."""
    cfg, f = W.random_state(21, 19, seed=2)
    out = []
    for ws in ("torch", "library"):
        with S.Solver(cfg, workspace=ws, **f) as s:
            s.step(4)
            out.append(s.macros())
    for k in out[0]:
        assert np.array_equal(out[0][k], out[1][k])


def test_zero_steps_is_identity(S):
    cfg, f = W.random_state(12, 11, seed=8)
    with S.Solver(cfg, **f) as s:
        a = s.macros()
        s.step(0)
        b = s.macros()
    for k in a:
        assert np.array_equal(a[k], b[k])


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_every_tile_shape(S, precision):
    """Each compiled tile shape of the step kernel against the oracle: periodic
    and walled grids with interior (TMA-staged) and ragged edge tiles, and the
    Allen-Cahn-only model."""
    cases = [W.random_state(150, 70, seed=21), W.random_state(37, 29, seed=22, bc_y="wall"),
             W.smoothed_deformation(L=48, U=0.04)]
    for k, shape in enumerate(S.tile_shapes(precision), start=1):
        for cfg, f in cases:
            c = dict(cfg, precision=precision, tile_shape=k)
            if precision == "fp32":
                c.setdefault("phi_ref", 0.5)
            with S.Solver(c, **f) as s:
                s.step(6)
                got = s.macros()
                dist = s.distributions() if precision == "fp64" else None
            o = Oracle(cfg, **f)
            o.step(6)
            ref = o.macros()
            what = "%s tile %dx%d %dx%d" % (precision, shape[0], shape[1], cfg["nx"], cfg["ny"])
            if precision == "fp64":
                assert_parity(got, ref, dist, o.state(), what=what)
            else:
                assert np.abs(got["phi"] - ref["phi"]).max() <= 2e-5, what
                assert np.abs(got["ux"] - ref["ux"]).max() <= 1e-7, what
                assert np.abs(got["p"] - ref["p"]).max() <= 1e-5, what


def test_autotune_picks_a_measured_shape(S):
    cfg, f = W.layered_poiseuille(ny=256, nx=4, mu_ratio=100.0)
    cfg = dict(cfg, precision="fp32", phi_ref=0.5)
    best, ms = S.autotune(cfg, **f, trial_steps=5)
    assert len(ms) == len(S.tile_shapes("fp32"))
    assert all(m > 0 for m in ms)
    assert 1 <= best <= len(ms) and ms[best - 1] == min(ms)


@pytest.mark.parametrize("nx,ny,steps,bc_y", [(150, 70, 6, "periodic"), (37, 29, 9, "periodic"), (5, 7, 3, "periodic"),
                                              (150, 70, 6, "wall"), (37, 29, 9, "wall"), (5, 7, 3, "wall"),
                                              (40, 3, 4, "wall")])
def test_upwind_reconstruction_fp64(S, nx, ny, steps, bc_y):
    """The upwind reconstruction (van Leer slopes) against the oracle, coupled
    model, with interior (TMA-staged) tiles, ragged tiles and a grid smaller
    than the halo; periodic and walled (R17: one-sided slopes next to a wall,
    the wall face from the adjacent cell's profile), down to three rows."""
    cfg, f = W.random_state(nx, ny, seed=nx * 7 + ny, bc_y=bc_y)
    cfg["recon"] = "upwind"
    got, ref, dist, st = run_both(S, cfg, f, steps)
    assert_parity(got, ref, dist, st, what="upwind %dx%d" % (nx, ny))


@pytest.mark.parametrize("bc_y", ["periodic", "wall"])
def test_upwind_allen_cahn_fp64_and_fp32(S, bc_y):
    cfg, f = W.smoothed_deformation(L=64, U=0.04)
    cfg.update(recon="upwind", bc_y=bc_y)
    got, ref, dist, st = run_both(S, cfg, f, 40)
    assert_parity(got, ref, dist, st, what="upwind A-C")
    with S.Solver(dict(cfg, precision="fp32"), **f) as s:
        s.step(40)
        g32 = s.macros()
    assert np.abs(g32["phi"] - ref["phi"]).max() <= 2e-5


@pytest.mark.parametrize("bc_y", ["periodic", "wall"])
def test_upwind_coupled_fp32(S, bc_y):
    """The FP32-shifted coupled kernel with the upwind reconstruction (the
    kernel of the bench's upwind leg) against the FP64 oracle, interior and
    edge tiles, periodic and walled, within FP32 round-off after a few steps."""
    cfg, f = W.random_state(150, 70, seed=29, bc_y=bc_y)
    cfg["recon"] = "upwind"
    with S.Solver(dict(cfg, precision="fp32", phi_ref=0.5), **f) as s:
        s.step(6)
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(6)
    ref = o.macros()
    assert np.abs(got["phi"] - ref["phi"]).max() <= 2e-5
    assert np.abs(got["ux"] - ref["ux"]).max() <= 1e-7
    assert np.abs(got["p"] - ref["p"]).max() <= 1e-5


def test_bounded_wait_times_out_and_context_survives(S):
    """Failure detection without a fault: a kernel waits, with the step
    kernel's wait function and poll limit, on a barrier nothing completes; it
    gives up, the host reads DUGKS_ERR_TIMEOUT, and the GPU keeps working."""
    import time

    t0 = time.perf_counter()
    assert S.check_bounded_wait() == -6
    assert time.perf_counter() - t0 < 5.0
    assert S.check_bounded_wait(max_polls=10) == -6
    cfg, f = W.random_state(20, 18, seed=3)
    got, ref, dist, st = run_both(S, cfg, f, 3)
    assert_parity(got, ref, dist, st, what="after the timeout check")


def _sampled_case(L=40, seed=1):
    cfg, f = W.zalesak_disk(L=L, R=15.0, slot=4.0, U=0.04)
    r = np.random.default_rng(seed)
    ux, uy = 0.02 * r.standard_normal((L, L)), 0.02 * r.standard_normal((L, L))
    return dict(cfg, velocity_field="sampled"), dict(f, ux0=ux, uy0=uy), ux, uy


@pytest.mark.parametrize("bc_y", ["periodic", "wall"])
def test_sampled_velocity_field_fp64(S, bc_y):
    """Sampled velocity (dugks_set_velocity_field): the field given at
    creation, then replaced mid-run by another one with face normals."""
    cfg, f, ux, uy = _sampled_case()
    cfg["bc_y"] = bc_y
    r = np.random.default_rng(7)
    ux2, uy2 = 0.02 * r.standard_normal(ux.shape), 0.02 * r.standard_normal(ux.shape)
    uxf, uyf = 0.02 * r.standard_normal(ux.shape), 0.02 * r.standard_normal(ux.shape)
    with S.Solver(cfg, **f) as s:
        s.step(5)
        s.set_velocity_field(ux2, uy2, uxf, uyf)
        s.step(6)
        got, dist = s.macros(), s.distributions()
    o = Oracle(cfg, **f)
    o.step(5)
    o.set_velocity(ux2, uy2, uxf, uyf)
    o.step(6)
    assert_parity(got, o.macros(), dist, o.state(), what="sampled " + bc_y)


def test_sampled_velocity_field_fp32_and_errors(S):
    """FP32 with a smooth sampled field (Eq. 42's shear at the cell centres;
    grid-scale random fields amplify FP32 round-off at a sharp step)."""
    import math

    L, U = 64, 0.04
    cfg, f = W.shear_elongation(L=L, U=U)
    c = np.arange(L) + 0.5
    X, Y = np.meshgrid(c, c)
    ux = U * math.pi * np.sin(math.pi * X / L) * np.cos(math.pi * Y / L)
    uy = -U * math.pi * np.cos(math.pi * X / L) * np.sin(math.pi * Y / L)
    cfg, f = dict(cfg, velocity_field="sampled"), dict(f, ux0=ux, uy0=uy)
    with S.Solver(dict(cfg, precision="fp32", phi_ref=0.5), **f) as s:
        s.step(8)
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(8)
    assert np.abs(got["phi"] - o.macros()["phi"]).max() <= 2e-5
    c2, f2 = W.translation_circle(L=16, R=4.0, U=0.02)
    with S.Solver(c2, **f2) as s:
        with pytest.raises(S.DugksError) as e:
            s.set_velocity_field(np.zeros((16, 16)), np.zeros((16, 16)))
        assert e.value.code == -7


def _laplace_jump(O_grad_lap, m, N, R, sigma, wd):
    """Jump of the thermodynamic pressure (Sec. IV.A) between the bubble's
    interior (r < R - 3) and the far liquid (r > R + 6), each averaged: the
    bulk values Laplace's law is about.  (Single cells are not used: inside a
    small bubble phi settles near 0.013, where the sharpening term of the
    conservative Allen-Cahn model makes the pointwise field depend on
    round-off over thousands of steps, in any precision.)"""
    phi = m["phi"]
    beta, kappa = 12 * sigma / wd, 1.5 * sigma * wd
    gx, gy, lp = O_grad_lap(phi)
    eps = beta * phi ** 2 * (phi - 1) ** 2
    deps = beta * (2 * phi * (phi - 1) ** 2 + 2 * phi ** 2 * (phi - 1))
    P = phi * deps - eps - kappa * phi * lp + 0.5 * kappa * (gx ** 2 + gy ** 2) + m["p"]
    c = np.arange(N) + 0.5
    X, Y = np.meshgrid(c, c)
    r = np.hypot(X - N / 2, Y - N / 2)
    return P[r < R - 3].mean() - P[r > R + 6].mean()


@pytest.mark.parametrize("rho_ratio", [1.0, 10.0])
def test_fp32_laplace_jump_within_one_percent(S, rho_ratio):
    """FP32-shifted budget: the Laplace pressure jump of a stationary bubble
    after 4000 steps within 1 % of the FP64 oracle's (and of sigma / R)."""
    from oracle import oracle as O

    N, R, sigma, wd = 32, 8.0, 0.01, 4.0
    cfg, f = W.stationary_bubble(N=N, R=R, rho_ratio=rho_ratio, sigma=sigma, width=wd)
    with S.Solver(dict(cfg, precision="fp32", phi_ref=0.5), **f) as s:
        s.step(4000)
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(4000)
    ref = o.macros()
    d32 = _laplace_jump(O.grad_lap, got, N, R, sigma, wd)
    d64 = _laplace_jump(O.grad_lap, ref, N, R, sigma, wd)
    assert abs(d32 - d64) <= 0.01 * abs(d64), (d32, d64)
    assert abs(d64 / (sigma / R) - 1.0) < 0.1


def test_fp32_poiseuille_profile_within_half_percent(S):
    """FP32-shifted budget: the layered Poiseuille profile (viscosity ratio
    100, the serving mix's channel) within 0.5 % of the FP64 oracle's."""
    cfg, f = W.layered_poiseuille(ny=64, nx=4, mu_ratio=100.0, start_from_analytic=True)
    with S.Solver(dict(cfg, precision="fp32", phi_ref=0.5), **f) as s:
        s.step(6000)
        u32 = s.macros()["ux"][:, 0]
    o = Oracle(cfg, **f)
    o.step(6000)
    u64 = o.macros()["ux"][:, 0]
    assert np.abs(u32 - u64).max() <= 0.005 * np.abs(u64).max(), np.abs(u32 - u64).max() / np.abs(u64).max()


def test_fp32_phi_mass_does_not_drift(S):
    """FP32-shifted storage conserves the phi mass to round-off (relative
    drift below 1e-6 in 4000 steps, against 1.6e-4 when the rounded
    coefficients biased every step): the rest direction of psi-bar-plus
    closes the f moments on phi', the FP32 weights sum to exactly 1 and the
    flux difference of each axis is formed before it is added."""
    cfg, f = W.stationary_bubble(N=32, R=8.0, rho_ratio=1.0, sigma=0.01, width=4.0)
    m0 = f["phi0"].sum()
    for ref in (0.5, 0.0):
        with S.Solver(dict(cfg, precision="fp32", phi_ref=ref), **f) as s:
            s.step(4000)
            m = s.macros()["phi"].sum()
        assert abs(m - m0) < 1e-6 * m0, (ref, (m - m0) / m0)


@pytest.mark.parametrize("precision,N", [("fp64", 16384), ("fp32", 16384)])
def test_maximum_size_by_periodic_tiling(S, precision, N):
    """The largest grids: a 16384^2 box (268M cells; the FP64 workspace is
    86 GB and plane offsets pass 2^32 elements) filled with a 64^2 periodic
    pattern.  One step of the tiled box must equal one step of the 64^2 box
    on every cell, so the oracle's 64^2 result checks all 268M cells."""
    n = 64
    cfg, f = W.random_state(n, n, seed=64)
    ref_o = Oracle(cfg, **f)
    ref_o.step(2)
    ref = ref_o.macros()
    reps = N // n
    big = {k: (None if v is None else np.tile(v, (reps, reps))) for k, v in f.items()}
    with S.Solver(dict(cfg, nx=N, ny=N, precision=precision, phi_ref=0.5), workspace="library", **big) as s:
        s.step(2)
        got = s.macros()
    del big
    tol = {"fp64": dict(phi=1e-10, p=1e-10, ux=1e-10, uy=1e-10),
           "fp32": dict(phi=2e-5, p=1e-5, ux=1e-7, uy=1e-7)}[precision]
    for k in ("phi", "p", "ux", "uy"):
        g = got[k].reshape(reps, n, reps, n)
        err = np.abs(g - ref[k][None, :, None, :]).max()
        assert err <= tol[k], (precision, k, err)


def _rti_positions(phi, L):
    """Bubble front (light fluid rising at x = 0) and spike tip (heavy fluid
    falling at x = L/2), as (y - 2L) / L of the phi = 1/2 crossing."""
    def up(c):          # first crossing from the bottom
        j = int(np.argmax(c >= 0.5))
        return j - 1 + (0.5 - c[j - 1]) / (c[j] - c[j - 1]) + 0.5
    def down(c):        # first crossing from the top
        j = len(c) - 1 - int(np.argmax(c[::-1] < 0.5))
        return j + (0.5 - c[j]) / (c[j + 1] - c[j]) + 0.5
    return (up(phi[:, 0]) - 2 * L) / L, (down(phi[:, L // 2]) - 2 * L) / L


def test_rayleigh_taylor_full_size_fp32_tracks_fp64(S):
    """Sec. IV.D at the paper's size (256 x 1024, At = 0.5, Re = 3000, walls,
    64,000 steps to t* = 2.5): the bubble rises and the spike falls
    monotonically, and the FP32-shifted run tracks the FP64 run's positions to
    1e-3 L; FP64 keeps the phi mass to 1e-10."""
    L = 256
    cfg, f = W.rayleigh_taylor(L=L)
    T = L / 0.04
    runs = {}
    for prec in ("fp64", "fp32"):
        c = dict(cfg, precision=prec, phi_ref=0.5) if prec == "fp32" else dict(cfg)
        rows, done = [], 0
        with S.Solver(c, **f) as s:
            for ts in (0.5, 1.0, 1.5, 2.0, 2.5):
                n = int(round(ts * T / cfg["cfl"]))
                s.step(n - done)
                done = n
                m = s.macros()
                rows.append(_rti_positions(m["phi"], L) + (m["phi"].sum(),))
        runs[prec] = rows
    b64 = [r[0] for r in runs["fp64"]]
    s64 = [r[1] for r in runs["fp64"]]
    assert all(b2 > b1 for b1, b2 in zip(b64, b64[1:])) and b64[0] > 0.1
    assert all(s2 < s1 for s1, s2 in zip(s64, s64[1:])) and s64[0] < -0.1
    for r32, r64 in zip(runs["fp32"], runs["fp64"]):
        assert abs(r32[0] - r64[0]) < 1e-3 and abs(r32[1] - r64[1]) < 1e-3, (r32, r64)
    m0 = f["phi0"].sum()
    assert abs(runs["fp64"][-1][2] - m0) < 1e-10 * m0
