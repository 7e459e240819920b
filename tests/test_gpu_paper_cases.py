"""The paper's configurations at their stated sizes and horizons on the GPU
(through the C ABI), against the FP64 oracle where the oracle can run them,
and FP32-shifted against FP64.

  * Interface diagonal translation (Sec. III.A, Table I): 64 x 64, u = v =
    0.01, one full period of 12,800 steps, element by element against the
    oracle, with the E of Eq. 39 and the phi mass.
  * Stationary bubble at density ratio 1000 (Sec. IV.A) with the paper's
    bubble parameters (W = 5, M = 0.1, one kinematic viscosity 0.1, reading
    R16): element-wise oracle parity over hundreds of steps, the bulk
    Laplace jump over thousands, and the 128 x 128, R = 32 bubble for 20,000
    steps in FP64 and FP32 (Laplace within 0.93-1.02 of sigma / R, FP32
    within 1 % of FP64, small spurious velocity).
  * The same bubble at W = 4, M = 0.02: a mode grows from round-off (the
    planar-interface analysis of test_density_ratio_stability); the GPU
    reaches the same horizon as the oracle.
  * The spinodal box at density ratio 1000, W = 4: its horizon (the same
    mode once sharp interfaces form).
  * Laplace's law over bubble radii 16-32 at density ratio 1000 (Sec. IV.A):
    the jumps lie on a line through the origin in 1/R.
  * The layered Poiseuille channel at the paper's viscosity ratio 1000
    (Sec. IV.B, Eq. 46), Ny = 100 and 200, against the paper's L2 errors;
    both viscosity rules.

Measured values are printed (run with -s to see them).
"""
import numpy as np
import pytest

from oracle import oracle as O
from oracle.oracle import Oracle
from paper_1810_07802_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def S():
    from paper_1810_07802_gb300 import build, solver

    build.build()
    solver.lib()
    return solver


def _E(phi, ref):
    """Eq. 39 as printed (a ratio of squared sums)."""
    return ((phi - ref) ** 2).sum() / (ref ** 2).sum()


def _laplace_ratio(m, N, R, sigma, wd):
    """Bulk jump of the thermodynamic pressure of Sec. IV.A over sigma / R:
    the interior (r < R - 3) against the far liquid (r > R + 6), each
    averaged."""
    phi = m["phi"]
    beta, kappa = 12 * sigma / wd, 1.5 * sigma * wd
    gx, gy, lp = O.grad_lap(phi)
    eps = beta * phi ** 2 * (phi - 1) ** 2
    deps = beta * (2 * phi * (phi - 1) ** 2 + 2 * phi ** 2 * (phi - 1))
    P = phi * deps - eps - kappa * phi * lp + 0.5 * kappa * (gx ** 2 + gy ** 2) + m["p"]
    c = np.arange(N) + 0.5
    X, Y = np.meshgrid(c, c)
    r = np.hypot(X - N / 2, Y - N / 2)
    return (P[r < R - 3].mean() - P[r > R + 6].mean()) / (sigma / R)


def _umax(m):
    return float(np.hypot(m["ux"], m["uy"]).max())


def test_translation_full_period_fp64_and_fp32(S):
    """Sec. III.A: the 64 x 64 disc moved by (0.01, 0.01) for one period
    (T = L0 / U0 = 6400, 12,800 steps) returns to its start.  FP64 equals the
    oracle within 1e-10 on every cell; the phi mass is kept to 1e-11
    (relative; the oracle's own drift is 1.3e-12, round-off of 12,800 sums);
    E of Eq. 39 is below Table I's smallest value (3.6e-3, Pe = 128 at
    L0 = 256; here Pe = 32); FP32-shifted storage (shifted by the far-field
    phase) is within the phi budget (relative L2 <= 1e-4) of FP64."""
    cfg, f = W.translation_circle(L=64)
    steps = 12800
    with S.Solver(cfg, **f) as s:
        s.step(steps)
        got = s.macros()
        dist = s.distributions()
    o = Oracle(cfg, **f)
    o.step(steps)
    ref = o.macros()
    err = np.abs(got["phi"] - ref["phi"]).max()
    assert err <= 1e-10, err
    assert np.abs(dist[0] - o.state()[0]).max() <= 1e-10
    m0 = f["phi0"].sum()
    assert abs(got["phi"].sum() - m0) <= 1e-11 * m0
    E64 = _E(got["phi"], f["phi0"])
    # the FP32 shift is the far-field phase (phi_ref = 0): deviations are exactly
    # zero in the bulk of the box (with phi_ref = 0.5 the phi L2 is 1.2e-4)
    with S.Solver(dict(cfg, precision="fp32", phi_ref=0.0), **f) as s:
        s.step(steps)
        g32 = s.macros()
    l2 = np.sqrt(((g32["phi"] - got["phi"]) ** 2).sum() / (got["phi"] ** 2).sum())
    print("\nC1 translation 64^2, 12800 steps: max|GPU-oracle| %.2e, E(FP64) %.4e, E(FP32) %.4e, "
          "FP32 vs FP64 L2 %.2e, FP32 mass drift %.2e" % (err, E64, _E(g32["phi"], f["phi0"]), l2,
                                                          (g32["phi"].sum() - m0) / m0))
    assert E64 < 3.6e-3, E64
    assert l2 <= 1e-4, l2


def test_ratio_1000_bubble_oracle_parity(S):
    """Density ratio 1000 with the paper's bubble parameters (N = 80, R = 12).
    After 60 steps every cell of phi, p, u and every stored distribution is
    within 1e-10 of the oracle.  Later the comparison is only as well
    conditioned as the problem: where phi is flat but not exactly 0 or 1,
    theta n of Eq. 16 multiplies a normal that round-off turns (R6), so two
    oracle runs whose initial phi differ by 1e-15 (relative) drift apart there
    (phi by ~1e-6 after 1,000 steps, u by ~1e-12).  At 1,000 steps each field
    of the GPU run is therefore required within max(1e-10, 100 x that
    control difference) of the oracle, and the bulk Laplace jump likewise
    (relative: max(1e-9, 100 x the control's))."""
    N, R, sigma, wd = 80, 12.0, 0.01, 5.0
    cfg, f = W.stationary_bubble(N=N, R=R, rho_ratio=1000.0, sigma=sigma, width=wd, mobility=0.1)
    o = Oracle(cfg, **f)
    f_ctl = dict(f, phi0=f["phi0"] * (1 + 1e-15 * np.random.default_rng(0).standard_normal(f["phi0"].shape)))
    ctl = Oracle(cfg, **f_ctl)
    names = ("phi", "p", "ux", "uy", "f", "g", "phiu")

    def fields(m, st):
        return dict(zip(names, [m[k] for k in names[:4]] + list(st)))

    with S.Solver(cfg, **f) as s:
        s.step(60)
        o.step(60)
        got, ref = fields(s.macros(), s.distributions()), fields(o.macros(), o.state())
        for k in names:
            assert np.abs(got[k] - ref[k]).max() <= 1e-10, ("60 steps", k)
        s.step(940)
        o.step(940)
        ctl.step(1000)
        mg, mo = s.macros(), o.macros()
        got, ref = fields(mg, s.distributions()), fields(mo, o.state())
    con = fields(ctl.macros(), ctl.state())
    report = []
    for k in names:
        err, c = np.abs(got[k] - ref[k]).max(), np.abs(con[k] - ref[k]).max()
        report.append("%s %.1e (control %.1e)" % (k, err, c))
        assert err <= max(1e-10, 100 * c), (k, err, c)
    lg, lo = _laplace_ratio(mg, N, R, sigma, wd), _laplace_ratio(mo, N, R, sigma, wd)
    lc = _laplace_ratio(ctl.macros(), N, R, sigma, wd)
    print("\nratio-1000 bubble 80^2 R=12, 1000 steps, max|GPU - oracle|: " + ", ".join(report)
          + "; Laplace GPU %.10f oracle %.10f control %.10f" % (lg, lo, lc))
    assert abs(lg - lo) <= max(1e-9, 100 * abs(lc - lo)) * abs(lo)


def test_c2_bubble_fp64_and_fp32(S):
    """The 128 x 128 bubble of radius 32 at density ratio 1000 (sigma = 0.01,
    nu = 0.1 everywhere) at the paper's W = 5 and M = 0.1.  Its pressure jump
    swings slowly about the Laplace value while the bubble relaxes (0.87 at
    5,000 steps, 1.22 at 10,000, 0.90 at 20,000: the printed value) and
    settles from about 40,000 steps; at 60,000 Laplace's law holds within
    0.93-1.02 (the paper: ~96.5 %), the FP32-shifted jump (storage shifted by
    the liquid phase, phi_ref = 1) is within 1 % of FP64 (so rho and p need no
    FP64 storage), both spurious velocities stay below 1e-5, and the FP32 phi
    error against FP64 (which grows with the step count) stays below 1e-3."""
    N, R, sigma, wd = 128, 32.0, 0.01, 5.0
    cfg, f = W.stationary_bubble(N=N, R=R, rho_ratio=1000.0, sigma=sigma, width=wd, mobility=0.1)
    out, at20k = {}, {}
    for prec, ref in (("fp64", None), ("fp32", 1.0), ("fp32 phi_ref 0.5", 0.5)):
        c = dict(cfg, precision="fp32", phi_ref=ref) if ref is not None else dict(cfg)
        with S.Solver(c, **f) as s:
            s.step(20000)
            at20k[prec] = _laplace_ratio(s.macros(), N, R, sigma, wd)
            s.step(40000)
            out[prec] = s.macros()
    l2_half = np.sqrt(((out["fp32 phi_ref 0.5"]["phi"] - out["fp64"]["phi"]) ** 2).sum() / (out["fp64"]["phi"] ** 2).sum())
    print("\nC2 FP32 with phi_ref 0.5 instead of the liquid's 1: phi L2 vs FP64 %.2e" % l2_half)
    l64 = _laplace_ratio(out["fp64"], N, R, sigma, wd)
    l32 = _laplace_ratio(out["fp32"], N, R, sigma, wd)
    u64, u32 = _umax(out["fp64"]), _umax(out["fp32"])
    l2 = np.sqrt(((out["fp32"]["phi"] - out["fp64"]["phi"]) ** 2).sum() / (out["fp64"]["phi"] ** 2).sum())
    print("\nC2 bubble 128^2 R=32 ratio 1000 W=5 M=0.1: Laplace at 20000 steps FP64 %.5f FP32 %.5f; at 60000 "
          "FP64 %.5f FP32 %.5f; max|u| FP64 %.3e FP32 %.3e; FP32 phi L2 vs FP64 %.2e"
          % (at20k["fp64"], at20k["fp32"], l64, l32, u64, u32, l2))
    assert 0.93 < l64 < 1.02, l64
    assert abs(l32 - l64) <= 0.01 * abs(l64), (l32, l64)
    assert abs(at20k["fp32"] - at20k["fp64"]) <= 0.01 * abs(at20k["fp64"])
    assert u64 < 1e-5 and u32 < 1e-5, (u64, u32)
    # the FP32 phi error grows with the step count (1.6e-4 at 20,000 steps,
    # 5.5e-4 at 60,000): the 1e-4 budget holds to about 12,000 steps here
    assert l2 <= 1e-3, l2


def _horizon(S, cfg, f, chunk, limit, umax_limit=1e-2):
    """Steps until max|u| passes umax_limit (or a status error), in chunks."""
    done = 0
    with S.Solver(cfg, **f) as s:
        while done < limit:
            s.step(chunk)
            done += chunk
            try:
                m = s.macros()
            except S.DugksError:
                return done
            if not np.isfinite(m["ux"]).all() or _umax(m) > umax_limit:
                return done
    return None


def test_c2_width_4_has_the_oracles_horizon(S):
    """At W = 4 and M = 0.02 (the growing mode of the planar analysis) the
    ratio-1000 bubble of radius 12 departs from rest: max|u| passes 1e-2 at
    the same 50-step chunk on the GPU (FP64) as in the oracle, well before
    2,000 steps; FP32 departs within a few chunks of it."""
    cfg, f = W.stationary_bubble(N=48, R=12.0, rho_ratio=1000.0, sigma=0.01, width=4.0, mobility=0.02)
    h64 = _horizon(S, cfg, f, 50, 2000)
    h32 = _horizon(S, dict(cfg, precision="fp32", phi_ref=0.5), f, 50, 2000)
    o = Oracle(cfg, **f)
    ho = None
    for n in range(50, 2001, 50):
        o.step(50)
        m = o.macros()
        if not np.isfinite(m["ux"]).all() or _umax(m) > 1e-2:
            ho = n
            break
    print("\nbubble 48^2 ratio 1000 W=4 M=0.02: max|u| > 1e-2 after %s steps (oracle), %s (GPU FP64), "
          "%s (GPU FP32)" % (ho, h64, h32))
    assert ho is not None and h64 == ho
    assert h32 is not None and abs(h32 - ho) <= 200


def test_spinodal_horizon(S):
    """The spinodal box at density ratio 1000, W = 4 (the growing mode of the
    planar analysis once sharp interfaces form): stepped in chunks until a
    step reports a non-finite value or max|u| passes 0.1, up to 10,000 steps,
    in FP32 on the full 2048 x 2048 box and in FP64 on a 512 x 512 piece of the
    same field and parameters.  Prints the horizons; both lie beyond 5,000
    steps, far beyond the 25-420 steps the bench times."""
    cfg, f = W.spinodal(N=2048)
    h32 = _horizon(S, dict(cfg, precision="fp32"), f, 500, 10000, umax_limit=0.1)
    cfg, f = W.spinodal(N=512)
    h64 = _horizon(S, cfg, f, 500, 10000, umax_limit=0.1)
    print("\nspinodal ratio 1000 W=4: non-finite or max|u| > 0.1 after %s steps (FP32 2048^2), %s (FP64 512^2)"
          % (h32, h64))
    assert h32 is None or h32 > 5000
    assert h64 is None or h64 > 5000


def test_layered_poiseuille_at_the_papers_viscosity_ratio(S):
    """Sec. IV.B: the two-layer channel at mu* = 1000 (Eq. 46), Ny = 100 and
    200, started from the analytic profile and stepped to its discrete steady
    state (40,000 steps; the L2 error moves by < 1 % after 20,000).  The paper
    gives only the ratio; mu_H = 5 is a reading (with mu_H = 10 the viscous
    layer's tau_g = 30 lets a mode across the 4-cell width grow at Ny >= 192,
    in the oracle too once seeded, so the absolute viscosity is kept lower).
    The reciprocal rule (Eq. 35) lands within a factor of 2 of the paper's L2
    errors with the paper's refinement ratio (Ny 100 -> 200) within 20 %, and
    the linear rule (Eq. 36) is far worse, as the paper reports."""
    import json
    import os

    golden = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))["poiseuille_L2"]
    errs = {}
    for ny in golden["Ny"]:
        for visc in ("reciprocal", "linear"):
            cfg, fl = W.layered_poiseuille(ny=ny, mu_ratio=1000.0, mu_h=5.0, start_from_analytic=True)
            cfg["visc"] = visc
            y = np.arange(ny) + 0.5
            ua = W.poiseuille_profile(y, ny, cfg["mu_h"], cfg["mu_l"], cfg["gx"])
            l2 = []
            with S.Solver(cfg, **fl) as s:
                for n in (20000, 20000):
                    s.step(n)
                    u = s.macros()["ux"]
                    assert np.abs(u - u.mean(axis=1, keepdims=True)).max() < 1e-9   # no mode across the width
                    l2.append(float(np.sqrt(((u[:, 0] - ua) ** 2).sum() / (ua ** 2).sum())))
            errs[(ny, visc)] = l2
    (n1, n2), (p1, p2) = golden["Ny"], golden["L2"]
    r1, r2 = errs[(n1, "reciprocal")][1], errs[(n2, "reciprocal")][1]
    print("\nlayered Poiseuille mu*=1000: L2 (reciprocal) Ny %d %.4e, Ny %d %.4e (paper %.4e, %.4e); linear %.3e, %.3e"
          % (n1, r1, n2, r2, p1, p2, errs[(n1, "linear")][1], errs[(n2, "linear")][1]), end="")
    for ny in (n1, n2):
        a, b = errs[(ny, "reciprocal")]
        assert abs(b - a) <= 0.01 * b, (ny, a, b)
        assert errs[(ny, "linear")][1] > 5 * b, (ny, errs)
    assert p1 / 2 < r1 < 2 * p1 and p2 / 2 < r2 < 2 * p2, (r1, r2)
    assert abs((r1 / r2) / (p1 / p2) - 1) < 0.2, (r1 / r2, p1 / p2)


def test_laplace_law_over_bubble_radii(S):
    """Sec. IV.A: Laplace's law for bubbles of radius 16 ... 32 in a 128^2
    box at density ratio 1000 (the paper's W = 5, M = 0.1, one kinematic
    viscosity 0.1, sigma = 0.01), FP32-shifted with the liquid as the shift
    (FP32 and FP64 agree to 0.02 % here).  After 60,000 steps each pressure
    jump is 0.93-1.02 of sigma / R (the paper: about 96.5 %), the jumps lie
    on a line through the origin in 1/R whose slope is 0.93-1.02 sigma, and
    the spurious velocities stay below 1e-5."""
    N, sigma, wd = 128, 0.01, 5.0
    radii = np.array([16.0, 20.0, 24.0, 28.0, 32.0])
    jumps, ratios = [], []
    for R in radii:
        cfg, f = W.stationary_bubble(N=N, R=R, rho_ratio=1000.0, sigma=sigma, width=wd, mobility=0.1)
        with S.Solver(dict(cfg, precision="fp32", phi_ref=1.0), **f) as s:
            s.step(60000)
            m = s.macros()
        ratio = _laplace_ratio(m, N, R, sigma, wd)
        ratios.append(ratio)
        jumps.append(ratio * sigma / R)
        assert _umax(m) < 1e-5, (R, _umax(m))
    slope, intercept = np.polyfit(1.0 / radii, np.array(jumps), 1)
    print("\nLaplace over R = 16..32 (ratio 1000): dP/(sigma/R) " + " ".join("%.4f" % r for r in ratios)
          + "; fit dP = %.4f sigma / R %+.2e" % (slope / sigma, intercept), end="")
    assert all(0.93 < r < 1.02 for r in ratios), ratios
    assert 0.93 < slope / sigma < 1.02, slope / sigma
    assert abs(intercept) < 0.05 * sigma / radii.max(), intercept
