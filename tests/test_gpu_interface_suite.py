"""The interface-capturing suite of Sec. III at the paper's sizes on the GPU
(through the C ABI): every Peclet number of Tables I, III, V and VII in FP64,
and the first of each in FP32-shifted storage; every mobility of Tables II,
IV, VI and VIII in FP64.

  Table I    diagonal translation, L0 = 256, R = L0/4, M = 0.02, W = 4,
             T = L0/U0 (Sec. III.A)
  Table III  Zalesak's disk, L0 = 256, R = 100, slot 20, M = 0.02, W = 4,
             T = 2 L0/U0 (Sec. III.B)
  Table V    circle in a reversing shear, L0 = 256, R = L0/5 at (0.5, 0.3) L0,
             M = 0.01, W = 4, T = 2 L0/U0 (Sec. III.C)
  Table VII  circle in the smoothed deformation field, L0 = 512, R = L0/5,
             M = 0.02, W = 4, T = L0/U0 (Sec. III.D)
with U0 = Pe M / L0 and dt = 0.5.  E of Eq. 39 after one period is printed
beside the paper's value (run with -s).  The paper's values are context: the
slot proportions of Zalesak's disk and other details it does not print are
read (R12, R13).  The FP32-shifted error against FP64 after one period is
printed for the storage shifted by 0.5 and by the background phase (0).
"""
import json
import os

import numpy as np
import pytest

from paper_1810_07802_gb300 import workloads as W

pytestmark = pytest.mark.gpu

GOLDEN = json.load(open(os.path.join(os.path.dirname(__file__), "golden", "paper_values.json")))


@pytest.fixture(scope="module")
def S():
    from paper_1810_07802_gb300 import build, solver

    build.build()
    solver.lib()
    return solver


def _case(table, pe, M=None):
    """(cfg, fields, steps) of one row of a table: the Pe tables (I, III, V,
    VII) at their fixed mobility, the mobility tables (II, IV, VI, VIII) of the
    same problems at their fixed Pe with mobility M (U0 = Pe M / L0 either way)."""
    problem = {"I": "translation", "II": "translation", "III": "zalesak", "IV": "zalesak",
               "V": "shear", "VI": "shear", "VII": "deformation", "VIII": "deformation"}[table]
    L = 512 if problem == "deformation" else 256
    if M is None:
        M = 0.01 if problem == "shear" else 0.02
    U = pe * M / L
    if problem == "translation":
        cfg, f = W.translation_circle(L=L, R=L / 4.0, U=U, mobility=M, width=4.0)
        T = L / U
    elif problem == "zalesak":
        cfg, f = W.zalesak_disk(L=L, R=100.0, slot=20.0, U=U, mobility=M, width=4.0)
        T = 2 * L / U
    elif problem == "shear":
        cfg, f = W.shear_elongation(L=L, U=U, mobility=M, width=4.0)
        T = 2 * L / U
    else:
        cfg, f = W.smoothed_deformation(L=L, U=U, mobility=M, width=4.0)
        T = L / U
    return cfg, f, int(round(T / cfg["cfl"]))


def _E(phi, phi0):
    return float(((phi - phi0) ** 2).sum() / (phi0 ** 2).sum())


# FP32 phi error after one period (51,200-102,400 steps): a guard against
# regressions, not the 1e-4 budget (which holds to about 20,000 steps)
FP32_L2_BOUND = 1e-2

TABLES = {"I": "table_I_translation_E_phi_vs_Pe", "III": "table_III_zalesak_E_phi_vs_Pe",
          "V": "table_V_shear_E_phi_vs_Pe", "VII": "table_VII_deformation_E_phi_vs_Pe"}


@pytest.mark.parametrize("table", list(TABLES))
def test_interface_capturing_table(S, table):
    """Eq. 39 after one period at every Pe of the table.  The tables' values
    match the square root of Eq. 39 as printed (the L2 norm the text names)
    for Zalesak's disk and the reversing shear, within 10 %, where E itself
    is 8-40 times smaller; for the translation sqrt(E) is 1.2-1.6 times the
    paper's from Pe 256 up and 3.2 times at Pe 128, and for the smoothed
    deformation 3-4 times.  Required: sqrt(E) within a factor of 5 of the
    table, E growing with Pe in Table I from Pe 256 up (the advection-bound
    rows) and largest at the top Pe, phi mass conserved, and FP32 within the
    regression guard.  Why Pe 128 sits above Pe 256 is the next test."""
    rows = GOLDEN[TABLES[table]]
    out = []
    for k, (pe, paper) in enumerate(zip(rows["Pe"], rows["E"])):
        cfg, f, steps = _case(table, pe)
        with S.Solver(cfg, **f) as s:
            s.step(steps)
            phi64 = s.macros()["phi"]
        e64 = _E(phi64, f["phi0"])
        line = "Table %s Pe %g (%d^2, %d steps): FP64 E %.4e sqrt(E) %.4e, paper %.4e" % (
            table, pe, cfg["nx"], steps, e64, np.sqrt(e64), paper)
        l2s = {}
        if k == 0:
            for ref in (0.5, 0.0):
                with S.Solver(dict(cfg, precision="fp32", phi_ref=ref), **f) as s:
                    s.step(steps)
                    phi32 = s.macros()["phi"]
                l2s[ref] = float(np.sqrt(((phi32 - phi64) ** 2).sum() / (phi64 ** 2).sum()))
                if ref == 0.5:
                    line += "; FP32 E %.4e" % _E(phi32, f["phi0"])
            line += " (FP32 vs FP64 phi L2 %.2e with phi_ref 0.5, %.2e with 0)" % (l2s[0.5], l2s[0.0])
        print("\n" + line, end="")
        m0 = f["phi0"].sum()
        assert abs(phi64.sum() - m0) <= 1e-10 * m0, (table, pe)
        assert paper / 5 < np.sqrt(e64) < 5 * paper, (table, pe, e64, paper)
        if k == 0:
            assert l2s[0.5] <= FP32_L2_BOUND, (table, pe, l2s)
        out.append(e64)
    if table == "I":
        assert all(b > a for a, b in zip(out[1:], out[2:])), out
        assert out[-1] == max(out), out


def test_translation_low_pe_error_is_relaxation_at_rest(S):
    """Table I's rows share L0, R, M and W and differ in U0 and so in the
    period T = L0 / U0 = L0^2 / (Pe M): the lowest Pe runs longest (51,200
    steps at Pe 128, twice Pe 256's).  The same disc left at rest for the
    Pe-128 period (U0 = 0) already has most of the error the moving disc
    has: at low Pe, E measures how far the conservative Allen-Cahn dynamics
    (Eq. 1) move a curved interface in time M T, not the advection, and that
    part halves from Pe 128 to Pe 256 while the advection part grows."""
    pe = GOLDEN[TABLES["I"]]["Pe"][0]
    cfg, f, steps = _case("I", pe)
    with S.Solver(dict(cfg, u0x=0.0, u0y=0.0), **f) as s:
        s.step(steps)
        e_rest = _E(s.macros()["phi"], f["phi0"])
    with S.Solver(cfg, **f) as s:
        s.step(steps)
        e_moving = _E(s.macros()["phi"], f["phi0"])
    half_cfg = dict(cfg, u0x=0.0, u0y=0.0)
    with S.Solver(half_cfg, **f) as s:
        s.step(steps // 2)
        e_rest_half = _E(s.macros()["phi"], f["phi0"])
    print("\nTable I Pe %g period (%d steps): E at rest %.4e (half the period %.4e), moving %.4e"
          % (pe, steps, e_rest, e_rest_half, e_moving), end="")
    assert e_rest >= 0.5 * e_moving, (e_rest, e_moving)
    assert e_rest > e_rest_half, (e_rest, e_rest_half)


MOBILITY_TABLES = {"II": ("table_II_translation_E_phi_vs_M", 256), "IV": ("table_IV_zalesak_E_phi_vs_M", 256),
                   "VI": ("table_VI_shear_E_phi_vs_M", 256), "VIII": ("table_VIII_deformation_E_phi_vs_M", 512)}


@pytest.mark.parametrize("table", list(MOBILITY_TABLES))
def test_interface_capturing_mobility_table(S, table):
    """Eq. 39 after one period at every mobility of Tables II, IV, VI and VIII
    (fixed Pe, so U0 grows with M and the period shrinks), FP64.  Required:
    sqrt(E) within a factor of 5 of the table (R11), phi mass conserved, and
    the tables' trends in M: Table II falls and rises again, Table IV stays
    flat (within 2 %), Table VI ends above where it starts, Table VIII falls
    with M throughout (sqrt(E) measured: II 0.0078-0.0066-0.0074, IV
    0.115-0.116, VI 0.025-0.028, VIII 0.042-0.023)."""
    key, pe = MOBILITY_TABLES[table]
    rows = GOLDEN[key]
    out = []
    for M, paper in zip(rows["M"], rows["E"]):
        cfg, f, steps = _case(table, pe, M)
        with S.Solver(cfg, **f) as s:
            s.step(steps)
            phi = s.macros()["phi"]
        e = _E(phi, f["phi0"])
        out.append(e)
        print("\nTable %s M %g (%d^2, %d steps): FP64 E %.4e sqrt(E) %.4e, paper %.4e" % (
            table, M, cfg["nx"], steps, e, np.sqrt(e), paper), end="")
        m0 = f["phi0"].sum()
        assert abs(phi.sum() - m0) <= 1e-10 * m0, (table, M)
        assert paper / 5 < np.sqrt(e) < 5 * paper, (table, M, e, paper)
    if table == "II":
        assert out[1] < out[0] and out[-1] > min(out), out
    elif table == "IV":
        assert max(out) < 1.04 * min(out), out          # E: sqrt within 2 %
    elif table == "VI":
        assert out[-1] > out[0], out
    else:
        assert all(b < a for a, b in zip(out, out[1:])), out


def test_upwind_reconstruction_at_high_peclet(S):
    """Sec. III.A names an upwind scheme as the remedy for the central
    scheme's error growth at high Pe.  Table I's translation at Pe 512 and
    1024 (256^2, one period) with the upwind reconstruction (R14): phi stays
    within [0, 1] up to a small tolerance where the central scheme over- and
    undershoots (by 0.019 at Pe 1024), and E of Eq. 39 is below the central
    scheme's at both Pe, by more than 5x at Pe 1024 (measured: 1.67e-4 vs
    2.02e-4 at Pe 512, 8.4e-5 vs 1.33e-3 at Pe 1024; sqrt(E) 0.0091 against
    Table I's 0.0234 there)."""
    out = {}
    for pe in (512, 1024):
        for recon in ("central", "upwind"):
            cfg, f, steps = _case("I", pe)
            with S.Solver(dict(cfg, recon=recon), **f) as s:
                s.step(steps)
                phi = s.macros()["phi"]
            e = _E(phi, f["phi0"])
            out[(pe, recon)] = (e, float(phi.min()), float(phi.max()))
            print("\nTable I Pe %d %s: E %.4e sqrt(E) %.4e, phi in [%.4f, %.4f]"
                  % (pe, recon, e, np.sqrt(e), phi.min(), phi.max()), end="")
    for pe in (512, 1024):
        e, lo, hi = out[(pe, "upwind")]
        assert lo > -0.02 and hi < 1.02, (pe, lo, hi)
    assert out[(512, "upwind")][0] < out[(512, "central")][0], out
    assert 5 * out[(1024, "upwind")][0] < out[(1024, "central")][0], out
