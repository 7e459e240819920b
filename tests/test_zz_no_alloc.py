"""dugks_reduce_fields_static, the allocation-free reduction entry point.

It exists for callers that cannot allocate device memory where they check
convergence (for example while recording a CUDA graph, or in a serving loop
whose memory is planned up front).  Here it is called through the C ABI on the
macro fields a solver wrote to device memory, and its results are compared
with those of dugks_reduce on the same solver, on two calls in a row (the
second one against a snapshot, so the residuals are exercised too).  This
file is collected last so that a failure here cannot hide another test's.
"""
import ctypes

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


def device_macros(s, torch):
    out = {k: torch.empty((s.ny, s.nx), dtype=torch.float64, device="cuda") for k in ("phi", "p", "ux", "uy")}
    s.macros_device(out)
    return out


def static_reduce(S, torch, m, snap):
    out = torch.full((4,), float("nan"), dtype=torch.float64, device="cuda")
    S.reduce_fields_static(m["phi"], m["ux"], m["uy"], out, snap=snap)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def test_static_reduce_matches_dugks_reduce(S):
    import torch

    cfg, f = W.random_state(40, 30, seed=21)
    with S.Solver(cfg, **f) as s:
        s.step(5)
        m1 = device_macros(s, torch)
        ref1 = np.array(s.reduce())
        got1 = static_reduce(S, torch, m1, None)
        snap = torch.cat([m1["phi"].reshape(-1), m1["ux"].reshape(-1), m1["uy"].reshape(-1)])

        s.step(7)
        m2 = device_macros(s, torch)
        ref2 = np.array(s.reduce())
        got2 = static_reduce(S, torch, m2, snap)

    for got, ref in ((got1, ref1), (got2, ref2)):
        assert got[0] == pytest.approx(ref[0], rel=1e-13)       # phi mass
        assert got[1] == pytest.approx(ref[1], rel=1e-6, abs=1e-20)
        assert got[2] == pytest.approx(ref[2], rel=1e-6, abs=1e-20)
        assert got[3] == pytest.approx(ref[3], rel=1e-9)        # max |u|
    assert got1[1] == 1.0 and got1[2] == 1.0                    # no snapshot yet
    assert got2[1] > 0.0 and got2[2] > 0.0                      # residuals against the snapshot
    assert got2[1] != 1.0 and got2[2] != 1.0


def test_static_reduce_rejects_oversize_and_null(S):
    import torch

    x = torch.zeros(8, dtype=torch.float64, device="cuda")
    out = torch.zeros(4, dtype=torch.float64, device="cuda")
    dp = ctypes.POINTER(ctypes.c_double)
    p = ctypes.cast(x.data_ptr(), dp)
    po = ctypes.cast(out.data_ptr(), dp)
    L = S.lib()
    assert L.dugks_reduce_fields_static(p, p, p, None, S.STATIC_REDUCE_MAX_CELLS + 1, po, None) == -1
    assert L.dugks_reduce_fields_static(p, p, p, None, 0, po, None) == -1
    assert L.dugks_reduce_fields_static(None, p, p, None, 8, po, None) == -1
    assert L.dugks_reduce_fields_static(p, p, p, None, 8, None, None) == -1
    with pytest.raises(ValueError):
        big = torch.zeros(S.STATIC_REDUCE_MAX_CELLS + 1, dtype=torch.float64, device="cuda")
        S.reduce_fields_static(big, big, big, out)
