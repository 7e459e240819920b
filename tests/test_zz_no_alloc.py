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


def _numpy_reduce(phi, ux, uy, snap):
    """The four outputs in FP64 on the host, from their definitions."""
    u2 = ux * ux + uy * uy
    out = [phi.sum(), 1.0, 1.0, np.sqrt(u2).max()]
    if snap is not None:
        n = phi.size
        sp, sx, sy = snap[:n], snap[n:2 * n], snap[2 * n:]
        out[1] = ((phi - sp) ** 2).sum() / (phi ** 2).sum()
        out[2] = ((ux - sx) ** 2 + (uy - sy) ** 2).sum() / u2.sum()
    return np.array(out)


@pytest.mark.parametrize("n", [300 * 217, 5 * 4096 + 123, 16777216 - 1000, 16777216])
def test_static_reduce_across_blocks(S, n):
    """Fields spanning many 4096-cell blocks, ending in a partly filled block
    (300 x 217 = 15 blocks + 3,660 cells; 5 blocks + 123), and the largest
    sizes, whose last block is the last record of the scratch array (partly
    filled, and full at n = DUGKS_STATIC_REDUCE_MAX_CELLS): all four outputs,
    with and without a snapshot, against an FP64 reduction on the host, on two
    calls in a row."""
    import torch

    assert n <= S.STATIC_REDUCE_MAX_CELLS
    g = torch.Generator(device="cuda").manual_seed(n % 1000003)
    phi = torch.rand(n, dtype=torch.float64, device="cuda", generator=g)
    ux = 1e-3 * (torch.rand(n, dtype=torch.float64, device="cuda", generator=g) - 0.5)
    uy = 1e-3 * (torch.rand(n, dtype=torch.float64, device="cuda", generator=g) - 0.5)
    snap = torch.cat([phi + 1e-6 * torch.rand(n, dtype=torch.float64, device="cuda", generator=g),
                      ux * 0.9, uy * 1.1])
    h = [t.cpu().numpy() for t in (phi, ux, uy, snap)]
    for sn, hs in ((None, None), (snap, h[3])):
        ref = _numpy_reduce(h[0], h[1], h[2], hs)
        for _ in range(2):
            got = static_reduce(S, torch, {"phi": phi, "ux": ux, "uy": uy}, sn)
            np.testing.assert_allclose(got[:3], ref[:3], rtol=1e-11, atol=0.0)
            # max |u|: the same cell, its sqrt(ux^2 + uy^2) rounded once more
            # or less where the device contracts a multiply-add
            assert got[3] == pytest.approx(ref[3], rel=1e-15)


def test_static_reduce_rejects_mismatched_tensors(S):
    """The binding refuses arguments that would make the kernel read or write
    past a tensor: wrong dtype, a short ux or uy, a snapshot of n instead of
    3n elements, a 3-element out, or a non-contiguous field."""
    import torch

    n = 64
    f = lambda k, dt=torch.float64: torch.zeros(k, dtype=dt, device="cuda")
    out = f(4)
    bad = [
        (f(n, torch.float32), f(n), f(n), out, None),
        (f(n), f(n - 1), f(n), out, None),
        (f(n), f(n), f(n + 1), out, None),
        (f(n), f(n), f(n), out, f(n)),
        (f(n), f(n), f(n), f(3), None),
        (torch.zeros(n, 2, dtype=torch.float64, device="cuda")[:, 0], f(n), f(n), out, None),
    ]
    for args in bad:
        with pytest.raises(ValueError):
            S.reduce_fields_static(*args[:4], snap=args[4])
