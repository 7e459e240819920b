"""The bounds-checked build (a stand-in for compute-sanitizer, which this GPU
pool does not offer): every step-kernel index is checked before its access
and a violation is reported as DUGKS_ERR_BOUNDS instead of being made.  Tiny,
one-tile, two-tile, ragged and walled grids, the upwind and Allen-Cahn
variants and every tile shape run through it against the oracle, in a child
process that loads the checked library."""
import json
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r'''
import json, sys
import numpy as np
sys.path.insert(0, ROOT)
from paper_1810_07802_gb300 import solver as S, workloads as W
from oracle.oracle import Oracle

def case(cfg, f, steps):
    with S.Solver(cfg, **f) as s:
        s.step(steps)
        s.sync()          # raises DugksError(-8) if an index was out of range
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(steps)
    ref = o.macros()
    return max(float(np.abs(got[k] - ref[k]).max()) for k in ref)

errs = {}
for nx, ny in ((8, 8), (9, 7), (32, 8), (64, 8), (3, 3), (150, 70)):
    cfg, f = W.random_state(nx, ny, seed=nx + ny)
    errs["periodic %dx%d" % (nx, ny)] = case(cfg, f, 4)
cfg, f = W.random_state(37, 29, seed=3, bc_y="wall")
errs["walls 37x29"] = case(cfg, f, 4)
cfg, f = W.random_state(131, 53, seed=4, bc_y="wall")
errs["walls 131x53"] = case(cfg, f, 3)
cfg, f = W.random_state(37, 29, seed=5)
errs["upwind 37x29"] = case(dict(cfg, recon="upwind"), f, 4)
cfg, f = W.random_state(150, 70, seed=6)
errs["upwind 150x70"] = case(dict(cfg, recon="upwind"), f, 3)
cfg, f = W.random_state(37, 29, seed=7, bc_y="wall")
errs["upwind walls 37x29"] = case(dict(cfg, recon="upwind"), f, 4)
cfg, f = W.random_state(131, 53, seed=8, bc_y="wall")
errs["upwind walls 131x53"] = case(dict(cfg, recon="upwind"), f, 3)
cfg, f = W.smoothed_deformation(L=40, U=0.04)
errs["A-C deformation"] = case(cfg, f, 6)
for k in range(1, len(S.tile_shapes("fp64")) + 1):
    cfg, f = W.random_state(37, 29, seed=10 + k)
    errs["tile %d" % k] = case(dict(cfg, tile_shape=k), f, 3)
# FP32 coupled periodic on the default tile shape: checked indices, FP32
# round-off of the FP64 oracle
for nx, ny in ((150, 70), (37, 29), (8, 8), (64, 24)):
    cfg, f = W.random_state(nx, ny, seed=40 + nx)
    c = dict(cfg, precision="fp32", phi_ref=0.5)
    with S.Solver(c, **f) as s:
        s.step(4)
        got = s.macros()
    o = Oracle(cfg, **f)
    o.step(4)
    ref = o.macros()
    errs["fp32 %dx%d" % (nx, ny)] = max(float(np.abs(got[k] - ref[k]).max()) / tol
                                        for k, tol in (("phi", 2e-5), ("ux", 1e-7), ("uy", 1e-7), ("p", 1e-5))) * 1e-10
print(json.dumps(errs))
'''


def test_checked_build_finds_no_out_of_range_index_and_keeps_parity():
    from paper_1810_07802_gb300 import build

    path = build.build(checked=True)
    env = dict(os.environ, DUGKS_LIBRARY=path)
    r = subprocess.run([sys.executable, "-c", CHILD.replace("ROOT", repr(ROOT))], env=env, capture_output=True,
                       text=True, timeout=900)
    assert r.returncode == 0, r.stderr[-3000:]
    errs = json.loads(r.stdout.strip().splitlines()[-1])
    for name, err in errs.items():
        assert err <= 1e-10, (name, err)
