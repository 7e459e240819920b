"""The C-ABI library loads, exports every symbol include/dugks.h declares, and
rejects invalid problems before touching a GPU."""
import ctypes
import os
import re

import pytest

from paper_1810_07802_gb300 import build as gpu_build
from paper_1810_07802_gb300 import solver, workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    gpu_build.build()
    return solver.lib()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "dugks.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(dugks_[a-z_]+)\s*\(", text)))


def test_header_and_binding_agree():
    assert declared_functions() == sorted(solver.SIGNATURES)


def test_library_exports_every_declared_symbol(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_params_struct_size_matches_header():
    # 10 int32 fields, 15 doubles, 2 int32 (velocity field, reserved), 2 doubles,
    # 2 int32 (reconstruction, reserved); no padding
    assert ctypes.sizeof(solver.DugksParams) == 10 * 4 + 15 * 8 + 2 * 4 + 2 * 8 + 2 * 4


def test_workspace_bytes_and_validation(lib):
    cfg, _ = workloads.spinodal(N=64)
    ws64 = solver.workspace_bytes(dict(cfg, precision="fp64"))
    ws32 = solver.workspace_bytes(dict(cfg, precision="fp32"))
    assert ws64 > ws32 > 0
    # two ping-pong copies of 18 distributions and 2 history planes, 64-column pitch
    assert ws64 >= 2 * 20 * 64 * 64 * 8
    bad = [dict(cfg, nx=2), dict(cfg, ny=0), dict(cfg, cfl=0.0), dict(cfg, mobility=-1.0),
           dict(cfg, width=0.0), dict(cfg, rho_l=0.0), dict(cfg, mu_h=float("nan")), dict(cfg, sigma=-1.0)]
    for b in bad:
        assert solver.workspace_bytes(b) == 0, b
    p = solver.make_params(cfg)
    p.lattice = 8
    assert lib.dugks_workspace_bytes(ctypes.byref(p)) == 0


def test_create_rejects_invalid_without_gpu(lib):
    import numpy as np

    cfg, f = workloads.spinodal(N=16)
    h = ctypes.c_void_p()
    phi = np.ascontiguousarray(f["phi0"])
    dp = ctypes.POINTER(ctypes.c_double)
    p = solver.make_params(dict(cfg, nx=2))
    assert lib.dugks_create(ctypes.byref(p), phi.ctypes.data_as(dp), None, None, None, None, 0, None,
                            ctypes.byref(h)) == -1
    p = solver.make_params(dict(cfg, bc_x="wall"))
    assert lib.dugks_create(ctypes.byref(p), phi.ctypes.data_as(dp), None, None, None, None, 0, None,
                            ctypes.byref(h)) == -7
    p = solver.make_params(cfg)
    assert lib.dugks_create(ctypes.byref(p), None, None, None, None, None, 0, None, ctypes.byref(h)) == -1
    assert lib.dugks_step(None, 1) == -1
    assert lib.dugks_step_count(None) == -1
    assert lib.dugks_status_string(-4) == b"non-finite value produced by a step"


def test_tile_shapes_and_their_validation(lib):
    """The compiled step-kernel tile shapes (no device work) and the range
    check of params.tile_shape."""
    f32 = solver.tile_shapes("fp32")
    f64 = solver.tile_shapes("fp64")
    assert f32[0] == (32, 8) and f64[0] == (16, 8)
    for shapes in (f32, f64):
        assert len(set(shapes)) == len(shapes) >= 2
        for tx, ty in shapes:
            assert tx % 4 == 0 and tx * ty >= 128
    assert lib.dugks_tile_shapes(7, None, None, 0) == -1
    cfg, _ = workloads.spinodal(N=64)
    for prec, shapes in (("fp32", f32), ("fp64", f64)):
        for k in range(len(shapes) + 1):
            assert solver.workspace_bytes(dict(cfg, precision=prec, tile_shape=k)) > 0
        assert solver.workspace_bytes(dict(cfg, precision=prec, tile_shape=len(shapes) + 1)) == 0
        assert solver.workspace_bytes(dict(cfg, precision=prec, tile_shape=-1)) == 0


def test_upwind_limits_rejected_without_gpu(lib):
    """The upwind reconstruction is compiled for the default tile shape only:
    another shape is refused before any device work, as is an unknown
    reconstruction."""
    import numpy as np

    cfg, f = workloads.random_state(16, 12, seed=1)
    phi = np.ascontiguousarray(f["phi0"])
    dp = ctypes.POINTER(ctypes.c_double)
    h = ctypes.c_void_p()
    for bad in (dict(cfg, recon="upwind", tile_shape=2), dict(cfg, recon="upwind", bc_y="wall", tile_shape=3)):
        p = solver.make_params(bad)
        assert lib.dugks_create(ctypes.byref(p), phi.ctypes.data_as(dp), None, None, None, None, 0, None,
                                ctypes.byref(h)) == -7
    p = solver.make_params(cfg)
    p.recon = 2
    assert lib.dugks_workspace_bytes(ctypes.byref(p)) == 0


def test_batch_calls_reject_a_null_batch(lib):
    """The batch entry points check their handle before any device work."""
    assert lib.dugks_batch_set_persistent(None, 1) == -1
    assert lib.dugks_batch_step(None, 1) == -1
    assert lib.dugks_batch_size(None) == -1


def test_row_calls_reject_a_null_handle(lib):
    """The row copies and row reductions of the slab decomposition check
    their handle and buffers before any device work."""
    import numpy as np

    buf = np.zeros(6)
    p = buf.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
    had = ctypes.c_int32()
    assert lib.dugks_reduce_rows(None, 0, 1, p, ctypes.byref(had)) == -1
    assert lib.dugks_get_rows(None, 0, 1, buf.ctypes.data_as(ctypes.c_void_p), 0) == -1
    assert lib.dugks_set_rows(None, 0, 1, buf.ctypes.data_as(ctypes.c_void_p), 0) == -1
    assert lib.dugks_state_element_bytes(None) == 0


def test_status_strings_cover_every_code(lib):
    for code, name in solver.STATUS.items():
        text = lib.dugks_status_string(code).decode()
        assert text and text != "unknown status", (code, name)
    assert lib.dugks_status_string(-99).decode() == "unknown status"


def test_static_reduce_binding_rejects_host_tensors():
    """The binding of dugks_reduce_fields_static refuses, before any call into
    the library, arguments the kernel could not read safely: host tensors,
    float32 fields and objects that are not tensors."""
    import torch

    n = 16
    h = torch.zeros(n, dtype=torch.float64)
    out = torch.zeros(4, dtype=torch.float64)
    for args in ((h, h, h, out), (h.float(), h, h, out), (h.numpy(), h, h, out)):
        with pytest.raises(ValueError):
            solver.reduce_fields_static(*args)
