"""Python binding of the C ABI in include/dugks.h (argument marshalling only).

Every step of the method runs in the CUDA library; this module converts a
workload dictionary (see `workloads`) into `dugks_params`, hands device memory
(a torch uint8 workspace) and the current torch stream to the library, and
copies host arrays in and out.  If the library is missing the import fails.
"""
import ctypes
import os

import numpy as np

from . import build as _build

_dp = ctypes.POINTER(ctypes.c_double)


class DugksParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int32), ("ny", ctypes.c_int32), ("lattice", ctypes.c_int32),
        ("model", ctypes.c_int32), ("precision", ctypes.c_int32),
        ("bc_x", ctypes.c_int32), ("bc_y", ctypes.c_int32),
        ("visc_interp", ctypes.c_int32), ("gravity_mode", ctypes.c_int32),
        ("tile_shape", ctypes.c_int32),
        ("cfl", ctypes.c_double), ("mobility", ctypes.c_double), ("width", ctypes.c_double),
        ("rho_h", ctypes.c_double), ("rho_l", ctypes.c_double),
        ("mu_h", ctypes.c_double), ("mu_l", ctypes.c_double), ("sigma", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double), ("rho_ref", ctypes.c_double),
        ("phi_ref", ctypes.c_double), ("p_ref", ctypes.c_double),
        ("u0x", ctypes.c_double), ("u0y", ctypes.c_double),
        ("velocity_field", ctypes.c_int32), ("reserved2", ctypes.c_int32),
        ("vel_u0", ctypes.c_double), ("vel_length", ctypes.c_double),
        ("recon", ctypes.c_int32), ("reserved3", ctypes.c_int32),
    ]


STATUS = {0: "DUGKS_OK", -1: "DUGKS_ERR_ARG", -2: "DUGKS_ERR_OOM", -3: "DUGKS_ERR_CUDA",
          -4: "DUGKS_ERR_NONFINITE", -5: "DUGKS_ERR_NONPHYSICAL", -6: "DUGKS_ERR_TIMEOUT",
          -7: "DUGKS_ERR_UNSUPPORTED", -8: "DUGKS_ERR_BOUNDS"}

# Every symbol include/dugks.h declares, with (restype, argtypes).
SIGNATURES = {
    "dugks_workspace_bytes": (ctypes.c_size_t, [ctypes.POINTER(DugksParams)]),
    "dugks_create": (ctypes.c_int, [ctypes.POINTER(DugksParams), _dp, _dp, _dp, _dp, ctypes.c_void_p,
                                    ctypes.c_size_t, ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "dugks_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "dugks_macros": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp, _dp, ctypes.c_int32]),
    "dugks_reduce": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp, _dp]),
    "dugks_get_distributions": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp]),
    "dugks_state_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "dugks_get_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "dugks_set_state": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_size_t]),
    "dugks_step_count": (ctypes.c_int64, [ctypes.c_void_p]),
    "dugks_state_element_bytes": (ctypes.c_size_t, [ctypes.c_void_p]),
    "dugks_get_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_int32]),
    "dugks_set_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32, ctypes.c_void_p,
                                      ctypes.c_int32]),
    "dugks_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "dugks_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "dugks_status_string": (ctypes.c_char_p, [ctypes.c_int]),
    "dugks_reduce_fields_static": (ctypes.c_int, [_dp, _dp, _dp, _dp, ctypes.c_int64, _dp, ctypes.c_void_p]),
    "dugks_batch_create": (ctypes.c_int, [ctypes.c_void_p, ctypes.POINTER(ctypes.c_void_p)]),
    "dugks_batch_add": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dugks_batch_remove": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_void_p]),
    "dugks_batch_size": (ctypes.c_int32, [ctypes.c_void_p]),
    "dugks_batch_step": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int64]),
    "dugks_batch_sync": (ctypes.c_int, [ctypes.c_void_p]),
    "dugks_batch_set_persistent": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32]),
    "dugks_check_batch_wait": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p]),
    "dugks_reduce_rows": (ctypes.c_int, [ctypes.c_void_p, ctypes.c_int32, ctypes.c_int32,
                                         ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int32)]),
    "dugks_batch_destroy": (ctypes.c_int, [ctypes.c_void_p]),
    "dugks_check_bounded_wait": (ctypes.c_int, [ctypes.c_int64, ctypes.c_void_p]),
    "dugks_set_velocity_field": (ctypes.c_int, [ctypes.c_void_p, _dp, _dp, _dp, _dp]),
    "dugks_tile_shapes": (ctypes.c_int32, [ctypes.c_int32, ctypes.POINTER(ctypes.c_int32),
                                           ctypes.POINTER(ctypes.c_int32), ctypes.c_int32]),
    "dugks_autotune": (ctypes.c_int, [ctypes.POINTER(DugksParams), _dp, _dp, _dp, _dp, ctypes.c_int32,
                                      ctypes.c_void_p, ctypes.POINTER(ctypes.c_int32), _dp]),
}

STATIC_REDUCE_MAX_CELLS = 16777216


class DugksError(RuntimeError):
    def __init__(self, code, what):
        self.code = code
        msg = lib().dugks_status_string(code).decode() if _lib is not None else ""
        super().__init__("%s failed: %s (%s)" % (what, STATUS.get(code, code), msg))


_lib = None


def library_path():
    return _build.LIB_PATH


def lib(build_if_missing=False):
    """Load the CUDA library.  Raises if it has not been built (no fallback).
    DUGKS_LIBRARY in the environment names another build of the same library
    to load instead (e.g. the bounds-checked one, build.CHECKED_LIB_PATH)."""
    global _lib
    if _lib is None:
        path = os.environ.get("DUGKS_LIBRARY") or _build.LIB_PATH
        if not os.path.exists(path):
            if not build_if_missing:
                raise ImportError("CUDA library %s is not built; run __graft_entry__.build()" % path)
            _build.build()
        L = ctypes.CDLL(path)
        for name, (res, args) in SIGNATURES.items():
            fn = getattr(L, name)
            fn.restype = res
            fn.argtypes = args
        _lib = L
    return _lib


def _check(code, what):
    if code != 0:
        raise DugksError(code, what)


_ENUM = {
    "model": {"coupled": 0, "ac": 1},
    "precision": {"fp64": 0, "fp32": 1},
    "bc": {"periodic": 0, "wall": 1},
    "visc": {"reciprocal": 0, "linear": 1},
    "velocity_field": {"uniform": 0, "rotation": 1, "shear": 2, "deformation": 3, "sampled": 4},
    "recon": {"central": 0, "upwind": 1},
}


def make_params(cfg):
    p = DugksParams()
    p.nx, p.ny = int(cfg["nx"]), int(cfg["ny"])
    p.lattice = 9
    p.model = _ENUM["model"][cfg.get("model", "coupled")]
    p.precision = _ENUM["precision"][cfg.get("precision", "fp64")]
    p.bc_x = _ENUM["bc"][cfg.get("bc_x", "periodic")]
    p.bc_y = _ENUM["bc"][cfg.get("bc_y", "periodic")]
    p.visc_interp = _ENUM["visc"][cfg.get("visc", "reciprocal")]
    p.gravity_mode = int(cfg.get("gravity_mode", 0))
    p.tile_shape = int(cfg.get("tile_shape", 0))
    for k in ("cfl", "mobility", "width", "rho_h", "rho_l", "mu_h", "mu_l", "sigma", "gx", "gy",
              "rho_ref", "phi_ref", "p_ref", "u0x", "u0y", "vel_u0", "vel_length"):
        setattr(p, k, float(cfg.get(k, 0.0)))
    p.velocity_field = _ENUM["velocity_field"][cfg.get("velocity_field", "uniform")]
    p.reserved2 = 0
    p.recon = _ENUM["recon"][cfg.get("recon", "central")]
    p.reserved3 = 0
    if p.precision == 0:
        # the FP64 path keeps absolute distributions unless asked otherwise
        p.phi_ref = float(cfg.get("phi_ref_fp64", 0.0))
        p.p_ref = float(cfg.get("p_ref_fp64", 0.0))
    return p


def check_bounded_wait(max_polls=0, stream=None):
    """Runs the bounded-wait self-check; returns the status code (-6 = the
    wait ran out as designed)."""
    return int(lib().dugks_check_bounded_wait(int(max_polls),
                                              ctypes.c_void_p(stream.cuda_stream) if stream is not None else None))


def check_batch_wait(budget_ns=0, stream=None):
    """Runs the persistent batched launch's wait self-check; returns the
    status code (-6 = the wait ran out as designed)."""
    return int(lib().dugks_check_batch_wait(int(budget_ns),
                                            ctypes.c_void_p(stream.cuda_stream) if stream is not None else None))


def tile_shapes(precision="fp32"):
    """Compiled step-kernel tile shapes [(tx, ty), ...]; cfg["tile_shape"] = k
    selects entry k - 1 (0: the library default, entry 0)."""
    prec = _ENUM["precision"][precision]
    n = int(lib().dugks_tile_shapes(prec, None, None, 0))
    tx, ty = (ctypes.c_int32 * n)(), (ctypes.c_int32 * n)()
    lib().dugks_tile_shapes(prec, tx, ty, n)
    return list(zip(tx[:], ty[:]))


def autotune(cfg, phi0, ux0=None, uy0=None, p0=None, trial_steps=20, stream=None):
    """Times every compiled tile shape on this problem (one at a time, in
    library-allocated workspaces) and returns (best tile_shape value,
    [ms per step of each shape, -1 where one failed])."""
    import torch

    params = make_params(cfg)
    n = len(tile_shapes(cfg.get("precision", "fp64")))
    shp = (params.ny, params.nx)
    arrs = [_host(phi0, shp), _host(ux0, shp), _host(uy0, shp), _host(p0, shp)]
    stream = stream if stream is not None else torch.cuda.current_stream()
    best = ctypes.c_int32(0)
    ms = np.zeros(n)
    code = lib().dugks_autotune(ctypes.byref(params), *[_ptr(a) for a in arrs], int(trial_steps),
                                ctypes.c_void_p(stream.cuda_stream), ctypes.byref(best), _ptr(ms))
    _check(code, "dugks_autotune")
    return int(best.value), [float(v) for v in ms]


def workspace_bytes(cfg):
    return int(lib().dugks_workspace_bytes(ctypes.byref(make_params(cfg))))


def _host(a, shape):
    if a is None:
        return None
    a = np.ascontiguousarray(a, dtype=np.float64).reshape(shape)
    return a


def _ptr(a):
    return None if a is None else a.ctypes.data_as(_dp)


def _check_static_args(torch, phi, ux, uy, out, snap):
    """The kernel reads n doubles of phi, ux, uy (3n of snap) and writes 4 of
    out on one device: anything else would read or write past a tensor."""
    named = [("phi", phi), ("ux", ux), ("uy", uy), ("out", out)] + ([("snap", snap)] if snap is not None else [])
    for name, t in named:
        if not isinstance(t, torch.Tensor):
            raise ValueError("%s must be a torch tensor" % name)
        if t.dtype != torch.float64 or not t.is_cuda or not t.is_contiguous():
            raise ValueError("%s must be a contiguous CUDA float64 tensor" % name)
        if t.device != phi.device:
            raise ValueError("%s is on %s, phi on %s" % (name, t.device, phi.device))
    n = phi.numel()
    if n < 1 or ux.numel() != n or uy.numel() != n:
        raise ValueError("phi, ux and uy must have the same number (>= 1) of elements")
    if snap is not None and snap.numel() != 3 * n:
        raise ValueError("snap must hold 3 n = %d elements, got %d" % (3 * n, snap.numel()))
    if out.numel() < 4:
        raise ValueError("out must hold at least 4 elements")


def reduce_fields_static(phi, ux, uy, out, snap=None, stream=None):
    """dugks_reduce_fields_static on CUDA float64 tensors (no allocation in the
    library): phi, ux, uy of n elements, snap of 3n or None, out of 4 elements
    receives (phi mass, residual of phi, residual of u, max |u|)."""
    import torch

    _check_static_args(torch, phi, ux, uy, out, snap)
    n = phi.numel()
    if n > STATIC_REDUCE_MAX_CELLS:
        raise ValueError("dugks_reduce_fields_static takes at most %d cells, got %d" % (STATIC_REDUCE_MAX_CELLS, n))
    st = stream if stream is not None else torch.cuda.current_stream()

    def p(t):
        return None if t is None else ctypes.cast(t.data_ptr(), _dp)

    code = lib().dugks_reduce_fields_static(p(phi), p(ux), p(uy), p(snap), n, p(out), ctypes.c_void_p(st.cuda_stream))
    _check(code, "dugks_reduce_fields_static")


class Solver:
    """One DUGKS problem resident on the GPU.

    workspace: "torch" (a torch.uint8 CUDA tensor owned by this object),
    "library" (cudaMalloc inside the library) or a caller tensor.
    stream: a torch.cuda.Stream, or None for torch's current stream.
    """

    def __init__(self, cfg, phi0, ux0=None, uy0=None, p0=None, workspace="torch", stream=None, device=None):
        import torch

        self.cfg = dict(cfg)
        self.params = make_params(cfg)
        self.nx, self.ny = self.params.nx, self.params.ny
        L = lib()
        need = int(L.dugks_workspace_bytes(ctypes.byref(self.params)))
        if need == 0:
            raise DugksError(-1, "dugks_workspace_bytes")
        self.device = torch.device("cuda" if device is None else device)
        self.stream = stream if stream is not None else torch.cuda.current_stream(self.device)
        self._ws = None
        ws_ptr, ws_len = None, 0
        if isinstance(workspace, str) and workspace == "torch":
            self._ws = torch.empty(need + 256, dtype=torch.uint8, device=self.device)
            base = self._ws.data_ptr()
            ws_ptr = (base + 255) // 256 * 256
            ws_len = need
        elif isinstance(workspace, str) and workspace == "library":
            pass
        else:
            self._ws = workspace
            ws_ptr, ws_len = workspace.data_ptr(), workspace.numel() * workspace.element_size()
        shp = (self.ny, self.nx)
        arrs = [_host(phi0, shp), _host(ux0, shp), _host(uy0, shp), _host(p0, shp)]
        h = ctypes.c_void_p()
        with torch.cuda.device(self.device):
            code = L.dugks_create(ctypes.byref(self.params), *[_ptr(a) for a in arrs],
                                  ctypes.c_void_p(ws_ptr) if ws_ptr else None, ws_len,
                                  ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h))
        _check(code, "dugks_create")
        self.h = h
        self.workspace_bytes = need

    # -- lifetime
    def close(self):
        if getattr(self, "h", None):
            code = lib().dugks_destroy(self.h)
            self.h = None
            _check(code, "dugks_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    # -- stepping
    def step(self, n=1):
        _check(lib().dugks_step(self.h, int(n)), "dugks_step")

    @property
    def step_count(self):
        return int(lib().dugks_step_count(self.h))

    def set_velocity_field(self, ux_cell, uy_cell, ux_xface=None, uy_yface=None):
        """Sampled velocity field (cfg velocity_field "sampled"): cell arrays and
        optional face normals, [ny][nx] each; used from the next step on."""
        shp = (self.ny, self.nx)
        arrs = [_host(a, shp) for a in (ux_cell, uy_cell, ux_xface, uy_yface)]
        _check(lib().dugks_set_velocity_field(self.h, *[_ptr(a) for a in arrs]), "dugks_set_velocity_field")

    def sync(self):
        _check(lib().dugks_sync(self.h), "dugks_sync")

    # -- outputs
    def macros(self):
        shp = (self.ny, self.nx)
        out = {k: np.empty(shp) for k in ("phi", "p", "ux", "uy")}
        _check(lib().dugks_macros(self.h, *[_ptr(out[k]) for k in ("phi", "p", "ux", "uy")], 0), "dugks_macros")
        return out

    def macros_device(self, out):
        """Write phi, p, ux, uy into CUDA float64 tensors of shape (ny, nx) (dict; missing keys skipped)."""
        ptrs = []
        for k in ("phi", "p", "ux", "uy"):
            t = out.get(k)
            ptrs.append(None if t is None else ctypes.cast(t.data_ptr(), _dp))
        _check(lib().dugks_macros(self.h, *ptrs, 1), "dugks_macros")

    def reduce(self):
        v = [ctypes.c_double() for _ in range(4)]
        _check(lib().dugks_reduce(self.h, *[ctypes.byref(x) for x in v]), "dugks_reduce")
        return tuple(x.value for x in v)

    def reduce_rows(self, row0, nrows):
        """The sums behind reduce() over rows [row0, row0 + nrows):
        (array [sum phi, sum phi^2, sum dphi^2, sum |u|^2, sum |du|^2, max |u|],
        whether there was a previous reduction to difference against)."""
        sums = np.zeros(6)
        had = ctypes.c_int32()
        _check(lib().dugks_reduce_rows(self.h, int(row0), int(nrows), _ptr(sums), ctypes.byref(had)),
               "dugks_reduce_rows")
        return sums, bool(had.value)

    def distributions(self):
        f = np.empty((9, self.ny, self.nx))
        g = np.empty((9, self.ny, self.nx))
        hh = np.empty((2, self.ny, self.nx))
        _check(lib().dugks_get_distributions(self.h, _ptr(f), _ptr(g), _ptr(hh)), "dugks_get_distributions")
        return f, g, hh

    def row_buffer(self, nrows):
        """A device tensor shaped [planes][nrows][nx] in the storage precision,
        for get_rows / set_rows."""
        import torch

        nq = 18 if self.cfg.get("model", "coupled") == "coupled" else 9
        dt = torch.float32 if int(lib().dugks_state_element_bytes(self.h)) == 4 else torch.float64
        return torch.empty((nq + 2, nrows, self.nx), dtype=dt, device=self.device)

    def _rows_arg(self, buf, nrows):
        import torch

        want = (18 if self.cfg.get("model", "coupled") == "coupled" else 9) + 2
        esz = int(lib().dugks_state_element_bytes(self.h))
        if not (isinstance(buf, torch.Tensor) and buf.is_cuda and buf.is_contiguous() and
                buf.element_size() == esz and buf.numel() == want * nrows * self.nx):
            raise ValueError("row buffer must be a contiguous CUDA tensor of %d x %d x %d elements of %d bytes"
                             % (want, nrows, self.nx, esz))
        return ctypes.c_void_p(buf.data_ptr())

    def get_rows(self, row0, nrows, buf):
        """Rows [row0, row0 + nrows) of the stored state into buf (see row_buffer); on the solver's stream."""
        _check(lib().dugks_get_rows(self.h, int(row0), int(nrows), self._rows_arg(buf, nrows), 1), "dugks_get_rows")

    def set_rows(self, row0, nrows, buf):
        """buf (see row_buffer) into rows [row0, row0 + nrows) of the stored state; on the solver's stream."""
        _check(lib().dugks_set_rows(self.h, int(row0), int(nrows), self._rows_arg(buf, nrows), 1), "dugks_set_rows")

    def get_state(self):
        n = int(lib().dugks_state_bytes(self.h))
        buf = np.empty(n, dtype=np.uint8)
        _check(lib().dugks_get_state(self.h, buf.ctypes.data_as(ctypes.c_void_p), n), "dugks_get_state")
        return buf

    def set_state(self, buf):
        buf = np.ascontiguousarray(buf, dtype=np.uint8)
        _check(lib().dugks_set_state(self.h, buf.ctypes.data_as(ctypes.c_void_p), buf.size), "dugks_set_state")


class Batch:
    """Members (Solver objects) advanced together by dugks_batch_step.
    persistent: K steps of each kernel group per launch, else (the default)
    one grid launch per group and step (dugks_batch_set_persistent)."""

    def __init__(self, stream=None, persistent=False):
        import torch

        self.stream = stream if stream is not None else torch.cuda.current_stream()
        h = ctypes.c_void_p()
        _check(lib().dugks_batch_create(ctypes.c_void_p(self.stream.cuda_stream), ctypes.byref(h)),
               "dugks_batch_create")
        self.h = h
        self.members = []
        self.set_persistent(persistent)

    def set_persistent(self, on):
        _check(lib().dugks_batch_set_persistent(self.h, 1 if on else 0), "dugks_batch_set_persistent")

    def add(self, solver):
        _check(lib().dugks_batch_add(self.h, solver.h), "dugks_batch_add")
        self.members.append(solver)

    def remove(self, solver):
        _check(lib().dugks_batch_remove(self.h, solver.h), "dugks_batch_remove")
        self.members.remove(solver)

    def __len__(self):
        return int(lib().dugks_batch_size(self.h))

    def step(self, n=1):
        _check(lib().dugks_batch_step(self.h, int(n)), "dugks_batch_step")

    def sync(self):
        _check(lib().dugks_batch_sync(self.h), "dugks_batch_sync")

    def mark(self):
        """A torch event recorded after the work enqueued so far."""
        import torch

        ev = torch.cuda.Event()
        ev.record(self.stream)
        return ev

    def close(self):
        if getattr(self, "h", None):
            code = lib().dugks_batch_destroy(self.h)
            self.h = None
            _check(code, "dugks_batch_destroy")

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()
