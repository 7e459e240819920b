"""ctypes binding of the FP64 CPU oracle (dugks_oracle.c).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the bench's
CPU-baseline leg use it; the product path never does.  It shares no code with
the CUDA library.  Fields are numpy float64 arrays of shape (ny, nx).
"""
import ctypes

import numpy as np

from . import build as _build

Q = 9


class OracleParams(ctypes.Structure):
    _fields_ = [
        ("nx", ctypes.c_int), ("ny", ctypes.c_int),
        ("model", ctypes.c_int), ("wall_y", ctypes.c_int),
        ("visc", ctypes.c_int), ("gravity_mode", ctypes.c_int),
        ("cfl", ctypes.c_double), ("mobility", ctypes.c_double),
        ("width", ctypes.c_double),
        ("rho_h", ctypes.c_double), ("rho_l", ctypes.c_double),
        ("mu_h", ctypes.c_double), ("mu_l", ctypes.c_double),
        ("sigma", ctypes.c_double),
        ("gx", ctypes.c_double), ("gy", ctypes.c_double),
        ("rho_ref", ctypes.c_double),
        ("u0x", ctypes.c_double), ("u0y", ctypes.c_double),
        ("velocity_field", ctypes.c_int), ("reserved", ctypes.c_int),
        ("vel_u0", ctypes.c_double), ("vel_length", ctypes.c_double),
        ("recon", ctypes.c_int), ("reserved2", ctypes.c_int),
    ]


_MODEL = {"coupled": 0, "ac": 1}
_VISC = {"reciprocal": 0, "linear": 1}
_FIELD = {"uniform": 0, "rotation": 1, "shear": 2, "deformation": 3, "sampled": 4}
_RECON = {"central": 0, "upwind": 1}

_lib = None
_dp = ctypes.POINTER(ctypes.c_double)


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        L.oracle_create.restype = ctypes.c_void_p
        L.oracle_create.argtypes = [ctypes.POINTER(OracleParams), _dp, _dp, _dp, _dp]
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.oracle_step_count.restype = ctypes.c_long
        L.oracle_step_count.argtypes = [ctypes.c_void_p]
        L.oracle_macros.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.oracle_get_state.argtypes = [ctypes.c_void_p, _dp, _dp, _dp]
        L.oracle_set_state.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, ctypes.c_long]
        L.oracle_reduce.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.oracle_lattice.argtypes = [ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int), _dp]
        L.oracle_feq.argtypes = [ctypes.c_double] * 3 + [_dp]
        L.oracle_sf.argtypes = [ctypes.c_double] * 5 + [_dp]
        L.oracle_geq.argtypes = [ctypes.c_double] * 4 + [_dp]
        L.oracle_sg.argtypes = [ctypes.c_double] * 6 + [_dp]
        L.oracle_prestep.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp, _dp]
        L.oracle_face_psi.argtypes = [ctypes.c_double, ctypes.c_double, _dp, _dp, _dp, _dp]
        L.oracle_grad_lap.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp, _dp, _dp, _dp]
        L.oracle_set_velocity.restype = ctypes.c_int
        L.oracle_set_velocity.argtypes = [ctypes.c_void_p, _dp, _dp, _dp, _dp]
        L.oracle_face_bar.argtypes = [ctypes.POINTER(OracleParams), _dp, ctypes.c_int, ctypes.c_int, ctypes.c_int, _dp]
        L.oracle_wall_face_bar.argtypes = [ctypes.POINTER(OracleParams), _dp, ctypes.c_int, ctypes.c_int, _dp]
        _lib = L
    return _lib


def _ptr(a):
    return a.ctypes.data_as(_dp)


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None:
        a = a.reshape(shape)
    return a


def make_params(cfg):
    """Oracle parameter struct from a workload dict (see the package's workloads module)."""
    p = OracleParams()
    p.nx, p.ny = int(cfg["nx"]), int(cfg["ny"])
    p.model = _MODEL[cfg.get("model", "coupled")]
    p.wall_y = 1 if cfg.get("bc_y", "periodic") == "wall" else 0
    p.visc = _VISC[cfg.get("visc", "reciprocal")]
    p.gravity_mode = int(cfg.get("gravity_mode", 0))
    for k in ("cfl", "mobility", "width", "rho_h", "rho_l", "mu_h", "mu_l", "sigma",
              "gx", "gy", "rho_ref", "u0x", "u0y", "vel_u0", "vel_length"):
        setattr(p, k, float(cfg.get(k, 0.0)))
    p.velocity_field = _FIELD[cfg.get("velocity_field", "uniform")]
    p.recon = _RECON[cfg.get("recon", "central")]
    if cfg.get("bc_x", "periodic") != "periodic":
        raise ValueError("the oracle supports periodic x only")
    return p


class Oracle:
    """One oracle run: create from initial fields, step, read macros/state."""

    def __init__(self, cfg, phi0, ux0=None, uy0=None, p0=None):
        self.cfg = dict(cfg)
        self.params = make_params(cfg)
        self.nx, self.ny = self.params.nx, self.params.ny
        shp = (self.ny, self.nx)
        self._keep = [_f64(phi0, shp)] + [None if a is None else _f64(a, shp) for a in (ux0, uy0, p0)]
        args = [None if a is None else _ptr(a) for a in self._keep]
        self.h = lib().oracle_create(ctypes.byref(self.params), *args)
        if not self.h:
            raise ValueError("oracle_create rejected the parameters")

    def close(self):
        if self.h:
            lib().oracle_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def step(self, n=1):
        lib().oracle_step(self.h, int(n))

    @property
    def step_count(self):
        return lib().oracle_step_count(self.h)

    def macros(self):
        shp = (self.ny, self.nx)
        out = {k: np.zeros(shp) for k in ("phi", "p", "ux", "uy")}
        lib().oracle_macros(self.h, *(_ptr(out[k]) for k in ("phi", "p", "ux", "uy")))
        return out

    def state(self):
        N = self.nx * self.ny
        f = np.zeros((Q, self.ny, self.nx))
        g = np.zeros((Q, self.ny, self.nx))
        h = np.zeros((2, self.ny, self.nx))
        lib().oracle_get_state(self.h, _ptr(f), _ptr(g), _ptr(h))
        assert f.size == Q * N
        return f, g, h

    def set_state(self, f, g, phiu_prev, step_count):
        f = _f64(f, (Q, self.ny, self.nx))
        g = _f64(g, (Q, self.ny, self.nx))
        h = _f64(phiu_prev, (2, self.ny, self.nx))
        lib().oracle_set_state(self.h, _ptr(f), _ptr(g), _ptr(h), int(step_count))

    def set_velocity(self, ux_cell, uy_cell, ux_xface=None, uy_yface=None):
        """Sampled velocity field (velocity_field "sampled"): cell arrays and
        optional normal components at x-faces ([j][i] = face i+1/2 of row j)
        and y-faces ([j][i] = face below row j)."""
        shp = (self.ny, self.nx)
        arrs = [_f64(ux_cell, shp), _f64(uy_cell, shp)] + [None if a is None else _f64(a, shp)
                                                          for a in (ux_xface, uy_yface)]
        self._vel = arrs
        if not lib().oracle_set_velocity(self.h, *[None if a is None else _ptr(a) for a in arrs]):
            raise ValueError("oracle_set_velocity rejected the arguments")

    def reduce(self):
        vals = [ctypes.c_double() for _ in range(4)]
        lib().oracle_reduce(self.h, *(ctypes.byref(v) for v in vals))
        return tuple(v.value for v in vals)


# ---- the pieces of one step, for the pins ----

def lattice():
    ex = (ctypes.c_int * Q)()
    ey = (ctypes.c_int * Q)()
    w = np.zeros(Q)
    lib().oracle_lattice(ex, ey, _ptr(w))
    return np.array(ex[:]), np.array(ey[:]), w


def feq(phi, ux, uy):
    out = np.zeros(Q)
    lib().oracle_feq(phi, ux, uy, _ptr(out))
    return out


def sf(theta, nx, ny, Dx, Dy):
    out = np.zeros(Q)
    lib().oracle_sf(theta, nx, ny, Dx, Dy, _ptr(out))
    return out


def geq(p, rho, ux, uy):
    out = np.zeros(Q)
    lib().oracle_geq(p, rho, ux, uy, _ptr(out))
    return out


def sg(drhox, drhoy, Fx, Fy, ux, uy):
    out = np.zeros(Q)
    lib().oracle_sg(drhox, drhoy, Fx, Fy, ux, uy, _ptr(out))
    return out


def prestep(tau, dt, tilde, eq, src):
    tilde, eq, src = _f64(tilde), _f64(eq), _f64(src)
    bp, tp = np.zeros(Q), np.zeros(Q)
    lib().oracle_prestep(tau, dt, _ptr(tilde), _ptr(eq), _ptr(src), _ptr(bp), _ptr(tp))
    return bp, tp


def face_psi(tau, h, bar, eq, src):
    bar, eq, src = _f64(bar), _f64(eq), _f64(src)
    out = np.zeros(Q)
    lib().oracle_face_psi(tau, h, _ptr(bar), _ptr(eq), _ptr(src), _ptr(out))
    return out


def grad_lap(phi, wall_y=False):
    phi = _f64(phi)
    ny, nx = phi.shape
    gx, gy, lp = np.zeros_like(phi), np.zeros_like(phi), np.zeros_like(phi)
    lib().oracle_grad_lap(nx, ny, 1 if wall_y else 0, _ptr(phi), _ptr(gx), _ptr(gy), _ptr(lp))
    return gx, gy, lp


def face_bar(cfg, B, i, j, xface):
    """psi_bar at one face from the grid B [Q][ny][nx] (central or upwind, per cfg["recon"])."""
    p = make_params(cfg)
    B = _f64(B, (Q, p.ny, p.nx))
    out = np.zeros(Q)
    lib().oracle_face_bar(ctypes.byref(p), _ptr(B), int(i), int(j), 1 if xface else 0, _ptr(out))
    return out


def wall_face_bar(cfg, B, i, top=False):
    """psi_bar at the wall face of column i (bottom or top wall) from B [Q][ny][nx]."""
    p = make_params(cfg)
    B = _f64(B, (Q, p.ny, p.nx))
    out = np.zeros(Q)
    lib().oracle_wall_face_bar(ctypes.byref(p), _ptr(B), int(i), 1 if top else 0, _ptr(out))
    return out
