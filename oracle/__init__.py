"""ctypes wrapper of the plain FP64 CPU oracle (``lbm_oracle.c``).

TEST INFRASTRUCTURE ONLY: the tests, the smoke check and the benchmark's CPU
baseline leg may import this package; the CUDA library and its Python binding
never do.  Every function here is a thin marshalling layer over the C code,
whose header comment lists the steps of the paper it follows.
"""
import ctypes
import os

import numpy as np

from . import build as _build

Q = 9
FSI = {"density": 0, "psi": 1, "modified": 2}
WALL = {"neq": 0, "bb": 1}
GHOST = {"copy": 0, "mirror": 1, "zero": 2, "skip": 3, "mean": 4}
EOS = {"pl": 0, "cs": 1}
OMEGA = {"w": 0, "cs2w": 1}
VISC = {"tau": 0, "mu": 1}


class OracleParams(ctypes.Structure):
    _fields_ = [("kV", ctypes.c_double), ("kM", ctypes.c_double), ("kL", ctypes.c_double),
                ("rho_1", ctypes.c_double), ("rho_2", ctypes.c_double),
                ("G", ctypes.c_double), ("sigma", ctypes.c_double),
                ("tau_rho", ctypes.c_double), ("tau_e", ctypes.c_double),
                ("tau_zeta", ctypes.c_double), ("tau_j", ctypes.c_double),
                ("tau_q", ctypes.c_double),
                ("tau_nu_L", ctypes.c_double), ("tau_nu_V", ctypes.c_double),
                ("rho_L", ctypes.c_double), ("rho_V", ctypes.c_double),
                ("wall", ctypes.c_int), ("ghost", ctypes.c_int), ("omega", ctypes.c_int),
                ("eos", ctypes.c_int), ("cs_a", ctypes.c_double), ("cs_b", ctypes.c_double),
                ("cs_R", ctypes.c_double), ("cs_T", ctypes.c_double),
                ("visc", ctypes.c_int)]


class OracleDiag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_long), ("mass", ctypes.c_double),
                ("rho_max", ctypes.c_double), ("rho_min", ctypes.c_double),
                ("u_max", ctypes.c_double), ("theta_deg", ctypes.c_double),
                ("fit_rms", ctypes.c_double), ("xc", ctypes.c_double),
                ("yc", ctypes.c_double), ("radius", ctypes.c_double),
                ("n_contour", ctypes.c_int), ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = ctypes.CDLL(path)
        dp = ctypes.POINTER(ctypes.c_double)
        L.oracle_create.restype = ctypes.c_void_p
        L.oracle_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.POINTER(OracleParams),
                                    ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_double]
        L.oracle_destroy.argtypes = [ctypes.c_void_p]
        L.oracle_set_threads.argtypes = [ctypes.c_int]
        L.oracle_set_density.argtypes = [ctypes.c_void_p, dp]
        L.oracle_init_droplet.argtypes = [ctypes.c_void_p] + [ctypes.c_double] * 4
        L.oracle_step.argtypes = [ctypes.c_void_p, ctypes.c_long]
        L.oracle_time.restype = ctypes.c_long
        L.oracle_time.argtypes = [ctypes.c_void_p]
        L.oracle_get_fields.argtypes = [ctypes.c_void_p] + [ctypes.c_void_p] * 6
        L.oracle_get_populations.argtypes = [ctypes.c_void_p, dp]
        L.oracle_set_populations.argtypes = [ctypes.c_void_p, dp, ctypes.c_void_p, ctypes.c_void_p]
        L.oracle_diagnostics.argtypes = [ctypes.c_void_p, ctypes.c_double, ctypes.c_double,
                                         ctypes.c_double, ctypes.POINTER(OracleDiag)]
        L.oracle_contact_angle.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_void_p,
                                           ctypes.c_double, ctypes.c_double, ctypes.c_double,
                                           ctypes.c_double, ctypes.POINTER(OracleDiag)]
        L.oracle_contact_radius.restype = ctypes.c_double
        L.oracle_contact_radius.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_void_p,
                                            ctypes.c_int, ctypes.c_double, ctypes.c_double]
        L.oracle_mrt_matrices.argtypes = [dp, dp]
        L.oracle_p_eos.restype = ctypes.c_double
        L.oracle_p_eos.argtypes = [ctypes.POINTER(OracleParams), ctypes.c_double]
        L.oracle_psi.restype = ctypes.c_double
        L.oracle_psi.argtypes = [ctypes.POINTER(OracleParams), ctypes.c_double]
        _lib = L
    return _lib


def paper_params(**over):
    """The parameters of Sec. III: piecewise-linear EOS (Eq. 15) with
    theta_V = 0.64 cs^2, theta_M = -0.04 cs^2, theta_L = cs^2, rho_1 = 1.36,
    rho_2 = 481.04; G = -1; sigma = 0.084; tau_rho = tau_j = 1,
    1/tau_e = 1/tau_zeta = 0.8, 1/tau_q = 1.1, tau_nu = 1.1."""
    d = dict(kV=0.64, kM=-0.04, kL=1.0, rho_1=1.36, rho_2=481.04, G=-1.0, sigma=0.084,
             tau_rho=1.0, tau_e=1.0 / 0.8, tau_zeta=1.0 / 0.8, tau_j=1.0, tau_q=1.0 / 1.1,
             tau_nu_L=1.1, tau_nu_V=1.1, rho_L=500.0, rho_V=1.0, wall="neq", ghost="copy",
             omega="w", eos="pl", cs_a=1.0, cs_b=4.0, cs_R=1.0, cs_T=0.0, visc="tau")
    d.update(over)
    return d


def to_struct(params):
    p = dict(params)
    p["wall"] = WALL[p["wall"]] if isinstance(p["wall"], str) else p["wall"]
    p["ghost"] = GHOST[p["ghost"]] if isinstance(p["ghost"], str) else p["ghost"]
    p["omega"] = OMEGA[p["omega"]] if isinstance(p["omega"], str) else p["omega"]
    p.setdefault("eos", "pl")
    p["eos"] = EOS[p["eos"]] if isinstance(p["eos"], str) else p["eos"]
    for k, v in (("cs_a", 1.0), ("cs_b", 4.0), ("cs_R", 1.0), ("cs_T", 0.0)):
        p.setdefault(k, v)
    p.setdefault("visc", "tau")
    p["visc"] = VISC[p["visc"]] if isinstance(p["visc"], str) else p["visc"]
    return OracleParams(**{k: p[k] for k, _ in OracleParams._fields_})


def set_threads(n):
    lib().oracle_set_threads(int(n))


def _dptr(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def p_eos(params, rho):
    return lib().oracle_p_eos(ctypes.byref(to_struct(params)), float(rho))


def psi(params, rho):
    return lib().oracle_psi(ctypes.byref(to_struct(params)), float(rho))


def mrt_matrices():
    M = np.zeros((Q, Q))
    Minv = np.zeros((Q, Q))
    lib().oracle_mrt_matrices(_dptr(M), _dptr(Minv))
    return M, Minv


def contact_angle(rho, solid, level, y_w, x_ref, d_min=3.0):
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    s = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8)
    d = OracleDiag()
    lib().oracle_contact_angle(nx, ny, _dptr(rho), None if s is None else s.ctypes.data,
                               level, y_w, x_ref, d_min, ctypes.byref(d))
    return d.as_dict()


def contact_radius(rho, solid, row, level, x_ref):
    """Spreading radius along node row `row` (oracle_contact_radius)."""
    rho = np.ascontiguousarray(rho, dtype=np.float64)
    ny, nx = rho.shape
    s = None if solid is None else np.ascontiguousarray(solid, dtype=np.uint8)
    return lib().oracle_contact_radius(nx, ny, _dptr(rho), None if s is None else s.ctypes.data,
                                       int(row), float(level), float(x_ref))


class Lattice:
    """One oracle lattice of ny x nx nodes (row-major, x fastest)."""

    def __init__(self, nx, ny, params, solid=None, fsi="modified", gw=0.0):
        self.nx, self.ny = int(nx), int(ny)
        self.params = dict(params)
        self._ps = to_struct(params)
        self.solid = (np.zeros((ny, nx), np.uint8) if solid is None
                      else np.ascontiguousarray(solid, dtype=np.uint8))
        gw_field = None
        gw_uniform = 0.0
        if np.ndim(gw) == 0:
            gw_uniform = float(gw)
        else:
            gw_field = np.ascontiguousarray(gw, dtype=np.float64)
        self._h = lib().oracle_create(self.nx, self.ny, ctypes.byref(self._ps),
                                      self.solid.ctypes.data,
                                      FSI[fsi] if isinstance(fsi, str) else int(fsi),
                                      None if gw_field is None else gw_field.ctypes.data,
                                      gw_uniform)
        if not self._h:
            raise ValueError("oracle_create rejected the configuration")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            lib().oracle_destroy(h)
            self._h = None

    @property
    def t(self):
        return lib().oracle_time(self._h)

    def init_droplet(self, x0, y0, R, width=2.0):
        lib().oracle_init_droplet(self._h, x0, y0, R, width)

    def set_density(self, rho):
        rho = np.ascontiguousarray(rho, dtype=np.float64)
        lib().oracle_set_density(self._h, _dptr(rho))

    def step(self, n=1):
        lib().oracle_step(self._h, int(n))

    def fields(self):
        shp = (self.ny, self.nx)
        out = {k: np.zeros(shp) for k in ("rho", "ux", "uy", "Fx", "Fy", "psi")}
        lib().oracle_get_fields(self._h, *[out[k].ctypes.data for k in
                                           ("rho", "ux", "uy", "Fx", "Fy", "psi")])
        return out

    def populations(self):
        f = np.zeros((Q, self.ny, self.nx))
        lib().oracle_get_populations(self._h, _dptr(f))
        return f

    def set_populations(self, f):
        f = np.ascontiguousarray(f, dtype=np.float64)
        lib().oracle_set_populations(self._h, _dptr(f), None, None)

    def diagnostics(self, y_w, x_ref, d_min=3.0):
        d = OracleDiag()
        lib().oracle_diagnostics(self._h, y_w, x_ref, d_min, ctypes.byref(d))
        return d.as_dict()
