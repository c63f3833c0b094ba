"""ctypes declarations of liblbm.so (include/lbm.h).  Marshalling only."""
import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "liblbm.so")

FSI = {"density": 0, "psi": 1, "modified": 2}
WALL = {"neq": 0, "bb": 1}
GHOST = {"copy": 0, "mirror": 1, "zero": 2, "skip": 3, "mean": 4}
OMEGA = {"w": 0, "cs2w": 1}
EOS = {"pl": 0, "cs": 1}
PREC = {"fp64": 0, "fp32": 1, "fp32_f64": 2}
VISC = {"tau": 0, "mu": 1}
STATUS = {0: "LBM_OK", 1: "LBM_ERR_ARG", 2: "LBM_ERR_OOM", 3: "LBM_ERR_CUDA",
          4: "LBM_ERR_NONFINITE", 5: "LBM_ERR_TIMEOUT", 6: "LBM_ERR_STATE"}

# every symbol include/lbm.h declares
EXPORTS = ["lbm_default_params", "lbm_create", "lbm_create_batch", "lbm_destroy",
           "lbm_instance_size", "lbm_init_droplet", "lbm_set_density", "lbm_step", "lbm_sync",
           "lbm_time", "lbm_get_fields", "lbm_get_populations", "lbm_diagnostics", "lbm_contact_radius",
           "lbm_set_density_async", "lbm_get_fields_async", "lbm_set_density_all_async",
           "lbm_get_fields_all_async", "lbm_selftest_fp32_math", "lbm_selftest_fp64_math",
           "lbm_selftest_fp64_rate",
           "lbm_strip_neighbours", "lbm_get_work_items",
           "lbm_set_gw_field", "lbm_set_launch", "lbm_get_launch", "lbm_selftest_wait_timeout",
           "lbm_diagnostics_noalloc", "lbm_adjoint", "lbm_save", "lbm_load", "lbm_autotune",
           "lbm_last_error"]


class LbmParams(ctypes.Structure):
    _fields_ = [("eos", ctypes.c_int), ("eos_p", ctypes.c_double * 6),
                ("G", ctypes.c_double), ("sigma", ctypes.c_double),
                ("tau_rho", ctypes.c_double), ("tau_e", ctypes.c_double),
                ("tau_zeta", ctypes.c_double), ("tau_j", ctypes.c_double),
                ("tau_q", ctypes.c_double),
                ("tau_nu_L", ctypes.c_double), ("tau_nu_V", ctypes.c_double),
                ("rho_L", ctypes.c_double), ("rho_V", ctypes.c_double),
                ("wall", ctypes.c_int), ("ghost", ctypes.c_int), ("omega", ctypes.c_int),
                ("prec", ctypes.c_int), ("rho_ref", ctypes.c_double), ("visc", ctypes.c_int)]


class LbmInstanceDesc(ctypes.Structure):
    _fields_ = [("nx", ctypes.c_int), ("ny", ctypes.c_int),
                ("params", ctypes.POINTER(LbmParams)), ("solid", ctypes.c_void_p),
                ("fsi", ctypes.c_int), ("gw_field", ctypes.c_void_p),
                ("gw_uniform", ctypes.c_double)]


class LbmDiag(ctypes.Structure):
    _fields_ = [("step", ctypes.c_long), ("mass", ctypes.c_double),
                ("rho_max", ctypes.c_double), ("rho_min", ctypes.c_double),
                ("u_max", ctypes.c_double), ("theta_deg", ctypes.c_double),
                ("fit_rms", ctypes.c_double), ("xc", ctypes.c_double), ("yc", ctypes.c_double),
                ("radius", ctypes.c_double), ("n_contour", ctypes.c_int),
                ("status", ctypes.c_int)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_}


class LbmError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"{STATUS.get(status, status)}: {msg}")
        self.status = status


_lib = None


def load(path=None):
    """Load liblbm.so (or the library named by the LBM_LIBRARY environment
    variable, e.g. the checked build liblbm_check.so).  There is no
    fallback: a missing library is an error."""
    global _lib
    if _lib is not None:
        return _lib
    if path is None:
        path = os.environ.get("LBM_LIBRARY") or LIB_PATH
    if not os.path.exists(path):
        raise ImportError(f"liblbm.so not found at {path}; build it with "
                          "`python -c 'import __graft_entry__ as g; g.build()'`")
    L = ctypes.CDLL(path)
    vp, i, d, l = ctypes.c_void_p, ctypes.c_int, ctypes.c_double, ctypes.c_long
    P = ctypes.POINTER
    sig = {
        "lbm_default_params": (i, [P(LbmParams)]),
        "lbm_create": (i, [i, i, P(LbmParams), vp, i, vp, d, vp, P(vp)]),
        "lbm_create_batch": (i, [i, P(LbmInstanceDesc), vp, P(vp)]),
        "lbm_destroy": (None, [vp]),
        "lbm_instance_size": (i, [vp, i, P(i), P(i)]),
        "lbm_init_droplet": (i, [vp, i, d, d, d, d]),
        "lbm_set_density": (i, [vp, i, vp, i]),
        "lbm_set_density_async": (i, [vp, i, vp, i]),
        "lbm_step": (i, [vp, l]),
        "lbm_sync": (i, [vp]),
        "lbm_time": (l, [vp]),
        "lbm_get_fields": (i, [vp, i, vp, vp, vp, i]),
        "lbm_get_fields_async": (i, [vp, i, vp, vp, vp, i]),
        "lbm_set_density_all_async": (i, [vp, vp, i]),
        "lbm_get_fields_all_async": (i, [vp, vp, vp, vp, i]),
        "lbm_selftest_fp32_math": (i, [ctypes.c_long, vp, vp]),
        "lbm_selftest_fp64_math": (i, [ctypes.c_long, vp, vp]),
        "lbm_selftest_fp64_rate": (i, [P(d)]),
        "lbm_strip_neighbours": (i, [i, i, i, P(i), vp, vp, vp, i, P(i)]),
        "lbm_get_work_items": (i, [vp, P(i), vp, vp, vp, i, P(i)]),
        "lbm_get_populations": (i, [vp, i, vp, i]),
        "lbm_diagnostics": (i, [vp, i, d, d, d, P(LbmDiag)]),
        "lbm_contact_radius": (i, [vp, i, i, d, d, P(ctypes.c_double)]),
        "lbm_set_gw_field": (i, [vp, i, vp]),
        "lbm_set_launch": (i, [vp, i, i, i, i, i]),
        "lbm_get_launch": (i, [vp, P(i), P(i), P(i)]),
        "lbm_selftest_wait_timeout": (i, [vp, d]),
        "lbm_adjoint": (i, [vp, l, d, d, d, d, P(d), P(d), vp]),
        "lbm_save": (i, [vp, ctypes.c_char_p]),
        "lbm_load": (i, [vp, ctypes.c_char_p]),
        "lbm_autotune": (i, [vp, i, P(i), P(i), P(i), P(d)]),
        "lbm_diagnostics_noalloc": (i, [i, i, vp, vp, vp, vp, d, d, d, d, vp, P(LbmDiag)]),
        "lbm_last_error": (ctypes.c_char_p, []),
    }
    for name, (res, args) in sig.items():
        fn = getattr(L, name)
        fn.restype = res
        fn.argtypes = args
    _lib = L
    return L


def check(status):
    if status != 0:
        raise LbmError(status, load().lbm_last_error().decode())
    return status
