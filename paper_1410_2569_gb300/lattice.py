"""Python face of liblbm: the same calls as include/lbm.h, argument
marshalling only.  Every step of the method runs in the library's CUDA
kernels; PyTorch supplies the CUDA stream and, optionally, device output
buffers."""
import ctypes

import numpy as np

from . import _lib
from ._lib import (EOS, FSI, GHOST, OMEGA, PREC, VISC, WALL, LbmDiag, LbmInstanceDesc, LbmParams,
                   check)

_PARAM_KEYS = ("G", "sigma", "tau_rho", "tau_e", "tau_zeta", "tau_j", "tau_q", "tau_nu_L",
               "tau_nu_V", "rho_L", "rho_V", "rho_ref")


def default_params(**over):
    """Parameters of Sec. III as a dict (lbm_default_params), with overrides.
    EOS keys: kV, kM, kL (theta_V, theta_M, theta_L over cs^2), rho_1, rho_2."""
    p = LbmParams()
    check(_lib.load().lbm_default_params(ctypes.byref(p)))
    d = {k: getattr(p, k) for k in _PARAM_KEYS}
    d.update(kV=p.eos_p[0], kM=p.eos_p[1], kL=p.eos_p[2], rho_1=p.eos_p[3], rho_2=p.eos_p[4],
             wall="neq", ghost="copy", omega="w", prec="fp64", visc="tau")
    d.update(over)
    return d


def to_struct(d):
    p = LbmParams()
    check(_lib.load().lbm_default_params(ctypes.byref(p)))
    for k in _PARAM_KEYS:
        if k in d:
            setattr(p, k, float(d[k]))
    for j, k in enumerate(("kV", "kM", "kL", "rho_1", "rho_2")):
        if k in d:
            p.eos_p[j] = float(d[k])

    def enum(v, table):
        return table[v] if isinstance(v, str) else int(v)
    p.eos = enum(d.get("eos", "pl"), EOS)
    if p.eos == EOS["cs"]:
        # Carnahan-Starling: a, b, R, T
        for j, (k, v) in enumerate((("cs_a", 1.0), ("cs_b", 4.0), ("cs_R", 1.0), ("cs_T", None))):
            p.eos_p[j] = float(d[k] if k in d or v is None else v)
    p.visc = enum(d.get("visc", "tau"), VISC)
    p.wall = enum(d.get("wall", "neq"), WALL)
    p.ghost = enum(d.get("ghost", "copy"), GHOST)
    p.omega = enum(d.get("omega", "w"), OMEGA)
    p.prec = enum(d.get("prec", "fp64"), PREC)
    return p


def _stream_handle(stream):
    if stream is None:
        try:
            import torch
            if torch.cuda.is_available():
                return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
        except ImportError:
            pass
        return ctypes.c_void_p(0)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


class Lattice:
    """One context: a single lattice (lbm_create) or a batch (lbm_create_batch).

    instances: list of dicts with keys nx, ny, params, solid, fsi, gw."""

    def __init__(self, instances, stream=None):
        L = _lib.load()
        self._L = L
        self._keep = []
        n = len(instances)
        descs = (LbmInstanceDesc * n)()
        self.shapes = []
        for k, inst in enumerate(instances):
            nx, ny = int(inst["nx"]), int(inst["ny"])
            ps = to_struct(inst.get("params") or default_params())
            self._keep.append(ps)
            solid = inst.get("solid")
            if solid is not None:
                solid = np.ascontiguousarray(solid, dtype=np.uint8).reshape(ny, nx)
                self._keep.append(solid)
            gw = inst.get("gw", 0.0)
            gw_field = None
            if np.ndim(gw) != 0:
                gw_field = np.ascontiguousarray(gw, dtype=np.float64).reshape(ny, nx)
                self._keep.append(gw_field)
            fsi = inst.get("fsi", "modified")
            descs[k].nx, descs[k].ny = nx, ny
            descs[k].params = ctypes.pointer(ps)
            descs[k].solid = None if solid is None else solid.ctypes.data
            descs[k].fsi = FSI[fsi] if isinstance(fsi, str) else int(fsi)
            descs[k].gw_field = None if gw_field is None else gw_field.ctypes.data
            descs[k].gw_uniform = 0.0 if gw_field is not None else float(gw)
            self.shapes.append((ny, nx))
        h = ctypes.c_void_p()
        check(L.lbm_create_batch(n, descs, _stream_handle(stream), ctypes.byref(h)))
        self._h = h
        self._keep = []

    @classmethod
    def single(cls, nx, ny, params=None, solid=None, fsi="modified", gw=0.0, stream=None):
        return cls([dict(nx=nx, ny=ny, params=params, solid=solid, fsi=fsi, gw=gw)], stream)

    def close(self):
        if getattr(self, "_h", None):
            self._L.lbm_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def t(self):
        return self._L.lbm_time(self._h)

    def init_droplet(self, x0, y0, R, width=2.0, inst=0):
        check(self._L.lbm_init_droplet(self._h, inst, x0, y0, R, width))

    def set_density(self, rho, inst=0, sync=True):
        """Fluid at rest with density rho (lbm_set_density).  sync=False
        enqueues only (lbm_set_density_async): a host array must then be
        C-contiguous FP64 and stay unchanged until sync()."""
        fn = self._L.lbm_set_density if sync else self._L.lbm_set_density_async
        if hasattr(rho, "data_ptr") and rho.is_cuda:
            check(fn(self._h, inst, ctypes.c_void_p(rho.data_ptr()), 1))
        else:
            if not sync:
                assert rho.dtype == np.float64 and rho.flags.c_contiguous
            r = np.ascontiguousarray(rho, dtype=np.float64)
            check(fn(self._h, inst, r.ctypes.data, 0))

    def step(self, n=1):
        check(self._L.lbm_step(self._h, int(n)))

    def sync(self):
        check(self._L.lbm_sync(self._h))

    def set_launch(self, bx=0, h=0, persistent=False, graph=False, stages=0):
        """Launch shape and pipeline of step() (lbm_set_launch): stages 0
        automatic, 4 FP32 warp strips with two columns per lane (every width
        a multiple of 4; the automatic choice there), 2 warp strips (two rows
        per lane with FP32 storage), 3 warp strips one row per lane, 1 block
        rows, 8/16 block rows with a TMA ring.  persistent=True runs all
        steps of a call in one cooperative launch (warp strips, each waiting
        only on its neighbours; block rows with a grid barrier); graph=True
        replays the launches of a call from a CUDA graph."""
        check(self._L.lbm_set_launch(self._h, int(bx), int(h), int(persistent), int(graph),
                                     int(stages)))

    def launch(self):
        """The launch shape in use (lbm_get_launch): dict(bx, pipeline,
        persistent); pipeline 4 is the FP32 warp strips with two columns
        per lane, 2 the FP32 warp strips with two rows per lane, 3 the warp
        strips with one row per lane, 1 the block rows."""
        bx, pl, pe = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        check(self._L.lbm_get_launch(self._h, ctypes.byref(bx), ctypes.byref(pl),
                                          ctypes.byref(pe)))
        return dict(bx=bx.value, pipeline=pl.value, persistent=bool(pe.value))

    def fields(self, inst=0, device=False, out=None, sync=True):
        """rho, ux, uy of instance inst: numpy (host) or torch CUDA tensors
        (device=True); `out` may supply the three host arrays (e.g. pinned).
        With `out` and sync=False the read-back is only enqueued
        (lbm_get_fields_async): the arrays hold the fields after sync()."""
        ny, nx = self.shapes[inst]
        if out is not None:
            for k in ("rho", "ux", "uy"):
                a = out[k]
                assert a.dtype == np.float64 and a.shape == (ny, nx) and a.flags.c_contiguous
            fn = self._L.lbm_get_fields if sync else self._L.lbm_get_fields_async
            check(fn(self._h, inst, *[out[k].ctypes.data for k in ("rho", "ux", "uy")], 0))
            return out
        if device:
            import torch
            out = {k: torch.empty((ny, nx), dtype=torch.float64, device="cuda")
                   for k in ("rho", "ux", "uy")}
            check(self._L.lbm_get_fields(self._h, inst, *[ctypes.c_void_p(out[k].data_ptr())
                                                          for k in ("rho", "ux", "uy")], 1))
            return out
        out = {k: np.empty((ny, nx)) for k in ("rho", "ux", "uy")}
        check(self._L.lbm_get_fields(self._h, inst, *[out[k].ctypes.data
                                                      for k in ("rho", "ux", "uy")], 0))
        return out

    def populations(self, inst=0):
        ny, nx = self.shapes[inst]
        f = np.empty((9, ny, nx))
        check(self._L.lbm_get_populations(self._h, inst, f.ctypes.data, 0))
        return f

    def diagnostics(self, inst=0, y_w=0.5, x_ref=None, d_min=3.0):
        ny, nx = self.shapes[inst]
        d = LbmDiag()
        st = self._L.lbm_diagnostics(self._h, inst, float(y_w),
                                     float(nx / 2 if x_ref is None else x_ref), float(d_min),
                                     ctypes.byref(d))
        out = d.as_dict()
        out["status"] = st
        return out

    @property
    def total_nodes(self):
        return sum(nx * ny for ny, nx in self.shapes)

    def split(self, flat):
        """Per-instance [ny][nx] views of a field concatenated in instance
        order (the layout of the *_all calls)."""
        out, o = [], 0
        for ny, nx in self.shapes:
            out.append(flat[o:o + nx * ny].reshape(ny, nx))
            o += nx * ny
        return out

    def set_density_all(self, rho_flat):
        """Every instance at rest with the concatenated densities (FP64,
        C-contiguous); enqueued only.  A host array must stay unchanged until
        sync(); a torch CUDA tensor is read in the context's stream order."""
        if hasattr(rho_flat, "data_ptr") and rho_flat.is_cuda:
            import torch
            assert rho_flat.dtype == torch.float64 and rho_flat.is_contiguous()
            assert rho_flat.numel() == self.total_nodes
            check(self._L.lbm_set_density_all_async(self._h, ctypes.c_void_p(rho_flat.data_ptr()),
                                                    1))
            return
        assert rho_flat.dtype == np.float64 and rho_flat.flags.c_contiguous
        assert rho_flat.size == self.total_nodes
        check(self._L.lbm_set_density_all_async(self._h, rho_flat.ctypes.data, 0))

    def fields_all(self, out):
        """Enqueue the read-back of rho, ux, uy of every instance into the
        concatenated FP64 host arrays out["rho"|"ux"|"uy"]; valid after sync()."""
        for k in ("rho", "ux", "uy"):
            a = out[k]
            assert a.dtype == np.float64 and a.flags.c_contiguous and a.size == self.total_nodes
        check(self._L.lbm_get_fields_all_async(self._h, *[out[k].ctypes.data
                                                          for k in ("rho", "ux", "uy")], 0))
        return out

    def contact_radius(self, inst=0, row=1, level=0.0, x_ref=None):
        """Spreading radius along node row `row` (lbm_contact_radius); level
        0 means (rho_L + rho_V) / 2."""
        ny, nx = self.shapes[inst]
        r = ctypes.c_double()
        check(self._L.lbm_contact_radius(self._h, inst, int(row), float(level),
                                         float(nx / 2 if x_ref is None else x_ref),
                                         ctypes.byref(r)))
        return r.value

    def set_gw_field(self, gw, inst=0):
        g = np.ascontiguousarray(gw, dtype=np.float64)
        check(self._L.lbm_set_gw_field(self._h, inst, g.ctypes.data))

    def adjoint(self, T, theta_target, y_w=0.5, x_ref=None, d_min=3.0, want_grad=True):
        """T steps from the current state, loss (theta - theta_target)^2 and its
        gradient with respect to the G_w field (lbm_adjoint).  Returns
        (loss, theta, grad[ny][nx] or None)."""
        ny, nx = self.shapes[0]
        loss = ctypes.c_double()
        theta = ctypes.c_double()
        grad = np.zeros((ny, nx)) if want_grad else None
        check(self._L.lbm_adjoint(self._h, int(T), float(theta_target), float(y_w),
                                  float(nx / 2 if x_ref is None else x_ref), float(d_min),
                                  ctypes.byref(loss), ctypes.byref(theta),
                                  None if grad is None else grad.ctypes.data))
        return loss.value, theta.value, grad

    def save(self, path):
        check(self._L.lbm_save(self._h, str(path).encode()))

    def load(self, path):
        check(self._L.lbm_load(self._h, str(path).encode()))

    def autotune(self, steps=20):
        """Pick the fastest launch shape for these lattices, per-step or
        persistent (lbm_autotune); returns dict(bx, h, stages, persistent,
        ms_per_step)."""
        bx, h, st = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        ms = ctypes.c_double()
        check(self._L.lbm_autotune(self._h, int(steps), ctypes.byref(bx), ctypes.byref(h),
                                   ctypes.byref(st), ctypes.byref(ms)))
        return dict(bx=bx.value, h=h.value, stages=st.value,
                    persistent=self.launch()["persistent"], ms_per_step=ms.value)
