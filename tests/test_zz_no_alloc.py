"""lbm_diagnostics_noalloc: diagnostics for callers that cannot call
cudaMalloc (device memory owned entirely by the caller's own allocator, or
a loop that must not pay the synchronisation an allocation can imply).

The entry point keeps its scratch in a fixed array inside the library, so
two calls in a row share it; each call is checked against lbm_diagnostics
on the same lattice state.  This file is collected last on purpose."""
import ctypes

import pytest

pytestmark = pytest.mark.gpu


def _ptr(t):
    return ctypes.c_void_p(t.data_ptr())


def test_noalloc_matches_diagnostics_on_two_calls_in_a_row(cuda):
    import torch

    import paper_1410_2569_gb300 as lbm
    from paper_1410_2569_gb300 import inputs
    from paper_1410_2569_gb300._lib import LbmDiag

    nx, ny, x_ref, y_w = 120, 64, 60.0, 0.5
    solid = inputs.flat_walls(nx, ny)
    p = lbm.default_params()
    lat = lbm.Lattice.single(nx, ny, p, solid, "modified", 0.2)
    lat.init_droplet(x_ref, y_w, 22.0, 2.0)
    L = lbm.load()
    d_solid = torch.from_numpy(solid).to("cuda")
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    level = 0.5 * (p["rho_L"] + p["rho_V"])
    for call in range(2):
        lat.step(300)
        ref = lat.diagnostics(y_w=y_w, x_ref=x_ref, d_min=3.0)
        f = lat.fields(device=True)
        torch.cuda.synchronize()
        out = LbmDiag()
        st = L.lbm_diagnostics_noalloc(nx, ny, _ptr(f["rho"]), _ptr(f["ux"]), _ptr(f["uy"]),
                                       _ptr(d_solid), level, y_w, x_ref, 3.0, stream,
                                       ctypes.byref(out))
        assert st == 0, L.lbm_last_error()
        got = out.as_dict()
        assert ref["status"] == 0 and got["status"] == 0
        assert got["n_contour"] == ref["n_contour"] > 20, call
        assert abs(got["mass"] - ref["mass"]) <= 1e-11 * ref["mass"], call
        for k in ("rho_max", "rho_min", "u_max", "radius", "xc", "yc", "fit_rms"):
            assert abs(got[k] - ref[k]) <= 1e-9 * max(1.0, abs(ref[k])), (call, k, got[k], ref[k])
        assert abs(got["theta_deg"] - ref["theta_deg"]) <= 1e-8, call


def test_noalloc_without_a_solid_mask(cuda):
    """solid = NULL: a lattice with no solid nodes (a free droplet, periodic
    both ways), compared with lbm_diagnostics on the same state, two calls
    in a row."""
    import torch

    import paper_1410_2569_gb300 as lbm
    from paper_1410_2569_gb300._lib import LbmDiag

    nx, ny, x_ref, y_w = 96, 80, 48.0, 40.0
    p = lbm.default_params()
    lat = lbm.Lattice.single(nx, ny, p, None, "modified", 0.0)
    lat.init_droplet(x_ref, y_w, 18.0, 2.0)
    L = lbm.load()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    level = 0.5 * (p["rho_L"] + p["rho_V"])
    for call in range(2):
        lat.step(200)
        ref = lat.diagnostics(y_w=y_w, x_ref=x_ref, d_min=3.0)
        f = lat.fields(device=True)
        torch.cuda.synchronize()
        out = LbmDiag()
        st = L.lbm_diagnostics_noalloc(nx, ny, _ptr(f["rho"]), _ptr(f["ux"]), _ptr(f["uy"]),
                                       None, level, y_w, x_ref, 3.0, stream, ctypes.byref(out))
        assert st == 0, L.lbm_last_error()
        got = out.as_dict()
        assert got["status"] == ref["status"], call
        assert got["n_contour"] == ref["n_contour"] > 20, call
        assert abs(got["mass"] - ref["mass"]) <= 1e-11 * ref["mass"], call
        for k in ("rho_max", "rho_min", "u_max", "radius", "xc", "yc", "fit_rms", "theta_deg"):
            assert abs(got[k] - ref[k]) <= 1e-9 * max(1.0, abs(ref[k])), (call, k, got[k], ref[k])


def test_noalloc_rejects_sizes_beyond_its_limit(cuda):
    import torch

    import paper_1410_2569_gb300 as lbm
    from paper_1410_2569_gb300._lib import LbmDiag

    L = lbm.load()
    out = LbmDiag()
    small = torch.zeros(16, dtype=torch.float64, device="cuda")  # rejected before any use
    st = L.lbm_diagnostics_noalloc(1 << 15, 1 << 14, _ptr(small), _ptr(small), _ptr(small), None,
                                   250.5, 0.5, 0.0, 3.0, None, ctypes.byref(out))
    assert st == 1  # LBM_ERR_ARG
    assert b"nx * ny" in L.lbm_last_error()
