"""Argument validation of the C ABI, on the CPU: every rejected creation
returns LBM_ERR_ARG with a message before any device work (lbm_create_batch
checks all instances before its first allocation)."""
import numpy as np
import pytest

import paper_1410_2569_gb300 as lbm
from paper_1410_2569_gb300 import inputs

ERR_ARG = 1


def _create(nx, ny, solid=None, fsi="modified", gw=0.0, **over):
    return lbm.Lattice.single(nx, ny, lbm.default_params(**over), solid, fsi, gw)


def _rejected(fn, *args, match=None, **kw):
    with pytest.raises(lbm.LbmError) as ei:
        fn(*args, **kw)
    assert ei.value.status == ERR_ARG, ei.value
    if match:
        assert match in str(ei.value), str(ei.value)


def test_size_limit_of_32bit_offsets():
    nx = 16384
    ny = (2 ** 31 - 1) // (9 * nx) + 1  # 9 nx ny reaches 2^31
    _rejected(_create, nx, ny, match="too large")


@pytest.mark.parametrize("nx,ny", [(2, 10), (10, 3), (0, 0)])
def test_too_small(nx, ny):
    _rejected(_create, nx, ny, match="at least")


@pytest.mark.parametrize("over,match", [
    (dict(G=1.0), "G must be negative"),
    (dict(rho_1=500.0, rho_2=400.0), "rho_1 < rho_2"),
    (dict(eos="cs", cs_T=0.0), "Carnahan-Starling"),
    (dict(tau_nu_L=0.5), "relaxation times"),
    (dict(tau_e=0.3), "relaxation times"),
    (dict(rho_L=0.5), "rho_L > rho_V"),
    (dict(sigma=-0.1), "sigma"),
    (dict(ghost=7), "unknown ghost"),
    (dict(wall=3), "unknown wall"),
])
def test_bad_parameters(over, match):
    _rejected(_create, 40, 30, **over)


def test_wall_rule_needs_whole_solid_rows():
    solid = inputs.pillars(40, 30, height=5, width=4, gap=3)
    _rejected(_create, 40, 30, solid=solid, wall="neq", ghost="zero", match="partly solid")
    _rejected(_create, 40, 30, solid=solid, wall="bb", ghost="copy", match="partly solid")


def test_copy_ghost_needs_two_row_walls():
    solid = np.zeros((30, 40), np.uint8)
    solid[10, :] = 1  # one solid row with fluid on both sides
    _rejected(_create, 40, 30, solid=solid, match="two rows thick")


def test_fluid_between_solid_rows_rejected():
    solid = inputs.flat_walls(40, 30)
    solid[2, :] = 1  # row 1 is fluid between solid rows 0 and 2
    _rejected(_create, 40, 30, solid=solid, wall="bb", ghost="zero", match="above and below")


def test_batch_precision_must_agree():
    specs = [dict(nx=40, ny=30, params=lbm.default_params(prec="fp64"),
                  solid=inputs.flat_walls(40, 30), fsi="density", gw=0.0),
             dict(nx=40, ny=30, params=lbm.default_params(prec="fp32"),
                  solid=inputs.flat_walls(40, 30), fsi="density", gw=0.0)]
    _rejected(lbm.Lattice, specs, match="share the precision")


def test_non_finite_gw_rejected():
    solid = inputs.flat_walls(40, 30)
    gw = inputs.wall_gw(solid, 0.1)
    gw[0, 5] = np.nan
    _rejected(_create, 40, 30, solid=solid, gw=gw, match="non-finite G_w")


def test_empty_batch_rejected():
    _rejected(lbm.Lattice, [], match="count > 0")


def test_null_context_rejected():
    """Every entry point taking a context checks it before anything else."""
    import ctypes
    L = lbm.load()
    d = ctypes.c_double()
    assert L.lbm_step(None, 1) == ERR_ARG
    assert L.lbm_sync(None) == ERR_ARG
    assert L.lbm_get_fields(None, 0, None, None, None, 0) == ERR_ARG
    assert L.lbm_contact_radius(None, 0, 1, 0.0, 0.0, ctypes.byref(d)) == ERR_ARG
    assert L.lbm_set_launch(None, 0, 0, 0, 0, 0) == ERR_ARG
    assert L.lbm_time(None) == -1
