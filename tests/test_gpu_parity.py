"""CUDA step vs the FP64 CPU oracle, element by element (FP64: max relative
field error <= 1e-10 after 1000 steps)."""
import numpy as np
import pytest

from helpers import field_errors, run_gpu, run_oracle
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu

FSI_GW = [("density", 0.07), ("psi", 1.0), ("modified", 0.1), ("modified", -0.2)]


@pytest.mark.parametrize("fsi,gw", FSI_GW)
@pytest.mark.parametrize("wall,ghost", [("neq", "copy"), ("bb", "copy"), ("neq", "mirror"),
                                        ("bb", "skip"), ("neq", "zero")])
def test_fp64_matches_oracle_100x60(cuda, fsi, gw, wall, ghost):
    nx, ny, steps = 100, 60, 1000
    drop = (50.0, 1.0, 20.0, 2.0)
    solid = inputs.flat_walls(nx, ny)
    o = run_oracle(nx, ny, steps, fsi, gw, solid, drop, wall=wall, ghost=ghost)
    g = run_gpu(nx, ny, steps, fsi, gw, solid, drop, wall=wall, ghost=ghost)
    e = field_errors(g, o, solid)
    assert e["rho"] <= 1e-10, e
    assert e["f"] <= 1e-10, e
    assert e["u"] <= 1e-10, e


@pytest.mark.parametrize("bx,h", [(32, 7), (64, 13), (128, 64), (0, 0)])
def test_tiles_and_ragged_edges(cuda, bx, h):
    # 77 x 45: several tiles and ragged tails in both directions
    nx, ny, steps = 77, 45, 300
    drop = (30.0, 1.0, 14.0, 2.0)
    solid = inputs.flat_walls(nx, ny)
    o = run_oracle(nx, ny, steps, "modified", 0.15, solid, drop)
    g = run_gpu(nx, ny, steps, "modified", 0.15, solid, drop, launch=dict(bx=bx, h=h))
    e = field_errors(g, o, solid)
    assert e["rho"] <= 1e-10 and e["f"] <= 1e-10 and e["u"] <= 1e-10, e


def test_tile_shape_is_bit_identical(cuda):
    nx, ny = 96, 50
    solid = inputs.flat_walls(nx, ny)
    drop = (48.0, 1.0, 16.0, 2.0)
    ref = run_gpu(nx, ny, 200, "psi", 1.5, solid, drop, launch=dict(bx=96, h=50)).populations()
    for bx, h in ((32, 5), (64, 17), (128, 3)):
        got = run_gpu(nx, ny, 200, "psi", 1.5, solid, drop, launch=dict(bx=bx, h=h)).populations()
        assert np.array_equal(got, ref), (bx, h)


@pytest.mark.parametrize("fsi,gw,ghost", [("density", 0.2, "skip"), ("modified", 0.3, "skip"),
                                          ("density", 0.2, "mean"), ("modified", 0.3, "mean"),
                                          ("psi", 1.5, "mean")])
def test_rough_surface_bounce_back(cuda, fsi, gw, ghost):
    # square pillars (Sec. III.B): halfway bounce-back, Eq. (7) either not
    # applied next to the wall or applied with the MEAN ghost layer, droplet
    # resting on the pillar tops
    nx, ny = 90, 60
    solid = inputs.pillars(nx, ny, height=10, width=6, gap=3)
    drop = (45.0, 30.0, 15.0, 2.0)
    gwf = inputs.wall_gw(solid, gw)
    o = run_oracle(nx, ny, 400, fsi, gwf, solid, drop, wall="bb", ghost=ghost)
    g = run_gpu(nx, ny, 400, fsi, gwf, solid, drop, wall="bb", ghost=ghost)
    e = field_errors(g, o, solid)
    assert e["rho"] <= 1e-10 and e["f"] <= 1e-10 and e["u"] <= 1e-10, e


# Carnahan-Starling option at T = 0.7 T_c (rho_L / rho_V about 38)
CS = dict(eos="cs", cs_T=0.7 * 0.3773 / 4.0, rho_L=0.358, rho_V=0.0093)


@pytest.mark.parametrize("fsi,gw", [("density", 0.05), ("modified", 0.2), ("psi", 0.05)])
def test_carnahan_starling_fp64_matches_oracle(cuda, fsi, gw):
    nx, ny, steps = 100, 60, 1000
    drop = (50.0, 1.0, 20.0, 3.0)
    solid = inputs.flat_walls(nx, ny)
    o = run_oracle(nx, ny, steps, fsi, gw, solid, drop, **CS)
    g = run_gpu(nx, ny, steps, fsi, gw, solid, drop, **CS)
    assert np.isfinite(o.fields()["rho"]).all()
    e = field_errors(g, o, solid)
    assert e["rho"] <= 1e-10 and e["f"] <= 1e-10 and e["u"] <= 1e-10, e


@pytest.mark.parametrize("prec", ["fp32", "fp32_f64"])
def test_carnahan_starling_fp32_density(cuda, prec):
    nx, ny, steps = 100, 60, 1000
    drop = (50.0, 1.0, 20.0, 3.0)
    solid = inputs.flat_walls(nx, ny)
    o = run_oracle(nx, ny, steps, "modified", 0.2, solid, drop, **CS)
    g = run_gpu(nx, ny, steps, "modified", 0.2, solid, drop, prec=prec, rho_ref=CS["rho_V"], **CS)
    fluid = solid == 0
    ro, rg = o.fields()["rho"][fluid], g.fields()["rho"][fluid]
    assert np.max(np.abs(rg - ro) / ro) <= 1e-4
