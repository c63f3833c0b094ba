"""Spurious currents of Sec. III.C (Figs. 9-11), modified interaction,
300 x 100 lattice, R = 30, 30000 FP64 steps (the step is tied to the oracle
by the parity tests).  Checked, on the liquid phase (rho above the mean of
rho_L and rho_V), where the currents settle to steady values:
  * they fall as the kinematic viscosity ratio nu_V / nu_L rises through
    1, 5 and 10 with nu_L = 1/30 (Fig. 10);
  * G_w = 0 gives the smallest currents (Fig. 9), at tau_nu = 0.6, 0.8, 1.1;
  * at G_w = 0 they grow as tau_nu falls (Fig. 9);
  * they are much smaller than in the vapour (Fig. 11).
The printed liquid maximum of about 0.012 (G_w = 0.4, ratio 10) is not
reproduced: with tau_nu linear in rho that droplet detaches at ratios 5
and 10; at G_w = 0.2 the liquid maximum is about 0.0014.  With the dynamic
viscosity rho nu linear in rho instead (LBM_VISC_MU_LINEAR, the other
reading of Sec. III.C) the G_w = 0.4 droplet stays on the wall at ratio 10,
as Fig. 11(b) shows it; that reading is parity-tested at ratio 5 against
the oracle, and its liquid maximum is compared with the oracle's.
"""
import numpy as np
import pytest

import paper_1410_2569_gb300 as lbm
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu

NX, NY, R, STEPS = 300, 100, 30.0, 30000
NU_L = 1.0 / 30.0
GWS = (-0.2, 0.0, 0.2)


def _cases():
    out = []
    for gw in GWS:
        for ratio in (1, 5, 10):
            out.append((("ratio", gw, ratio), 0.5 + 3 * NU_L, 0.5 + 3 * NU_L * ratio, gw))
        for tau in (0.8, 1.1):
            out.append((("tau", gw, tau), tau, tau, gw))
    return out


@pytest.fixture(scope="module")
def currents(cuda):
    flat = inputs.flat_walls(NX, NY)
    cases = _cases()
    lat = lbm.Lattice([dict(nx=NX, ny=NY, solid=flat, fsi="modified", gw=inputs.wall_gw(flat, gw),
                            params=lbm.default_params(prec="fp64", tau_nu_L=tl, tau_nu_V=tv))
                       for (_, tl, tv, gw) in cases])
    for k in range(len(cases)):
        lat.init_droplet(NX / 2, 0.5, R, 4.0, inst=k)
    lat.step(STEPS)
    out = {}
    fluid = flat == 0
    for k, c in enumerate(cases):
        f = lat.fields(k)
        u = np.hypot(f["ux"], f["uy"])
        liq = f["rho"] > 250.5
        out[c[0]] = (u[liq].max(), u[fluid & ~liq].max())
    lat.close()
    return out


def test_liquid_currents_fall_with_viscosity_ratio(currents):
    for gw in GWS:
        u = [currents[("ratio", gw, r)][0] for r in (1, 5, 10)]
        assert u[0] > u[1] > u[2], (gw, u)


def test_neutral_wall_gives_smallest_currents(currents):
    for tau_key in [("ratio", 1)] + [("tau", t) for t in (0.8, 1.1)]:
        u = {gw: currents[(tau_key[0], gw, tau_key[1])][0] for gw in GWS}
        assert u[0.0] < min(u[-0.2], u[0.2]), (tau_key, u)


def test_currents_grow_as_tau_falls(currents):
    u = [currents[("ratio", 0.0, 1)][0], currents[("tau", 0.0, 0.8)][0],
         currents[("tau", 0.0, 1.1)][0]]  # tau_nu = 0.6, 0.8, 1.1
    assert u[0] > u[1] > u[2], u


def test_liquid_currents_below_vapour(currents):
    for key, (ul, uv) in currents.items():
        assert ul < 0.5 * uv, (key, ul, uv)


@pytest.mark.parametrize("visc", ["tau", "mu"])
def test_viscosity_ratio_5_parity(cuda, visc):
    """Density-dependent viscosity at nu_V / nu_L = 5 (Sec. III.C) under
    both readings: FP64 within 1e-10 of the oracle after 1000 steps, FP32
    density within 1e-4."""
    from helpers import field_errors, run_gpu, run_oracle
    nx, ny, steps = 100, 60, 1000
    solid = inputs.flat_walls(nx, ny)
    gw = inputs.wall_gw(solid, 0.2)
    drop = (50.0, 0.5, 20.0, 4.0)
    over = dict(tau_nu_L=0.5 + 3 * NU_L, tau_nu_V=0.5 + 3 * NU_L * 5, visc=visc)
    o = run_oracle(nx, ny, steps, "modified", gw, solid, drop, **over)
    g = run_gpu(nx, ny, steps, "modified", gw, solid, drop, **over)
    e = field_errors(g, o, solid)
    assert e["rho"] <= 1e-10 and e["f"] <= 1e-10 and e["u"] <= 1e-10, e
    g32 = run_gpu(nx, ny, steps, "modified", gw, solid, drop, prec="fp32", **over)
    fluid = solid == 0
    ro, rg = o.fields()["rho"][fluid], g32.fields()["rho"][fluid]
    assert np.max(np.abs(rg - ro) / ro) <= 1e-4


def test_mu_linear_keeps_the_gw04_droplet_on_the_wall(cuda):
    """G_w = 0.4, nu_V / nu_L = 10 (Fig. 11b): with tau_nu linear in rho the
    droplet leaves the wall (180 deg), with mu linear in rho it stays; both
    at 20,000 steps of the FP32 step."""
    flat = inputs.flat_walls(NX, NY)
    theta = {}
    for visc in ("tau", "mu"):
        lat = lbm.Lattice.single(NX, NY, lbm.default_params(prec="fp32", tau_nu_L=0.5 + 3 * NU_L,
                                                             tau_nu_V=0.5 + 3 * NU_L * 10,
                                                             visc=visc),
                                 flat, "modified", inputs.wall_gw(flat, 0.4))
        lat.init_droplet(NX / 2, 0.5, R, 4.0)
        lat.step(20000)
        theta[visc] = lat.diagnostics(y_w=0.5, x_ref=NX / 2)["theta_deg"]
        lat.close()
    assert theta["tau"] == 180.0 and theta["mu"] < 175.0, theta


def test_liquid_current_matches_oracle(cuda):
    """The liquid-phase maximum of |v| (rho above (rho_L + rho_V) / 2) of the
    G_w = 0.4, ratio 10 droplet under the mu-linear reading, FP64 step
    against the oracle after 5000 steps, to 1e-8 relative."""
    import oracle
    from helpers import run_gpu
    flat = inputs.flat_walls(NX, NY)
    gw = inputs.wall_gw(flat, 0.4)
    over = dict(tau_nu_L=0.5 + 3 * NU_L, tau_nu_V=0.5 + 3 * NU_L * 10, visc="mu")
    oracle.set_threads(16)
    o = oracle.Lattice(NX, NY, oracle.paper_params(**over), flat, "modified", gw)
    o.init_droplet(NX / 2, 0.5, R, 4.0)
    o.step(5000)
    g = run_gpu(NX, NY, 5000, "modified", gw, flat, (NX / 2, 0.5, R, 4.0), **over)
    vals = []
    for f in (o.fields(), g.fields()):
        u = np.hypot(f["ux"], f["uy"])
        vals.append(u[f["rho"] > 250.5].max())
    assert vals[0] > 1e-4
    assert abs(vals[1] - vals[0]) <= 1e-8 * vals[0], vals
