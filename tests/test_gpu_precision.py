"""FP32 storage against the FP64 oracle on a settled sessile droplet: the
gates of the metric (density within 1e-4 relative, contact angle within
0.5 deg), for storage shifts rho_ref = 0, rho_V and rho_L and for the mode
that sums the density in FP64 instructions.  A shift of rho_L stores the
vapour populations as small differences of large numbers, so its vapour
error is larger; the angle gate still holds."""
import numpy as np
import pytest

from helpers import run_gpu, run_oracle
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu

NX, NY, STEPS = 150, 80, 3000
DROP = (75.0, 0.5, 25.0, 2.0)


@pytest.fixture(scope="module")
def reference():
    solid = inputs.flat_walls(NX, NY)
    gw = inputs.wall_gw(solid, 0.1)
    o = run_oracle(NX, NY, STEPS, "modified", gw, solid, DROP, threads=8)
    return solid, gw, o.fields()["rho"], o.diagnostics(0.5, NX / 2, 3.0)


@pytest.mark.parametrize("prec,rho_ref,rho_tol", [("fp32", 0.0, 1e-4), ("fp32", 1.0, 1e-4),
                                                  ("fp32", 500.0, 1e-3), ("fp32_f64", 1.0, 1e-4)])
def test_fp32_gates(cuda, reference, prec, rho_ref, rho_tol):
    solid, gw, ro, do = reference
    g = run_gpu(NX, NY, STEPS, "modified", gw, solid, DROP, prec=prec, rho_ref=rho_ref)
    fluid = solid == 0
    err = np.max(np.abs(g.fields()["rho"][fluid] - ro[fluid]) / ro[fluid])
    assert err <= rho_tol, err
    dg = g.diagnostics(y_w=0.5, x_ref=NX / 2, d_min=3.0)
    assert do["status"] == 0 and dg["status"] == 0
    assert abs(dg["theta_deg"] - do["theta_deg"]) <= 0.5, (dg["theta_deg"], do["theta_deg"])
