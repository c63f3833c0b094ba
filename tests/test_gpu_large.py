"""The large workload at full size: 8192 x 4096, striped bottom wall, 2000
droplets, modified interaction; the first steps in FP64 and FP32 against the
FP64 oracle on the whole lattice."""
import numpy as np
import pytest

import oracle
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu

STEPS = 6


@pytest.fixture(scope="module")
def case():
    nx, ny = 8192, 4096
    solid, gw, drops = inputs.large_striped(nx, ny, 2000, seed=0)
    assert len(drops) == 2000
    rho0 = inputs.droplet_field(nx, ny, drops, 4.0)
    oracle.set_threads(16)
    o = oracle.Lattice(nx, ny, oracle.paper_params(), solid, "modified", gw)
    o.set_density(rho0)
    o.step(STEPS)
    ref = o.fields()["rho"]
    del o
    return nx, ny, solid, gw, rho0, ref


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_large_striped_lattice_matches_oracle(cuda, case, prec, tol):
    import paper_1410_2569_gb300 as lbm
    nx, ny, solid, gw, rho0, ref = case
    lat = lbm.Lattice.single(nx, ny, lbm.default_params(prec=prec), solid, "modified", gw)
    lat.set_density(rho0)
    lat.step(STEPS)
    got = lat.fields()["rho"]
    lat.close()
    fluid = solid == 0
    err = np.max(np.abs(got[fluid] - ref[fluid]) / ref[fluid])
    assert err <= tol, err
