"""The bench workload at full size, in the launch configuration bench.py
times: the 72-lattice sweep (400 x 200 each) as one batched context.  Sampled
lattices are checked against the FP64 oracle run on their own."""
import numpy as np
import pytest

import oracle
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu

NX, NY, R, STEPS = 400, 200, 50.0, 60
SAMPLES = [0, 23, 31, 47, 71]  # density, psi, modified; both viscosity ratios


def _sweep(prec):
    import bench
    import paper_1410_2569_gb300 as lbm
    insts = bench.sweep_instances(prec)
    lat = lbm.Lattice(insts)
    for k in range(len(insts)):
        lat.init_droplet(NX / 2, 0.5, R, inputs.SWEEP_WIDTH, inst=k)
    lat.step(STEPS)
    lat.sync()
    return lat


def _oracle(k):
    c = inputs.sweep_cases()[k]
    oracle.set_threads(8)
    p = oracle.paper_params(tau_nu_L=c["tau_nu_L"], tau_nu_V=c["tau_nu_V"])
    solid = inputs.flat_walls(NX, NY)
    o = oracle.Lattice(NX, NY, p, solid, c["fsi"], inputs.wall_gw(solid, c["gw"]))
    o.init_droplet(NX / 2, 0.5, R, inputs.SWEEP_WIDTH)
    o.step(STEPS)
    return o.fields()


@pytest.fixture(scope="module")
def oracle_fields():
    return {k: _oracle(k) for k in SAMPLES}


@pytest.mark.parametrize("prec,tol", [("fp64", 1e-10), ("fp32", 1e-4)])
def test_sweep_batch_matches_oracle_on_sampled_lattices(cuda, oracle_fields, prec, tol):
    lat = _sweep(prec)
    fluid = inputs.flat_walls(NX, NY) == 0
    for k in SAMPLES:
        g, o = lat.fields(k), oracle_fields[k]
        err = np.max(np.abs(g["rho"][fluid] - o["rho"][fluid]) / o["rho"][fluid])
        assert err <= tol, (prec, k, err)
