"""Run-to-run determinism, the race check that stands in for a sanitizer:
the same case run twice in fresh contexts, in every pipeline, gives
bit-identical populations (a data race would show as run-to-run noise)."""
import numpy as np
import pytest

import paper_1410_2569_gb300 as lbm
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu


def _run(prec, launch):
    specs = []
    # widths multiples of 4: the FP32 default is the column-pair strips,
    # stages=2 the row-pair strips
    for fsi, gw, nx, ny in [("density", 0.07, 96, 48), ("psi", 0.75, 132, 40),
                            ("modified", -0.1, 36, 20)]:
        solid = inputs.flat_walls(nx, ny)
        specs.append(dict(nx=nx, ny=ny, params=lbm.default_params(prec=prec), solid=solid,
                          fsi=fsi, gw=inputs.wall_gw(solid, gw)))
    lat = lbm.Lattice(specs)
    lat.set_launch(**launch)
    for k, s in enumerate(specs):
        lat.init_droplet(s["nx"] / 2, 0.5, s["ny"] / 3, 2.0, inst=k)
    lat.step(300)
    out = [lat.populations(k) for k in range(len(specs))]
    lat.close()
    return out


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
@pytest.mark.parametrize("launch", [dict(), dict(stages=2), dict(stages=3), dict(stages=1),
                                    dict(persistent=True), dict(stages=1, persistent=True),
                                    dict(graph=True)])
def test_same_case_twice_is_bit_identical(cuda, prec, launch):
    a, b = _run(prec, launch), _run(prec, launch)
    for k, (x, y) in enumerate(zip(a, b)):
        assert np.array_equal(x, y), (k, prec, launch)
