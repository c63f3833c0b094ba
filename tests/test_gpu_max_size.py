"""The largest lattice the step's 32-bit offsets allow (9 nx ny just below
2^31): a droplet hanging from the top wall across the periodic seam, at the
highest node indices, evolves bit for bit as the same droplet on a small
lattice.  A node's step reads psi of its neighbours, which were pulled
from one node further, so influence travels at most two nodes per step:
after 20 steps the top 70 rows within 80 columns of the seam see only the
droplet, the top wall and the vapour, the same in both lattices."""
import numpy as np
import pytest

import paper_1410_2569_gb300 as lbm
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu

NX = 16384
NY = (2 ** 31 - 1) // (9 * NX)  # 14563
STEPS, ROWS, HALF = 20, 70, 80
SX, SY = 256, 128


def _run(nx, ny, prec):
    lat = lbm.Lattice.single(nx, ny, lbm.default_params(prec=prec), inputs.flat_walls(nx, ny),
                             "modified", 0.1)
    # centred on the top wall surface, 10 nodes left of the seam
    lat.init_droplet(nx - 10.0, ny - 1.5, 12.0, 2.0)
    lat.step(STEPS)
    rho = lat.fields()["rho"]
    lat.close()
    # the top rows, columns [nx - HALF, nx) followed by [0, HALF)
    cols = np.r_[nx - HALF:nx, 0:HALF]
    return rho[ny - ROWS:, cols]


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_largest_lattice_matches_small_one(cuda, prec):
    assert 9 * NX * NY < 2 ** 31 <= 9 * NX * (NY + 1)
    small = _run(SX, SY, prec)
    big = _run(NX, NY, prec)
    assert np.isfinite(big).all() and big.max() > 400.0
    assert np.array_equal(big, small)
