"""Shared test helpers: run the same seeded case on the oracle and on the
CUDA library and compare element by element."""
import numpy as np

import oracle
from paper_1410_2569_gb300 import inputs


def oracle_params(**over):
    return oracle.paper_params(**over)


def gpu_params(**over):
    import paper_1410_2569_gb300 as lbm
    return lbm.default_params(**over)


def run_oracle(nx, ny, steps, fsi, gw, solid=None, drop=None, threads=4, **over):
    oracle.set_threads(threads)
    solid = inputs.flat_walls(nx, ny) if solid is None else solid
    o = oracle.Lattice(nx, ny, oracle_params(**over), solid, fsi, gw)
    x0, y0, R, W = drop if drop is not None else (nx / 2, 1.0, ny / 3, 2.0)
    o.init_droplet(x0, y0, R, W)
    o.step(steps)
    return o


def run_gpu(nx, ny, steps, fsi, gw, solid=None, drop=None, launch=None, **over):
    import paper_1410_2569_gb300 as lbm
    solid = inputs.flat_walls(nx, ny) if solid is None else solid
    g = lbm.Lattice.single(nx, ny, gpu_params(**over), solid, fsi, gw)
    if launch:
        g.set_launch(**launch)
    x0, y0, R, W = drop if drop is not None else (nx / 2, 1.0, ny / 3, 2.0)
    g.init_droplet(x0, y0, R, W)
    g.step(steps)
    return g


def rel_err(a, b, floor=0.0):
    """max |a - b| / max(|b|, floor) over all elements"""
    a = np.asarray(a)
    b = np.asarray(b)
    den = np.maximum(np.abs(b), floor)
    with np.errstate(divide="ignore", invalid="ignore"):
        r = np.where(den > 0, np.abs(a - b) / np.where(den > 0, den, 1.0), np.abs(a - b))
    return float(np.max(r))


def field_errors(g, o, solid):
    gf, of = g.fields(), o.fields()
    fluid = solid == 0
    umax = max(np.max(np.abs(of["ux"][fluid])), np.max(np.abs(of["uy"][fluid])), 1e-300)
    gp, op = g.populations(), o.populations()
    return {
        "rho": rel_err(gf["rho"][fluid], of["rho"][fluid]),
        "u": max(np.max(np.abs(gf["ux"][fluid] - of["ux"][fluid])),
                 np.max(np.abs(gf["uy"][fluid] - of["uy"][fluid]))) / umax,
        "f": rel_err(gp[:, fluid], op[:, fluid], floor=1e-2),
    }
