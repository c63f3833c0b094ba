"""lbm_set_density_async / lbm_get_fields_async: queued for several
instances back to back (the context's scratch fields are reused in stream
order), they give exactly what the synchronising calls give."""
import numpy as np
import pytest
import torch

import paper_1410_2569_gb300 as lbm
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu


def _batch(prec):
    specs = []
    for k, (nx, ny) in enumerate([(64, 40), (96, 48), (33, 20), (130, 36)]):
        solid = inputs.flat_walls(nx, ny)
        specs.append(dict(nx=nx, ny=ny, params=lbm.default_params(prec=prec), solid=solid,
                          fsi=("density", "psi", "modified", "modified")[k],
                          gw=inputs.wall_gw(solid, (0.1, -0.8, 0.2, -0.1)[k])))
    return specs


def _density(nx, ny, k):
    yy, xx = np.mgrid[0:ny, 0:nx]
    r = np.sqrt((xx - nx / 2) ** 2 + (yy - 0.5) ** 2)
    return 1.0 + 0.5 * 499.0 * (1.0 - np.tanh(2.0 * (r - (8 + 2 * k)) / 2.0))


def _pinned(shape):
    return torch.empty(shape, dtype=torch.float64).pin_memory().numpy()


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_async_calls_match_sync(cuda, prec):
    specs = _batch(prec)
    rhos = []
    for k, s in enumerate(specs):
        r = _pinned((s["ny"], s["nx"]))
        r[:] = _density(s["nx"], s["ny"], k)
        rhos.append(r)
    a, b = lbm.Lattice(specs), lbm.Lattice(specs)
    for k in range(len(specs)):
        a.set_density(rhos[k], inst=k)
        b.set_density(rhos[k], inst=k, sync=False)
    b.sync()
    for lat in (a, b):
        lat.step(57)
    outs = [{q: _pinned((s["ny"], s["nx"])) for q in ("rho", "ux", "uy")} for s in specs]
    for k in range(len(specs)):
        b.fields(k, out=outs[k], sync=False)
    b.sync()
    for k in range(len(specs)):
        ref = a.fields(k)
        for q in ("rho", "ux", "uy"):
            assert np.array_equal(ref[q], outs[k][q]), (k, q)
        assert np.array_equal(a.populations(k), b.populations(k)), k


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_batch_calls_match_per_instance(cuda, prec):
    specs = _batch(prec)
    a, b = lbm.Lattice(specs), lbm.Lattice(specs)
    flat = _pinned((b.total_nodes,))
    for k, r in enumerate(b.split(flat)):
        r[:] = _density(specs[k]["nx"], specs[k]["ny"], k)
    for k in range(len(specs)):
        a.set_density(b.split(flat)[k].copy(), inst=k)
    b.set_density_all(flat)
    b.sync()
    for lat in (a, b):
        lat.step(33)
    out = {q: _pinned((b.total_nodes,)) for q in ("rho", "ux", "uy")}
    b.fields_all(out)
    b.sync()
    for k in range(len(specs)):
        ref = a.fields(k)
        for q in ("rho", "ux", "uy"):
            assert np.array_equal(ref[q], b.split(out[q])[k]), (k, q)
        assert np.array_equal(a.populations(k), b.populations(k)), k
