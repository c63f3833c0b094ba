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


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
def test_pipelined_batch_iterations(cuda, prec):
    """Uploads, steps and read-backs of several iterations queued back to
    back with one synchronisation (the copies run on the context's copy
    streams beside the steps) give what one synchronised iteration at a
    time gives; each iteration starts from densities of its own."""
    specs = _batch(prec)
    a, b = lbm.Lattice(specs), lbm.Lattice(specs)
    total = b.total_nodes
    iters = 3
    rho_in = []
    for it in range(iters):
        r = _pinned((total,))
        for k, v in enumerate(b.split(r)):
            v[:] = _density(specs[k]["nx"], specs[k]["ny"], k + it)
        rho_in.append(r)
    outs = [{q: _pinned((total,)) for q in ("rho", "ux", "uy")} for _ in range(iters)]
    for it in range(iters):
        b.set_density_all(rho_in[it])
        b.step(21 + it)
        b.fields_all(outs[it])
    b.sync()
    for it in range(iters):
        ref = {q: _pinned((total,)) for q in ("rho", "ux", "uy")}
        a.set_density_all(rho_in[it])
        a.sync()
        a.step(21 + it)
        a.fields_all(ref)
        a.sync()
        for q in ("rho", "ux", "uy"):
            assert np.array_equal(ref[q], outs[it][q]), (it, q)
    assert np.array_equal(a.populations(2), b.populations(2))


def test_batch_calls_interleaved_with_per_instance_calls(cuda):
    """A per-instance read-back queued right after a batch read-back reuses
    the scratch fields only after the batch copies have left them."""
    specs = _batch("fp32")
    lat = lbm.Lattice(specs)
    total = lat.total_nodes
    flat = _pinned((total,))
    for k, v in enumerate(lat.split(flat)):
        v[:] = _density(specs[k]["nx"], specs[k]["ny"], k)
    lat.set_density_all(flat)
    lat.step(17)
    out = {q: _pinned((total,)) for q in ("rho", "ux", "uy")}
    lat.fields_all(out)
    one = {q: _pinned((specs[3]["ny"], specs[3]["nx"])) for q in ("rho", "ux", "uy")}
    lat.fields(3, out=one, sync=False)
    lat.sync()
    for k in range(len(specs)):
        ref = lat.fields(k)
        for q in ("rho", "ux", "uy"):
            assert np.array_equal(lat.split(out[q])[k], ref[q]), (k, q)
    for q in ("rho", "ux", "uy"):
        assert np.array_equal(lat.split(out[q])[3], one[q]), q


def test_batch_density_from_device(cuda):
    """A device density source is read in place, in stream order."""
    specs = _batch("fp32")
    a, b = lbm.Lattice(specs), lbm.Lattice(specs)
    flat = _pinned((a.total_nodes,))
    for k, v in enumerate(a.split(flat)):
        v[:] = _density(specs[k]["nx"], specs[k]["ny"], k)
    a.set_density_all(flat)
    dev = torch.from_numpy(flat).cuda()
    torch.cuda.synchronize()
    b.set_density_all(dev)
    for lat in (a, b):
        lat.step(9)
        lat.sync()
    for k in range(len(specs)):
        assert np.array_equal(a.populations(k), b.populations(k)), k
