"""Batches mixing parameter sets: instances that differ only in viscosity
share one step launch, other differences split the step into one launch per
parameter set.  Either way every instance must evolve bit for bit as it does
alone, in every step pipeline, including the two-rows-per-lane warp strips on
bounce-back pillars (non-plain rows everywhere) with odd segment heights."""
import numpy as np
import pytest

import paper_1410_2569_gb300 as lbm
from helpers import gpu_params, run_gpu
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu

# tau_nu,V != tau_nu,L switches on the density-dependent viscosity
RATIO1 = dict(tau_nu_L=1.1, tau_nu_V=1.1)
RATIO2 = dict(tau_nu_L=1.1, tau_nu_V=1.7)


def _mixed_specs(prec, w4=False):
    # two viscosity ratios (same launch), and a different sigma (own launch);
    # w4: every width a multiple of 4 (the FP32 column-pair strips apply)
    ratio1, ratio10, other = RATIO1, RATIO2, dict(sigma=0.1)
    widths = (96, 72, 64, 36, 132) if w4 else (96, 70, 64, 33, 130)
    specs = []
    for (fsi, gw, ny, over), nx in zip([("modified", 0.2, 48, ratio1),
                                        ("density", 0.05, 41, ratio10),
                                        ("psi", -0.9, 40, other),
                                        ("modified", -0.1, 27, ratio10),
                                        ("density", -0.05, 36, ratio1)], widths):
        specs.append(dict(nx=nx, ny=ny, params=gpu_params(prec=prec, **over),
                          solid=inputs.flat_walls(nx, ny), fsi=fsi, gw=gw,
                          drop=(nx / 2, 0.5, ny / 3, 3.0), over=over))
    return specs


def _run(specs, steps, launch=None):
    b = lbm.Lattice([{k: v for k, v in s.items() if k not in ("drop", "over")} for s in specs])
    if launch:
        b.set_launch(**launch)
    for i, s in enumerate(specs):
        b.init_droplet(*s["drop"], inst=i)
    b.step(steps)
    return b


@pytest.mark.parametrize("prec", ["fp32", "fp64"])
@pytest.mark.parametrize("launch", [None, dict(stages=3), dict(stages=1), dict(stages=2, h=5),
                                    dict(graph=True)])
def test_mixed_batch_matches_instances_alone(cuda, prec, launch):
    specs = _mixed_specs(prec)
    b = _run(specs, 120, launch)
    for i, s in enumerate(specs):
        alone = run_gpu(s["nx"], s["ny"], 120, s["fsi"], s["gw"], s["solid"], s["drop"],
                        launch=dict(stages=1), prec=prec, **s["over"])
        assert np.array_equal(b.populations(i), alone.populations()), (i, launch)


@pytest.mark.parametrize("launch", [None, dict(stages=4, h=5), dict(stages=4, bx=64, h=3),
                                    dict(stages=4, graph=True)])
def test_mixed_batch_column_pairs(cuda, launch):
    """The column-pair strips on a batch of two parameter classes and two
    viscosity ratios, instance by instance against block rows alone."""
    specs = _mixed_specs("fp32", w4=True)
    b = _run(specs, 120, launch)
    assert b.launch()["pipeline"] == 4
    for i, s in enumerate(specs):
        alone = run_gpu(s["nx"], s["ny"], 120, s["fsi"], s["gw"], s["solid"], s["drop"],
                        launch=dict(stages=1), prec="fp32", **s["over"])
        assert np.array_equal(b.populations(i), alone.populations()), (i, launch)


def test_persistent_needs_one_parameter_set(cuda):
    specs = _mixed_specs("fp32")
    b = lbm.Lattice([{k: v for k, v in s.items() if k not in ("drop", "over")} for s in specs])
    with pytest.raises(lbm.LbmError):
        b.set_launch(stages=1, persistent=True)
    # viscosity alone does not split the batch: persistent is accepted
    same = [s for s in specs if "sigma" not in s["over"]]
    c = lbm.Lattice([{k: v for k, v in s.items() if k not in ("drop", "over")} for s in same])
    c.set_launch(stages=1, persistent=True)


@pytest.mark.parametrize("ghost", ["skip", "mean"])
@pytest.mark.parametrize("launch", [dict(stages=2), dict(stages=2, bx=64, h=7),
                                    dict(stages=2, bx=256, h=3), dict(stages=3, h=9),
                                    dict(stages=8, bx=64, h=5)])
def test_pair_strips_on_pillars_bitwise(cuda, launch, ghost):
    nx, ny = 92, 61
    solid = inputs.pillars(nx, ny, height=10, width=6, gap=3)
    drop = (45.0, 30.0, 15.0, 2.0)
    kw = dict(prec="fp32", wall="bb", ghost=ghost, **RATIO2)
    a = run_gpu(nx, ny, 300, "modified", 0.3, solid, drop, launch=dict(stages=1), **kw)
    b = run_gpu(nx, ny, 300, "modified", 0.3, solid, drop, launch=launch, **kw)
    assert np.array_equal(a.populations(), b.populations())
