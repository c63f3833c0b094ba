"""FP32 shifted storage against the FP64 oracle, batched uneven instances,
the persistent and CUDA-graph launch modes, and device-side error latching."""
import ctypes

import numpy as np
import pytest

import paper_1410_2569_gb300 as lbm
from helpers import gpu_params, run_gpu, run_oracle
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("prec", ["fp32", "fp32_f64"])
@pytest.mark.parametrize("fsi,gw", [("density", 0.07), ("psi", 1.0), ("modified", 0.1)])
def test_fp32_density_within_1e4_of_fp64_oracle(cuda, prec, fsi, gw):
    nx, ny, steps = 100, 60, 1000
    solid = inputs.flat_walls(nx, ny)
    drop = (50.0, 0.5, 20.0, 2.0)
    o = run_oracle(nx, ny, steps, fsi, gw, solid, drop)
    g = run_gpu(nx, ny, steps, fsi, gw, solid, drop, prec=prec)
    fo, fg = o.fields(), g.fields()
    fluid = solid == 0
    err = np.max(np.abs(fg["rho"][fluid] - fo["rho"][fluid]) / fo["rho"][fluid])
    assert err <= 1e-4, err
    du = max(np.max(np.abs(fg["ux"] - fo["ux"])), np.max(np.abs(fg["uy"] - fo["uy"])))
    assert du <= 1e-4, du


def _batch_specs(prec="fp64"):
    specs = []
    for k, (fsi, gw, nx, ny) in enumerate([("density", 0.1, 64, 40), ("psi", -1.0, 130, 48),
                                           ("modified", 0.25, 96, 70), ("modified", -0.1, 33, 20),
                                           ("density", -0.05, 257, 36)]):
        specs.append(dict(nx=nx, ny=ny, params=gpu_params(prec=prec), solid=inputs.flat_walls(nx, ny),
                          fsi=fsi, gw=gw, drop=(nx / 2, 0.5, ny / 3, 2.0)))
    return specs


def _run_batch(specs, steps, launch=None):
    b = lbm.Lattice([{k: v for k, v in s.items() if k != "drop"} for s in specs])
    if launch:
        b.set_launch(**launch)
    for i, s in enumerate(specs):
        b.init_droplet(*s["drop"], inst=i)
    b.step(steps)
    return b


def test_batch_matches_single_instances_bitwise(cuda):
    specs = _batch_specs()
    b = _run_batch(specs, 150)
    for i, s in enumerate(specs):
        alone = run_gpu(s["nx"], s["ny"], 150, s["fsi"], s["gw"], s["solid"], s["drop"])
        assert np.array_equal(b.populations(i), alone.populations()), i


def test_batch_matches_oracle(cuda):
    specs = _batch_specs()
    b = _run_batch(specs, 200)
    for i, s in enumerate(specs):
        o = run_oracle(s["nx"], s["ny"], 200, s["fsi"], s["gw"], s["solid"], s["drop"])
        fluid = s["solid"] == 0
        gr, orr = b.fields(i)["rho"], o.fields()["rho"]
        assert np.max(np.abs(gr[fluid] - orr[fluid]) / orr[fluid]) <= 1e-10, i


@pytest.mark.parametrize("launch", [dict(persistent=True), dict(graph=True),
                                    dict(bx=64, h=9, persistent=True), dict(stages=2),
                                    dict(stages=2, bx=64, h=11), dict(stages=2, graph=True),
                                    dict(stages=3), dict(stages=3, bx=96, h=7),
                                    dict(stages=2, bx=256, h=1), dict(stages=2, bx=32, h=4)])
def test_launch_modes_bitwise(cuda, launch):
    specs = _batch_specs("fp32")
    ref = _run_batch(specs, 120)
    got = _run_batch(specs, 120, launch)
    for i in range(len(specs)):
        assert np.array_equal(got.populations(i), ref.populations(i)), (i, launch)


def test_graph_replay_advances_time(cuda):
    specs = _batch_specs("fp32")
    a = _run_batch(specs, 0, dict(graph=True))
    for _ in range(3):
        a.step(40)
    b = _run_batch(specs, 120)
    assert a.t == 120
    for i in range(len(specs)):
        assert np.array_equal(a.populations(i), b.populations(i))


def test_nonfinite_is_latched_and_context_recovers(cuda):
    # tau_nu = 0.6 from a width-2 interface diverges within a few steps
    nx, ny = 200, 100
    p = gpu_params(tau_nu_L=0.6, tau_nu_V=0.6)
    lat = lbm.Lattice.single(nx, ny, p, inputs.flat_walls(nx, ny), "density", -0.14)
    lat.init_droplet(nx / 2, 0.5, 25.0, 2.0)
    lat.step(50)
    with pytest.raises(lbm.LbmError) as ei:
        lat.sync()
    assert ei.value.status == 4  # LBM_ERR_NONFINITE
    # a wider interface is stable; the context stays usable
    lat2 = lbm.Lattice.single(nx, ny, p, inputs.flat_walls(nx, ny), "density", -0.14)
    lat2.init_droplet(nx / 2, 0.5, 25.0, 4.0)
    lat2.step(50)
    lat2.sync()


def test_bounded_wait_gives_up(cuda):
    L = lbm.load()
    st = L.lbm_selftest_wait_timeout(None, 0.05)
    assert st == 5, lbm._lib.STATUS.get(st)  # LBM_ERR_TIMEOUT
    # the device is still usable afterwards
    g = run_gpu(40, 20, 10, "modified", 0.1)
    g.sync()


def _batch_specs_w4(prec="fp32"):
    # every width a multiple of 4: the TMA row pipeline applies
    specs = []
    for fsi, gw, nx, ny in [("density", 0.1, 64, 40), ("psi", -1.0, 132, 48),
                            ("modified", 0.25, 96, 70), ("modified", -0.1, 36, 20),
                            ("density", -0.05, 252, 36)]:
        specs.append(dict(nx=nx, ny=ny, params=gpu_params(prec=prec),
                          solid=inputs.flat_walls(nx, ny), fsi=fsi, gw=gw,
                          drop=(nx / 2, 0.5, ny / 3, 2.0)))
    return specs


@pytest.mark.parametrize("prec", ["fp32", "fp32_f64"])
@pytest.mark.parametrize("launch", [dict(stages=8), dict(stages=16, bx=128),
                                    dict(stages=8, bx=32, h=5), dict(stages=8, persistent=True),
                                    dict(stages=8, bx=64, h=7, persistent=True),
                                    dict(stages=2), dict(stages=2, bx=256, h=3), dict(stages=2, bx=32, h=2),
                                    dict(stages=3), dict(stages=3, bx=64, h=5)])
def test_tma_pipeline_bitwise_equal_to_register_pipeline(cuda, prec, launch):
    specs = _batch_specs_w4(prec)
    ref = _run_batch(specs, 130, dict(stages=1))
    got = _run_batch(specs, 130, launch)
    for i in range(len(specs)):
        assert np.array_equal(got.populations(i), ref.populations(i)), (i, launch)


@pytest.mark.parametrize("launch", [dict(), dict(stages=4), dict(stages=4, h=1),
                                    dict(stages=4, bx=64, h=5), dict(stages=4, bx=256, h=3),
                                    dict(stages=4, bx=32, h=2), dict(stages=4, h=7, graph=True),
                                    dict(persistent=True), dict(persistent=True, h=5),
                                    dict(persistent=True, bx=128, h=2),
                                    dict(stages=4, persistent=True, graph=True)])
def test_column_pair_strips_bitwise(cuda, launch):
    """FP32 warp strips with two columns per lane (every width a multiple of
    4; the automatic choice there), launched per step or all steps in one
    persistent launch, against the block rows, bit for bit, on ragged strips
    (36 .. 252 columns) and segment heights 1 .. 7."""
    specs = _batch_specs_w4("fp32")
    ref = _run_batch(specs, 130, dict(stages=1))
    got = _run_batch(specs, 130, launch)
    assert got.launch()["pipeline"] == 4
    for i in range(len(specs)):
        assert np.array_equal(got.populations(i), ref.populations(i)), (i, launch)


@pytest.mark.parametrize("launch", [dict(), dict(persistent=True)])
def test_column_pair_strips_narrow_and_exact_widths(cuda, launch):
    """Widths at the edges of the column-pair geometry: 4 columns (every
    16-byte piece of a row buffer wraps around the lattice many times, the
    lanes past the lattice hold repeated columns), 8, and strips that end
    exactly at 60 and 64 columns, bit for bit against the block rows."""
    specs = []
    for fsi, gw, nx, ny in [("modified", 0.1, 4, 9), ("density", -0.05, 8, 12),
                            ("psi", 0.75, 60, 20), ("modified", -0.1, 64, 18),
                            ("density", 0.07, 120, 23)]:
        specs.append(dict(nx=nx, ny=ny, params=gpu_params(prec="fp32"),
                          solid=inputs.flat_walls(nx, ny), fsi=fsi, gw=gw,
                          drop=(nx / 2, 0.5, min(nx, ny) / 3, 2.0)))
    ref = _run_batch(specs, 90, dict(stages=1))
    got = _run_batch(specs, 90, launch)
    assert got.launch()["pipeline"] == 4
    for i in range(len(specs)):
        assert np.array_equal(got.populations(i), ref.populations(i)), (i, launch)


def test_fp64_automatic_pipeline(cuda):
    """FP64 with the automatic pipeline: block rows for a batch of 1.5 waves
    of them or more (the 72 lattices of 400x200: 288 block rows), warp strips
    for a small one; the two give the same populations."""
    specs = []
    for k in range(72):
        nx, ny = 400, 200
        specs.append(dict(nx=nx, ny=ny, params=gpu_params(prec="fp64"),
                          solid=inputs.flat_walls(nx, ny), fsi=("density", "psi", "modified")[k % 3],
                          gw=0.05 * (k % 5 - 2), drop=(nx / 2, 0.5, 50.0, 4.0)))
    big = _run_batch(specs, 20)
    assert big.launch()["pipeline"] == 1
    strips = _run_batch(specs, 20, dict(stages=3))
    for i in (0, 35, 71):
        assert np.array_equal(big.populations(i), strips.populations(i)), i
    small = _run_batch(specs[:3], 2)
    assert small.launch()["pipeline"] == 3


def test_column_pairs_need_widths_multiple_of_4(cuda):
    """A batch with a width that is not a multiple of 4 keeps the two-row
    strips, asked for or not."""
    b = _run_batch(_batch_specs("fp32"), 2)
    assert b.launch()["pipeline"] == 2
    b.set_launch(stages=4)
    assert b.launch()["pipeline"] == 2


@pytest.mark.parametrize("ghost", ["skip", "mean"])
def test_column_pair_strips_pillars(cuda, ghost):
    nx, ny = 92, 60
    solid = inputs.pillars(nx, ny, height=10, width=6, gap=3)
    drop = (45.0, 30.0, 15.0, 2.0)
    a = run_gpu(nx, ny, 300, "modified", 0.3, solid, drop, launch=dict(stages=1), prec="fp32",
                wall="bb", ghost=ghost)
    b = run_gpu(nx, ny, 300, "modified", 0.3, solid, drop, launch=dict(stages=4, h=9),
                prec="fp32", wall="bb", ghost=ghost)
    assert np.array_equal(a.populations(), b.populations())


def test_tma_pipeline_bounce_back_pillars(cuda):
    nx, ny = 92, 60
    solid = inputs.pillars(nx, ny, height=10, width=6, gap=3)
    drop = (45.0, 30.0, 15.0, 2.0)
    a = run_gpu(nx, ny, 300, "modified", 0.3, solid, drop, launch=dict(stages=1), prec="fp32",
                wall="bb", ghost="skip")
    b = run_gpu(nx, ny, 300, "modified", 0.3, solid, drop, launch=dict(stages=8, bx=64, h=9),
                prec="fp32", wall="bb", ghost="skip")
    assert np.array_equal(a.populations(), b.populations())


def test_fp64_warp_strips_bitwise(cuda):
    specs = _batch_specs("fp64")
    ref = _run_batch(specs, 90, dict(stages=1))
    got = _run_batch(specs, 90, dict(stages=2, bx=96, h=13))
    for i in range(len(specs)):
        assert np.array_equal(got.populations(i), ref.populations(i)), i


@pytest.mark.parametrize("prec", ["fp64", "fp32", "fp32_f64"])
@pytest.mark.parametrize("ghost,wall", [("copy", "neq"), ("mirror", "neq"), ("mean", "bb")])
@pytest.mark.parametrize("shape", [dict(h=2), dict(h=3, bx=64), dict()])
def test_persistent_warp_strips_bitwise(cuda, prec, ghost, wall, shape):
    """Warp strips in one persistent launch, each strip starting a step when
    the strips within four nodes of it have finished the previous one, give
    the populations of one launch per step bit for bit.  Short segments make
    every strip wait on many neighbours; the mirror ghost reads deepest."""
    specs = []
    for fsi, gw, nx, ny in [("density", 0.1, 64, 40), ("psi", -1.0, 130, 48),
                            ("modified", 0.25, 96, 70), ("modified", -0.1, 33, 20)]:
        specs.append(dict(nx=nx, ny=ny, params=gpu_params(prec=prec, ghost=ghost, wall=wall),
                          solid=inputs.flat_walls(nx, ny), fsi=fsi, gw=gw,
                          drop=(nx / 2, 0.5, ny / 3, 2.0)))
    ref = _run_batch(specs, 150)
    got = _run_batch(specs, 150, dict(persistent=True, **shape))
    for i in range(len(specs)):
        assert np.array_equal(got.populations(i), ref.populations(i)), (i, prec, ghost, shape)
