"""Checkpoint/resume, the launch-shape autotuner, graph-captured persistent
launches, and the batched workload of 64 uneven lattices."""
import numpy as np
import pytest

import oracle
import paper_1410_2569_gb300 as lbm
from helpers import gpu_params
from paper_1410_2569_gb300 import inputs

pytestmark = pytest.mark.gpu


def _specs(prec, widths=((64, 40), (132, 48), (96, 70), (36, 20), (252, 36))):
    out = []
    for k, (nx, ny) in enumerate(widths):
        fsi = ("density", "psi", "modified")[k % 3]
        gw = {"density": 0.1, "psi": -1.0, "modified": 0.25}[fsi]
        out.append(dict(nx=nx, ny=ny, params=gpu_params(prec=prec), solid=inputs.flat_walls(nx, ny),
                        fsi=fsi, gw=gw, drop=(nx / 2, 0.5, ny / 3, 2.0)))
    return out


def _make(specs, launch=None):
    b = lbm.Lattice([{k: v for k, v in s.items() if k != "drop"} for s in specs])
    if launch:
        b.set_launch(**launch)
    for i, s in enumerate(specs):
        b.init_droplet(*s["drop"], inst=i)
    return b


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_save_load_resume_is_bitwise(cuda, tmp_path, prec):
    specs = _specs(prec)
    a = _make(specs)
    a.step(101)
    path = tmp_path / "state.bin"
    a.save(path)
    a.step(70)
    b = _make(specs)
    b.load(path)
    assert b.t == 101
    b.step(70)
    assert b.t == a.t == 171
    for i in range(len(specs)):
        assert np.array_equal(a.populations(i), b.populations(i)), i


def test_load_rejects_other_lattices(cuda, tmp_path):
    a = _make(_specs("fp32"))
    a.step(3)
    path = tmp_path / "state.bin"
    a.save(path)
    other = _specs("fp32")
    other[2]["gw"] = 0.26
    b = _make(other)
    with pytest.raises(lbm.LbmError) as ei:
        b.load(path)
    assert ei.value.status == 1


def test_autotune_changes_only_the_launch_shape(cuda):
    specs = _specs("fp32", widths=((128, 64), (256, 128), (200, 100)))
    a = _make(specs)
    a.step(40)
    before = [a.populations(i) for i in range(len(specs))]
    best = a.autotune(steps=4)
    assert best["ms_per_step"] > 0 and best["stages"] in (1, 2, 3, 4, 8)
    assert best["persistent"] == a.launch()["persistent"]
    assert a.t == 40
    for i in range(len(specs)):
        assert np.array_equal(a.populations(i), before[i])
    a.step(30)
    ref = _make(specs)
    ref.step(70)
    for i in range(len(specs)):
        assert np.array_equal(a.populations(i), ref.populations(i))


@pytest.mark.parametrize("launch", [dict(stages=1, persistent=True, graph=True),
                                    dict(stages=8, persistent=True, graph=True),
                                    dict(stages=2, persistent=True, graph=True),
                                    dict(stages=3, bx=64, h=5, persistent=True, graph=True),
                                    dict(stages=4, persistent=True, graph=True)])
def test_graph_captured_persistent_launch(cuda, launch):
    specs = _specs("fp32", widths=((64, 40), (132, 48), (96, 70), (36, 20), (252, 36)))
    ref = _make(specs)
    ref.step(240)
    got = _make(specs, launch)
    for _ in range(3):
        got.step(80)  # the second and third calls replay the captured graph
    for i in range(len(specs)):
        assert np.array_equal(got.populations(i), ref.populations(i)), i


@pytest.mark.parametrize("launch", [dict(stages=1, persistent=True, graph=True),
                                    dict(stages=2, persistent=True, graph=True),
                                    dict(stages=4, persistent=True, graph=True)])
def test_batched_uneven_lattices(cuda, launch):
    """64 lattices, widths 128..512 drawn log-uniform from a seed, random
    interaction and G_w, radius 0.25 ny, FP32 populations with compensated
    density; one persistent launch per 100 steps replayed from a CUDA graph
    (block rows with a grid barrier, or warp strips, one row or two
    columns per lane, waiting on their neighbours)."""
    insts = inputs.batch_instances(64, seed=0)
    specs = []
    for d in insts:
        nx, ny = d["nx"], d["ny"]
        specs.append(dict(nx=nx, ny=ny, params=gpu_params(prec="fp32"),
                          solid=inputs.flat_walls(nx, ny), fsi=d["fsi"], gw=d["gw"],
                          drop=(nx / 2, 0.5, d["R"], 2.0)))
    steps = 300
    ref = _make(specs)
    ref.step(steps)
    got = _make(specs, launch)
    for _ in range(steps // 100):
        got.step(100)
    got.sync()
    for i in (0, 17, 40, 63):
        assert np.array_equal(got.populations(i), ref.populations(i)), i
    # sampled lattices against the FP64 oracle
    oracle.set_threads(16)
    for i in (3, 29, 51):
        s = specs[i]
        o = oracle.Lattice(s["nx"], s["ny"], oracle.paper_params(), s["solid"], s["fsi"], s["gw"])
        o.init_droplet(*s["drop"])
        o.step(steps)
        fluid = s["solid"] == 0
        r_o, r_g = o.fields()["rho"], got.fields(i)["rho"]
        assert np.max(np.abs(r_g[fluid] - r_o[fluid]) / r_o[fluid]) <= 1e-4, i
