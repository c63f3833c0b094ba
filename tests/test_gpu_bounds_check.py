"""The checked build (liblbm_check.so, compiled with -DLBM_BOUNDS_CHECK):
every global and shared-memory index of the step kernels is tested against
its buffer, and a bad one latches an error (LBM_ERR_STATE at the next
synchronising call) instead of an access.  On tiny, odd and ragged lattices,
one-row segments and every pipeline, the checked build must report no bad
index and give the populations of the normal build bit for bit.  The
checked library runs in a child process (the library is loaded once per
process)."""
import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)

# (nx, ny, precision, launch, parameter overrides, solid pattern)
CASES = [
    (8, 8, "fp32", {}, {}, "flat"),
    (8, 8, "fp64", {}, {}, "flat"),
    (9, 7, "fp32", dict(h=1), {}, "flat"),
    (9, 7, "fp32_f64", dict(h=1), {}, "flat"),
    (33, 12, "fp32", dict(h=3, bx=64), {}, "flat"),
    (61, 9, "fp64", dict(stages=3, h=1), {}, "flat"),
    (33, 12, "fp32", dict(stages=1, bx=32), {}, "flat"),
    (36, 20, "fp32", dict(stages=8, bx=32, h=5), {}, "flat"),
    (61, 13, "fp32", dict(persistent=True, h=2), {}, "flat"),
    (33, 12, "fp64", dict(persistent=True, stages=1, h=3), {}, "flat"),
    (38, 24, "fp32", dict(h=3), dict(wall="bb", ghost="mean"), "pillars"),
    (9, 7, "fp32", dict(h=1), dict(ghost="mirror"), "flat"),
    (36, 20, "fp32", dict(stages=4, h=3), {}, "flat"),
    (68, 9, "fp32", dict(stages=4, h=1, bx=64), {}, "flat"),
    (12, 10, "fp32", dict(stages=4, h=2), dict(ghost="mirror"), "flat"),
    (40, 24, "fp32", dict(stages=4, h=5), dict(wall="bb", ghost="mean"), "pillars"),
]
STEPS = 40


def _run_all(out_path):
    import paper_1410_2569_gb300 as lbm
    from paper_1410_2569_gb300 import inputs
    res = {}
    for k, (nx, ny, prec, launch, over, pat) in enumerate(CASES):
        solid = (inputs.pillars(nx, ny, height=6, width=4, gap=3) if pat == "pillars"
                 else inputs.flat_walls(nx, ny))
        lat = lbm.Lattice.single(nx, ny, lbm.default_params(prec=prec, **over), solid,
                                 "modified", inputs.wall_gw(solid, 0.1))
        if launch:
            lat.set_launch(**launch)
        if pat == "pillars":  # resting on the pillar tops (rows up to 6 are solid)
            lat.init_droplet(nx / 2, 16.0, 6.0, 2.0)
        else:
            lat.init_droplet(nx / 2, 0.5, min(nx, ny) / 3, 2.0)
        lat.step(STEPS)
        status = "ok"
        try:
            lat.sync()
        except lbm.LbmError as e:
            status = str(e)
        res[k] = dict(status=status, f=lat.populations().tolist())
        lat.close()
    with open(out_path, "w") as fh:
        json.dump(res, fh)


def test_checked_build_reports_nothing_and_matches(cuda, tmp_path):
    from paper_1410_2569_gb300 import build
    path = build.LIB_CHECK
    assert os.path.exists(path), "liblbm_check.so is built with liblbm.so"
    normal = tmp_path / "normal.json"
    checked = tmp_path / "checked.json"
    _run_all(str(normal))
    env = dict(os.environ, LBM_LIBRARY=path)
    code = ("import sys; sys.path[:0] = [%r, %r]; import test_gpu_bounds_check as t; "
            "t._run_all(%r)" % (ROOT, HERE, str(checked)))
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=600)
    assert r.returncode == 0, r.stderr[-2000:]
    a = json.load(open(normal))
    b = json.load(open(checked))
    for k in range(len(CASES)):
        assert b[str(k)]["status"] == "ok", (CASES[k], b[str(k)]["status"])
        assert a[str(k)]["status"] == "ok", (CASES[k], a[str(k)]["status"])
        assert np.array_equal(np.array(a[str(k)]["f"]), np.array(b[str(k)]["f"])), CASES[k]


def test_checked_build_is_the_checked_one(cuda, tmp_path):
    """The child really loads liblbm_check.so (its path in /proc/self/maps)."""
    from paper_1410_2569_gb300 import build
    env = dict(os.environ, LBM_LIBRARY=build.LIB_CHECK)
    code = ("import sys; sys.path.insert(0, %r); import paper_1410_2569_gb300 as lbm; lbm.load(); "
            "print(any('liblbm_check.so' in ln for ln in open('/proc/self/maps')))" % ROOT)
    r = subprocess.run([sys.executable, "-c", code], env=env, capture_output=True, text=True,
                       timeout=120)
    assert r.returncode == 0 and r.stdout.strip() == "True", (r.stdout, r.stderr[-500:])
